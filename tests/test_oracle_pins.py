"""Pins of the FP64 oracle against what mathematics and the paper fix.

Nothing here compares the oracle with itself: transforms against the O(n^2)
definition, Parseval and known spectra; the resampler against interpolation
identities; a(t), b(t) against an independent tensor contraction; the statistic
against the textbook periodogram, closed-form signal recovery, the brute-force
demodulated DFT and the chi-square law of 2F in noise.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_1410_3677_gb300 import synth as S

RNG = np.random.default_rng(12345)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ----------------------------------------------------------------- transforms
def test_brute_dft_known_spectra():
    """The O(n^2) definition itself: a delta has a flat spectrum and a pure
    exponential e^{2 pi i m j/n} has all its weight n at bin m."""
    for n in (1, 5, 16, 30):
        d = np.zeros(n, complex)
        d[0] = 1
        assert np.allclose(O.dft_brute(d), np.ones(n), atol=1e-14)
        for m in range(n):
            e = np.exp(2j * np.pi * m * np.arange(n) / n)
            ref = np.zeros(n, complex)
            ref[m] = n
            assert np.allclose(O.dft_brute(e), ref, atol=1e-11 * n)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 512, 2048])
def test_fft_pow2_matches_definition(n):
    z = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    assert _rel(O.fft(z), O.dft_brute(z)) < 1e-12
    assert _rel(O.fft(z, +1), O.dft_brute(z, +1)) < 1e-12


@pytest.mark.parametrize("n", [3, 5, 6, 7, 12, 100, 1000, 1331])
def test_fft_bluestein_matches_definition(n):
    z = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    assert _rel(O.fft(z), O.dft_brute(z)) < 1e-12
    assert _rel(O.fft(z, +1), O.dft_brute(z, +1)) < 1e-12


def test_fft_parseval_and_inverse():
    n = 1 << 16
    z = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    Z = O.fft(z)
    assert abs(np.sum(np.abs(Z) ** 2) - n * np.sum(np.abs(z) ** 2)) / (n * np.sum(np.abs(z) ** 2)) < 1e-12
    assert _rel(O.fft(Z, +1) / n, z) < 1e-12


@pytest.mark.parametrize("n", [1 << 18, 86164, 43082])
def test_fft_matches_library(n):
    """Cross-check with numpy's pocketfft at the workload lengths (2^18 and the
    two-sidereal-day / one-sidereal-day sample counts, which take Bluestein)."""
    z = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    assert _rel(O.fft(z), np.fft.fft(z)) < 1e-12


# ----------------------------------------------------------------- resampling
@pytest.mark.parametrize("n,U", [(64, 2), (65, 2), (100, 4), (4096, 2)])
def test_upsample_keeps_samples_and_is_bandlimited(n, U):
    x = RNG.standard_normal(n)
    xu = O.upsample(x, U)
    assert np.max(np.abs(xu[::U] - x)) < 1e-12
    # a tone at bin m < n/2 is interpolated by the analytic cosine
    m = n // 3
    j = np.arange(U * n)
    tone = np.cos(2 * np.pi * m * np.arange(n) / n + 0.3)
    assert np.max(np.abs(O.upsample(tone, U) - np.cos(2 * np.pi * m * j / (U * n) + 0.3))) < 1e-11


def test_upsample_nyquist_split():
    """(-1)^k at even n lies on the Nyquist bin; with the bin split between +n/2
    and -n/2 the interpolant is the real cosine cos(pi j / U)."""
    n, U = 64, 2
    x = (-1.0) ** np.arange(n)
    xu = O.upsample(x, U)
    assert np.max(np.abs(xu - np.cos(np.pi * np.arange(U * n) / U))) < 1e-12


def test_keys_interpolation_identities():
    m = 200
    i = np.arange(m, dtype=float)
    q = 0.7 - 0.03 * i + 0.0011 * i * i        # quadratics are reproduced exactly (a = -1/2)
    for p in RNG.uniform(2, m - 3, 50):
        assert abs(O.keys(q, p) - (0.7 - 0.03 * p + 0.0011 * p * p)) < 1e-11
    x = RNG.standard_normal(m)
    for k in (1, 50, 150):
        assert O.keys(x, float(k)) == pytest.approx(x[k], abs=1e-15)
    # the half-way weights of the Catmull-Rom spline are (-1, 9, 9, -1)/16
    e = np.zeros(m)
    for j, wj in zip(range(9, 13), (-1 / 16, 9 / 16, 9 / 16, -1 / 16)):
        e[:] = 0
        e[j] = 1
        assert O.keys(e, 10.5) == pytest.approx(wj, abs=1e-15)
    # periodic indexing at the ends
    assert O.keys(x, 0.0) == pytest.approx(x[0], abs=1e-15)
    e[:] = 0
    e[m - 1] = 1
    assert O.keys(e, 0.5) == pytest.approx(-1 / 16, abs=1e-15)


# ----------------------------------------------------------------- geometry
def test_ab_match_tensor_contraction():
    """The closed-form a(t), b(t) equal the plus/cross responses at psi = 0
    obtained by contracting the detector tensor with the polarisation tensors
    (an independent vector computation in the input generator)."""
    for _ in range(300):
        lat, gam = RNG.uniform(-1.5, 1.5), RNG.uniform(0, 2 * np.pi)
        al, de, lst = RNG.uniform(0, 2 * np.pi), RNG.uniform(-1.5, 1.5), RNG.uniform(0, 2 * np.pi)
        a, b = O.ab(lat, gam, al, de, lst)
        fp, fx = S.antenna_response(lat, gam, lst, al, de, 0.0, 0.0)
        assert a == pytest.approx(float(fp), abs=1e-14)
        assert b == pytest.approx(float(fx), abs=1e-14)


def test_ab_daily_means():
    """Over one sidereal day b has no constant part and a averages to
    (3/4) sin 2gamma cos^2 lat cos^2 delta."""
    lat, gam, al, de = 0.76, 2.03, 1.1, -0.4
    lsts = 2 * np.pi * (np.arange(4096) + 0.5) / 4096
    ab = np.array([O.ab(lat, gam, al, de, s) for s in lsts])
    assert abs(ab[:, 1].mean()) < 1e-14
    assert ab[:, 0].mean() == pytest.approx(0.75 * math.sin(2 * gam) * math.cos(lat) ** 2 * math.cos(de) ** 2, abs=1e-14)


def _band(n=4096, seed=3, **kw):
    w = S.workload(1)
    return S.make_band(n, 2.0, seed, 1.0, w.alpha, w.delta, w.fdot, [], n_fft=S.n_fft_auto(n), **kw), w


def test_geometry_identity_and_constant_delay():
    b, w = _band()
    prm = O.params(w.lat, w.gamma, 2, 1.0)
    b.r = np.zeros_like(b.r)
    xu = O.upsample(b.x, 2)
    p = O.sky_prepare(b, prm, xu, 1.0, 0.3)
    assert np.all(p["mask"]) and np.max(np.abs(p["u"] - np.arange(b.n))) == 0
    assert np.max(np.abs(p["y"] - b.x)) < 1e-12
    # a constant delay d shifts every position by -d/dt exactly
    al, de = 0.4, -0.2
    nh = np.array([math.cos(de) * math.cos(al), math.cos(de) * math.sin(al), math.sin(de)])
    b.r = np.tile(nh * 37.3, (b.n, 1))
    p = O.sky_prepare(b, prm, xu, al, de)
    assert np.max(np.abs(p["u"] - (np.arange(b.n) - 37.3 / 2.0))) < 1e-10
    assert np.array_equal(p["mask"], p["u"] >= 0)


def test_time_inversion_residual_and_delay_bound():
    """With the real ephemeris the detector time t of barycentric sample k obeys
    t + nhat.r(t) = k dt to within the two-step fixed-point error |d'|^2 |d|
    (~1e-8 * 500 s), and |nhat.r| <= 1 AU/c + R_E/c."""
    b, w = _band(n=20000)
    prm = O.params(w.lat, w.gamma, 2, 1.0)
    xu = O.upsample(b.x, 2)
    for al, de in ((0.3, 0.1), (2.0, -1.2), (4.0, 0.9)):
        p = O.sky_prepare(b, prm, xu, al, de)
        nh = np.array([math.cos(de) * math.cos(al), math.cos(de) * math.sin(al), math.sin(de)])
        dk = b.r @ nh
        assert np.max(np.abs(dk)) <= S.AU_LIGHT_S + S.R_EARTH_LIGHT_S + 1e-9
        m = p["mask"]
        t = p["u"][m] * 2.0
        d_t = np.interp(t, np.arange(b.n) * 2.0, dk)
        assert np.max(np.abs(t + d_t - np.arange(b.n)[m] * 2.0)) < 2e-5


def test_S_sums_match_tensor_amplitudes():
    b, w = _band()
    prm = O.params(w.lat, w.gamma, 2, 1.0)
    b.r = np.zeros_like(b.r)
    p = O.sky_prepare(b, prm, O.upsample(b.x, 2), 2.2, 0.5)
    fp, fx = S.antenna_response(w.lat, w.gamma, b.phi0, 2.2, 0.5, 0.0, np.arange(b.n) * 2.0)
    assert p["S"] == pytest.approx([np.sum(fp * fp), np.sum(fx * fx), np.sum(fp * fx)], rel=1e-12)


def test_sigma2_compensated():
    x = RNG.standard_normal(100000) * 3 + 1e3
    assert O.sigma2(x) == pytest.approx(math.fsum(x * x) / x.size, rel=1e-15)


# ----------------------------------------------------------------- statistic
def test_identity_geometry_is_periodogram():
    """r = 0, a = 1, b = 0, fdot = 0: F is the textbook periodogram of the
    zero-padded series |X_l|^2 / (sigma^2 N)."""
    b, w = _band()
    b.r = np.zeros_like(b.r)
    prm = O.params(w.lat, w.gamma, 2, 1.7, False, 1)
    F = O.cells_F(b, prm, w.alpha, w.delta, np.array([0.0]), [0], [0])[0]
    X = np.fft.fft(b.x, b.n_fft)[1:b.n_fft // 2]
    assert _rel(F, np.abs(X) ** 2 / (1.7 * b.n)) < 1e-12


def test_spindown_demodulation_dechirps():
    """A unit chirp cos(2 pi f t + pi fdot t^2) at a bin frequency, with r = 0 and
    a = 1, b = 0, gives F = N/(4 sigma^2) at its bin when fdot matches (up to the
    O(1/cycles) cross term), and loses it when the sign of fdot is wrong."""
    b, w = _band()
    b.r = np.zeros_like(b.r)
    n, nf, fd = b.n, b.n_fft, -1e-7
    t = np.arange(n) * 2.0
    l0 = 2000
    b.x = np.cos(2 * np.pi * (l0 / (nf * 2.0)) * t + np.pi * fd * t * t)
    prm = O.params(w.lat, w.gamma, 2, 1.0, False, 1)
    F = O.cells_F(b, prm, w.alpha, w.delta, np.array([fd, -fd]), [0, 0], [0, 1], l0, l0)[:, 0]
    assert F[0] == pytest.approx(n / 4.0, rel=2e-3)
    assert F[1] < 0.05 * n / 4.0


def _noiseless_injection(f_off=0.0, n=4096):
    w = S.workload(1)
    inj0 = w.bands[0].injections[0]
    inj = S.Injection(sky=inj0.sky, spin=inj0.spin, bin=int(round(0.1 * S.n_fft_auto(n) * 2.0)),
                      snr=20.0,
                      cos_iota=inj0.cos_iota, psi=inj0.psi, phi0=inj0.phi0)
    b = S.make_band(n, 2.0, 1000, 1.0, w.alpha, w.delta, w.fdot, [inj], f_off=f_off,
                    n_fft=S.n_fft_auto(n), noise=False)
    return w, b, inj


def _window_closed_forms(w, b, inj):
    """Closed forms over the samples whose barycentric time lies in [0, (N-1) dt]:
    full form 2F = sum h^2 / sigma^2; the S_ab-free form from the amplitudes."""
    al, de = float(w.alpha[inj.sky]), float(w.delta[inj.sky])
    nh = np.array([math.cos(de) * math.cos(al), math.cos(de) * math.sin(al), math.sin(de)])
    t = np.arange(b.n) * b.dt
    tau = t + b.r @ nh
    win = (tau >= 0) & (tau <= (b.n - 1) * b.dt)
    h, _ = S.signal(inj, al, de, inj.fdot, b.n, b.dt, b.r, b.phi0, b.f_off, b.n_fft, w.lat,
                    w.gamma, inj.h0)
    full = 0.5 * np.sum(h[win] ** 2)
    fp, fx = S.antenna_response(w.lat, w.gamma, b.phi0, al, de, 0.0, t[win])
    Saa, Sbb, Sab = np.sum(fp * fp), np.sum(fx * fx), np.sum(fp * fx)
    ci, c2, s2 = inj.cos_iota, math.cos(2 * inj.psi), math.sin(2 * inj.psi)
    Ap, Ax = inj.h0 * (1 + ci * ci) / 2, inj.h0 * ci
    ca, cb = Ap * c2 + 1j * Ax * s2, Ap * s2 - 1j * Ax * c2
    simp = 0.25 * (abs(ca * Saa + cb * Sab) ** 2 / Saa + abs(ca * Sab + cb * Sbb) ** 2 / Sbb)
    return full, simp


@pytest.mark.parametrize("f_off,n", [(0.0, 4096), (100.0 + (1 - 2 ** -5) * 7, 4096),
                                     (100.0 + (1 - 2 ** -5) * 7, 43082)])
def test_noiseless_injection_closed_form(f_off, n):
    """Noiseless JKS signal exactly on (sky, fdot, bin): F equals the closed forms
    (full: half the in-window SNR^2) times the interpolation kernel's coherent gain
    at the signal frequency, within 0.3%.  The
    band offset exercises the f_off phase demodulation (Eq. 1 band numbering);
    the one-sidereal-day case makes the delay vary enough to expose errors in it."""
    w, b, inj = _noiseless_injection(f_off, n)
    full, simp = _window_closed_forms(w, b, inj)
    # the interpolation kernel passes a tone at nu cycles per upsampled sample
    # with the position-averaged coherent gain |E_mu H(nu, mu)|^2
    g = _keys_coherent_gain(inj.bin / (b.n_fft * 2))
    for full_form, ref in ((True, full), (False, simp)):
        prm = O.params(w.lat, w.gamma, 2, 1.0, full_form, 0)
        F = O.cells_F(b, prm, w.alpha, w.delta, w.fdot, [inj.sky], [inj.spin], inj.bin, inj.bin)
        assert float(F[0, 0]) == pytest.approx(ref * g, rel=3e-3)


def test_resampled_matches_brute_force_demodulated_dft():
    """The resampled-FFT statistic against the brute-force demodulated DFT (no
    resampling) on the same window, at every bin within 40 of an injection, with
    and without noise: |dF| <= 1% of the peak F.  The residual is the Keys-on-2x
    amplitude error at 0.1 Hz (about 0.4% of the peak)."""
    w = S.workload(1)
    inj0 = w.bands[0].injections[0]
    for noise in (False, True):
        inj = S.Injection(sky=inj0.sky, spin=inj0.spin, bin=inj0.bin, snr=20.0,
                          cos_iota=inj0.cos_iota, psi=inj0.psi, phi0=inj0.phi0)
        b = S.make_band(4096, 2.0, 1000, 1.0, w.alpha, w.delta, w.fdot, [inj], n_fft=8192,
                        noise=noise)
        al, de = float(w.alpha[inj.sky]), float(w.delta[inj.sky])
        bins = np.arange(inj.bin - 40, inj.bin + 41)
        for full_form in (False, True):
            prm = O.params(w.lat, w.gamma, 2, 1.0, full_form, 0)
            Fr = O.cells_F(b, prm, w.alpha, w.delta, w.fdot, [inj.sky], [inj.spin],
                           int(bins[0]), int(bins[-1]))[0]
            Fe = O.exact_F(b, prm, al, de, float(w.fdot[inj.spin]), 1.0, bins)
            assert np.max(np.abs(Fr - Fe)) < 1e-2 * Fe.max()
            assert abs(Fr[40] - Fe[40]) < 1e-2 * Fe[40]


def _noise_2F(geom, full_form, reps, seed0):
    w = S.workload(1)
    out = []
    for s in range(reps):
        b = S.make_band(4096, 2.0, seed0 + s, 1.0, w.alpha, w.delta, w.fdot, [], n_fft=8192)
        if geom == "identity":
            b.r = np.zeros_like(b.r)
        prm = O.params(w.lat, w.gamma, 2, 1.0, full_form, 0)
        F = O.cells_F(b, prm, w.alpha, w.delta, w.fdot, [s % 32], [s % 4], nthreads=1)[0]
        out.append(2 * F[1::2])     # every second zero-padded bin: the independent ones
    return np.array(out)


def test_noise_identity_geometry_chi2_4():
    """Pure Gaussian noise, integer resampling positions: E[2F] = 4 for both forms,
    and the full form follows chi-square with 4 degrees of freedom."""
    for full_form in (True, False):
        v = _noise_2F("identity", full_form, 100, 9000).ravel()
        assert abs(v.mean() - 4.0) < 4 * v.std() / math.sqrt(v.size)
        if full_form:
            assert stats.kstest(v, "chi2", args=(4,)).pvalue > 1e-3
            assert v.var() == pytest.approx(8.0, rel=0.03)


def _keys_coherent_gain(nu):
    """|E_mu sum_j w_j(mu) e^{2 pi i nu (j - mu)}|^2 for the Catmull-Rom weights
    w_j (Keys 1981, a = -1/2) over taps j = -1..2 and uniform offsets mu."""
    mu = (np.arange(4000) + 0.5) / 4000
    w = np.stack([((-0.5 * mu + 1) * mu - 0.5) * mu, (1.5 * mu - 2.5) * mu * mu + 1,
                  ((-1.5 * mu + 2) * mu + 0.5) * mu, (0.5 * mu - 0.5) * mu * mu])
    h = np.sum(w * np.exp(2j * np.pi * nu * (np.arange(-1, 3)[:, None] - mu[None, :])), axis=0)
    return float(np.abs(h.mean()) ** 2)


def _keys_power_gain(nu):
    """Position-averaged power gain of the Catmull-Rom kernel at nu cycles per
    upsampled sample, from its weights (Keys 1981, a = -1/2)."""
    mu = (np.arange(4000) + 0.5) / 4000
    w = np.stack([((-0.5 * mu + 1) * mu - 0.5) * mu, (1.5 * mu - 2.5) * mu * mu + 1,
                  ((-1.5 * mu + 2) * mu + 0.5) * mu, (0.5 * mu - 0.5) * mu * mu])
    ph = np.exp(2j * np.pi * nu * np.arange(-1, 3))
    return float(np.mean(np.abs(ph @ w) ** 2))


def test_noise_real_geometry_follows_kernel_gain():
    """With the real ephemeris the positions are fractional and white noise is
    filtered by the interpolation kernel, so E[2F] at bin l is 4 G(nu_l),
    nu_l = l/(N_fft U) cycles per upsampled sample; checked per eighth of the band."""
    v = _noise_2F("real", True, 150, 9500)
    nb = v.shape[1]
    for q in range(8):
        blk = v[:, q * nb // 8:(q + 1) * nb // 8]
        ls = 2 * np.arange(q * nb // 8, (q + 1) * nb // 8) + 2
        pred = 4 * np.mean([_keys_power_gain(l / (8192 * 2)) for l in ls[::8]])
        assert abs(blk.mean() - pred) < 4 * blk.std() / math.sqrt(blk.size) + 2e-3


# ----------------------------------------------------------------- search
def test_search_recovers_injection_and_thresholds():
    w = S.workload(1)
    b = w.bands[0]
    inj = b.injections[0]
    prm = O.params(w.lat, w.gamma, 2, 0.0, False, 0)
    c, total = O.search(w.bands, prm, w.alpha, w.delta, w.fdot, w.thr_2F)
    assert total == c.size > 0
    key = np.stack([c["band"], c["sky"], c["spin"], c["bin"]], 1)
    assert np.all(np.diff(key[:, 1] * 10**10 + key[:, 2] * 10**6 + key[:, 3]) > 0)  # sorted
    assert np.all(2 * c["F"] > w.thr_2F)
    hit = c[(c["sky"] == inj.sky) & (c["spin"] == inj.spin)]
    assert hit["bin"][np.argmax(hit["F"])] == inj.bin
    # every (sky, spin) cell agrees with the per-cell F thresholded strictly
    F = O.cells_F(b, prm, w.alpha, w.delta, w.fdot, np.repeat(np.arange(32), 4),
                  np.tile(np.arange(4), 32))
    ref = np.argwhere(2 * F > w.thr_2F)
    assert ref.shape[0] == total
    assert np.array_equal(ref[:, 0], c["sky"] * 4 + c["spin"])
    assert np.array_equal(ref[:, 1] + 1, c["bin"])
    # capacity: count stays exact, the prefix is written
    c2, total2 = O.search(w.bands, prm, w.alpha, w.delta, w.fdot, w.thr_2F, cap=10)
    assert total2 == total and c2.size == 10 and np.array_equal(c2, c[:10])


def test_paper_sizes_golden():
    rows = {}
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_sizes.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                rows[k] = float(v)
    n = int(rows["frame_sidereal_days"] * S.SIDEREAL_DAY_S / rows["sampling_interval_s"])
    assert n == rows["n_samples"]
    r, _, _ = S.ephemeris(1000, 0.5, 1)
    assert r.size * n // 1000 + 2 == rows["ephemeris_doubles"]
    assert 100 + (1 - 2 ** -5) * 0 == rows["f_off_band_0"]
    assert 100 + (1 - 2 ** -5) * 100 == rows["f_off_band_100"]
    assert rows["band_overlap_hz"] == 2 ** -5
    assert S.N_2SID == int(2 * S.SIDEREAL_DAY_S / S.DT)


# ----------------------------------------------------------------- interbinning
# The paper's "Fourier transform interpolation ... twice as long" (Sect. 2) as
# interbinning: a transform of length n_fft / 2, odd bins (pi/4)(X_k - X_{k+1}).
def test_interbin_even_bins_are_the_zero_padded_ones():
    """Even bins of the interbinned statistic are the zero-padded transform's
    (X_{2M}(2k) = X_M(k) for a series of at most M samples): both forms, noise."""
    b, w = _band()
    for full in (False, True):
        F = [O.cells_F(b, O.params(w.lat, w.gamma, 2, 0.0, full, 0, ib), w.alpha, w.delta, w.fdot,
                       [3, 7], [1, 2], 0, b.n_fft - 1) for ib in (False, True)]
        assert _rel(F[1][:, 0::2], F[0][:, 0::2]) < 1e-11
        assert _rel(F[1][:, 1::2], F[0][:, 1::2]) > 1e-3        # odd bins are interpolated


def test_interbin_recovers_a_half_bin_tone():
    """A tone half-way between two Fourier frequencies of the M-point transform
    (r = 0, a = 1, b = 0, no spindown): the interbinned value at the odd bin
    equals the zero-padded one to O(1/M^2); the odd bin below it does not."""
    w = S.workload(1)
    M, k0 = 4096, 1000
    b = S.make_band(M, 2.0, 1, 1.0, w.alpha, w.delta, w.fdot, [], n_fft=2 * M)
    b.r = np.zeros_like(b.r)
    b.x = np.cos(2 * np.pi * (k0 + 0.5) * np.arange(M) / M)
    F = [O.cells_F(b, O.params(w.lat, w.gamma, 2, 1.0, False, 1, ib), w.alpha, w.delta,
                   np.array([0.0]), [0], [0], 0, 2 * M - 1)[0] for ib in (False, True)]
    assert F[0][2 * k0 + 1] == pytest.approx(M / 4, rel=1e-9)      # |M/2|^2 / (sigma^2 M)
    assert F[1][2 * k0 + 1] == pytest.approx(F[0][2 * k0 + 1], rel=1e-5)
    assert F[1][2 * k0 - 1] < 0.2 * F[1][2 * k0 + 1]


def test_interbin_loss_against_zero_padding():
    """The point of the interpolation (Sect. 2: it keeps the loss of signal-to-noise
    small when the signal frequency falls between grid frequencies): for a tone at
    offset d of a Fourier bin of the M-point transform, the largest F over the
    bins, relative to F at the true frequency, follows the closed forms
    sinc^2(pi e) (e the distance to the nearest bin: 1/2 at most without
    interpolation, 1/4 with the transform zero-padded to 2M) and, for the
    interbinned odd bin, (pi/4)^2 (sinc(pi d) + sinc(pi (1 - d)))^2 -- at
    d = 1/4 interbinning keeps 0.889 where zero-padding keeps 0.811 and the plain
    M-point transform 0.811 too; at d = 1/2 they keep 1, 1 and 0.405."""
    w = S.workload(1)
    M, k0 = 4096, 1000

    def sinc(x):
        return 1.0 if x == 0 else math.sin(x) / x
    for d in (0.0, 0.125, 0.25, 0.375, 0.5, 0.625, 0.75):
        b = S.make_band(M, 2.0, 1, 1.0, w.alpha, w.delta, w.fdot, [], n_fft=2 * M)
        b.r = np.zeros_like(b.r)
        b.x = np.cos(2 * np.pi * (k0 + d) * np.arange(M) / M)
        F = [O.cells_F(b, O.params(w.lat, w.gamma, 2, 1.0, False, 1, ib), w.alpha, w.delta,
                       np.array([0.0]), [0], [0], 0, 2 * M - 1)[0] for ib in (False, True)]
        true = M / 4.0                                   # |M/2|^2 / (sigma^2 M)
        zp = F[0][2 * k0 - 2:2 * k0 + 5].max() / true    # zero-padded to 2M
        plain = F[0][2 * k0:2 * k0 + 3:2].max() / true   # the M-point bins alone
        ib = F[1][2 * k0 - 2:2 * k0 + 5].max() / true    # interbinned
        e_plain = min(d, 1 - d)
        e_zp = min(abs(d - h) for h in (0.0, 0.5, 1.0))
        assert plain == pytest.approx(sinc(math.pi * e_plain) ** 2, rel=2e-3), d
        assert zp == pytest.approx(sinc(math.pi * e_zp) ** 2, rel=2e-3), d
        odd = (math.pi / 4) ** 2 * (sinc(math.pi * d) + sinc(math.pi * (1 - d))) ** 2
        assert ib == pytest.approx(max(sinc(math.pi * e_plain) ** 2, odd), rel=5e-3), d
        assert ib >= 0.88 and zp >= 0.81 - 2e-3 and plain >= 0.405 - 2e-3


def test_interbin_noise_level():
    """White noise, n = M (independent Fourier bins), r = 0, a = 1, b = 0: E[2F] is
    2 at even bins (the periodogram) and 2 (pi/4)^2 * 2 = pi^2/4 at odd bins."""
    w = S.workload(1)
    M = 4096
    ev, od = [], []
    for s in range(40):
        b = S.make_band(M, 2.0, 7000 + s, 1.0, w.alpha, w.delta, w.fdot, [], n_fft=2 * M)
        b.r = np.zeros_like(b.r)
        F = O.cells_F(b, O.params(w.lat, w.gamma, 1, 1.0, False, 1, True), w.alpha, w.delta,
                      np.array([0.0]), [0], [0], 0, 2 * M - 1, 1)[0]
        ev.append(2 * F[2:M:2])
        od.append(2 * F[1:M:2])
    ev, od = np.concatenate(ev), np.concatenate(od)
    assert abs(ev.mean() - 2.0) < 4 * ev.std() / math.sqrt(ev.size)
    assert abs(od.mean() - math.pi ** 2 / 4) < 4 * od.std() / math.sqrt(od.size)
