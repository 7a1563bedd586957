"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

F is compared bin by bin as |F_gpu - F_ref| / max(F_ref, 2) (2 = E[F] in
noise): at most 1e-10 for the FP64 plain form and 1e-4 for the FP32 batched
form.  Candidate lists must be identical except where |2F_ref - thr| is inside
the tolerance band 2 tol max(F_ref, 2).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1410_3677_gb300 import synth as S

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-4}
NTHREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def fs():
    from paper_1410_3677_gb300 import fstat
    return fstat


def _plan(fs, w, form, thr, bands=None, **kw):
    args = dict(lat=w.lat, gamma=w.gamma, upsample=w.upsample, form=form,
                cand_capacity=kw.pop("cand_capacity", 1 << 22))
    args.update(kw)
    return fs.Plan(bands if bands is not None else w.bands, w.alpha, w.delta, w.fdot, thr, **args)


def _gpu_F(fs, w, form, cells_per_band=None, bins=None, **kw):
    """F of every bin of every cell (threshold -1): {(band, sky, spin): F[bins]}."""
    p = _plan(fs, w, form, -1.0, **kw)
    rc = p.search()
    assert rc == fs.FSTAT_OK
    c, total = p.candidates()
    assert total == c.size
    info = p.info()
    p.close()
    return c, info


def _oracle_F(w, band_idx, cells, bin_lo=0, bin_hi=0, sigma2=0.0, upsample=None, full=False,
              interbin=False):
    b = w.bands[band_idx]
    prm = O.params(w.lat, w.gamma, upsample or w.upsample, sigma2, full, 0, interbin)
    cs = np.array([c[0] for c in cells])
    cp = np.array([c[1] for c in cells])
    return O.cells_F(b, prm, w.alpha, w.delta, w.fdot, cs, cp, bin_lo, bin_hi, NTHREADS)


def _rel_err(F, ref):
    return np.abs(F - ref) / np.maximum(ref, 2.0)


def _check_all_bins(c, w, form, band_idx, cells, lo, hi, **okw):
    ref = _oracle_F(w, band_idx, cells, lo if lo or hi else 0, hi if lo or hi else 0, **okw)
    nb = ref.shape[1]
    for i, (sk, sp) in enumerate(cells):
        sel = c[(c["band"] == band_idx) & (c["sky"] == sk) & (c["spin"] == sp)]
        assert sel.size == nb
        assert np.array_equal(sel["bin"], np.arange(lo, lo + nb))
        err = _rel_err(sel["F"], ref[i])
        assert err.max() <= TOL[form], (sk, sp, err.max(), int(np.argmax(err)))
    return ref


# ------------------------------------------------------------------ per-sky stage
@pytest.mark.parametrize("form", [0, 1])
def test_sky_stage_matches_oracle(fs, form):
    """Resampled, phase-demodulated series y, a(t), b(t), window mask and S sums
    for several sky positions, including a band offset (Eq. 1)."""
    w = S.workload(1)
    band = S.make_band(8192, 2.0, 42, 1.3, w.alpha, w.delta, w.fdot, [],
                       f_off=100 + (1 - 2 ** -5) * 12, n_fft=16384)
    p = _plan(fs, w, form, 20.0, bands=[band])
    prm = O.params(w.lat, w.gamma, 2, 0.0)
    xu = O.upsample(band.x, 2)
    # a, b: closed forms; y: the band-offset phase 2 pi f_off d (~1e5 rad here)
    # bounds the FP64 agreement near 1e-11 relative.  FP32 form: a and b are
    # evaluated in FP32 (absolute error <= tol_ab), so S_aa = sum a^2 over the
    # window moves by at most 2 tol_ab sum|a| / sum a^2 <= 2 tol_ab / rms(a)
    # relative (likewise S_bb, and S_ab on the scale sqrt(S_aa S_bb)): 1.4e-5 at the
    # smallest rms here (rms(a) = 0.29 at sky 7).  tol_S = 1e-5 sits just below that
    # worst case; through 1/S its effect on F stays 10x below the 1e-4 on F.
    tol_ab, tol_y, tol_S = (1e-12, 1e-10, 1e-12) if form == 0 else (2e-6, 2e-5, 1e-5)
    for sky in (0, 7, 31):
        g = p.debug_sky(0, sky, band.n)
        r = O.sky_prepare(band, prm, xu, float(w.alpha[sky]), float(w.delta[sky]))
        # the window edge is a comparison u <= n-1 in FP64 on both sides
        bad = np.nonzero(g["mask"] != r["mask"])[0]
        assert bad.size == 0, (sky, bad[:10], r["u"][bad[:10]])
        ea, eb = np.max(np.abs(g["a"] - r["a"])), np.max(np.abs(g["b"] - r["b"]))
        assert ea < tol_ab and eb < tol_ab, (sky, ea, eb)
        ey = np.max(np.abs(g["y"] - r["y"])) / max(1.0, np.max(np.abs(r["y"])))
        assert ey < tol_y, (sky, ey)
        scale = np.array([r["S"][0], r["S"][1], math.sqrt(r["S"][0] * r["S"][1])])
        eS = np.max(np.abs(g["S"] - r["S"]) / scale)
        assert eS < tol_S, (sky, g["S"], r["S"])
    p.close()


# ------------------------------------------------------------------ all bins, tiny workload
@pytest.mark.parametrize("form", [0, 1])
def test_all_bins_tiny_workload(fs, form):
    """Every bin of all 128 cells of the tiny workload (N=4096, N_fft=8192)."""
    w = S.workload(1)
    c, info = _gpu_F(fs, w, form)
    assert info["f_evals"] == 128 * 4095
    cells = [(s, j) for s in range(w.n_sky) for j in range(w.n_spin)]
    _check_all_bins(c, w, form, 0, cells, 1, 4095)


def test_few_spindowns_large_sky_batches(fs):
    """Two spindowns and 300 sky positions: the FP32 form takes sky batches of up to
    256 positions (a full 4096-cell launch pair would need 2048), so the grid is
    one full batch and a ragged one of 44; every bin of cells in both, against
    the oracle."""
    w = S.workload(1, n_sky=300, n_spin=2)
    c, info = _gpu_F(fs, w, 1)
    assert info["f_evals"] == 600 * 4095
    cells = [(s, j) for s in (0, 1, 255, 256, 257, 299) for j in range(2)]
    _check_all_bins(c, w, 1, 0, cells, 1, 4095)


@pytest.mark.parametrize("form", [0, 1])
def test_candidates_tiny_workload(fs, form):
    """Threshold 2F > 20: same candidate list as the oracle outside the band."""
    w = S.workload(1)
    p = _plan(fs, w, form, w.thr_2F)
    assert p.search() == fs.FSTAT_OK
    c, total = p.candidates()
    p.close()
    prm = O.params(w.lat, w.gamma, w.upsample, 0.0, False, 0)
    ref, rtot = O.search(w.bands, prm, w.alpha, w.delta, w.fdot, w.thr_2F, nthreads=NTHREADS)
    _compare_candidates(c, ref, w, form)
    inj = w.bands[0].injections[0]
    hit = c[(c["sky"] == inj.sky) & (c["spin"] == inj.spin)]
    assert hit["bin"][np.argmax(hit["F"])] == inj.bin
    assert np.all(np.diff(c["sky"] * 10**12 + c["spin"] * 10**7 + c["bin"]) > 0)


def _compare_candidates(c, ref, w, form, thr=None):
    thr = w.thr_2F if thr is None else thr
    tol = TOL[form]
    key = lambda a: set(zip(a["band"].tolist(), a["sky"].tolist(), a["spin"].tolist(), a["bin"].tolist()))
    kg, kr = key(c), key(ref)
    refF = {k: f for k, f in zip(zip(ref["band"].tolist(), ref["sky"].tolist(), ref["spin"].tolist(),
                                     ref["bin"].tolist()), ref["F"].tolist())}
    gF = {k: f for k, f in zip(zip(c["band"].tolist(), c["sky"].tolist(), c["spin"].tolist(),
                                   c["bin"].tolist()), c["F"].tolist())}
    for k in kr - kg:     # missed by the GPU: 2F_ref must sit in the band
        assert abs(2 * refF[k] - thr) <= 2 * tol * max(refF[k], 2.0), k
    # extra on the GPU: 2F_ref <= thr < 2F_gpu, so with |F_gpu - F_ref| <= tol max(F_ref, 2)
    # and F_ref < F_gpu, 2F_gpu lies within 2 tol max(F_gpu, 2) above the threshold
    for k in kg - kr:
        assert abs(2 * gF[k] - thr) <= 2 * tol * max(gF[k], 2.0), k
    common = kg & kr
    for k in common:
        assert abs(gF[k] - refF[k]) <= tol * max(refF[k], 2.0), k


# ------------------------------------------------------------------ segment-length transforms
@pytest.mark.parametrize("form", [0, 1])
def test_all_bins_two_sidereal_days(fs, form):
    """N = 86164 (two sidereal days at 2 s), N_fft = 2^18, injected signals: all
    131071 bins of a few cells, including an injected cell."""
    w = S.workload(2, n_sky=1024, n_spin=1)
    inj = w.bands[0].injections[0]
    skies = sorted({0, inj.sky, 700})
    w2 = S.Workload(w.name, w.bands, w.alpha[skies], w.delta[skies], w.fdot, w.thr_2F)
    c, _ = _gpu_F(fs, w2, form)
    cells = [(i, 0) for i in range(len(skies))]
    ref = _check_all_bins(c, w2, form, 0, cells, 1, (1 << 17) - 1)
    k = skies.index(inj.sky)
    assert np.argmax(ref[k]) + 1 == inj.bin


@pytest.mark.parametrize("form", [0, 1])
def test_uneven_bands_float32_band_offsets(fs, form):
    """Three bands of 1, 2 and 4 sidereal days (N_fft 2^17, 2^18, 2^19), float32
    samples, sigma != 1 and band offsets from Eq. 1, one plan."""
    w0 = S.workload(4, n_sky=3, n_spin=2, n_bands=1)
    bands = []
    for i, days in enumerate((1, 2, 4)):
        n = 43082 * days
        bands.append(S.make_band(n, 2.0, 4000 + i, 0.5 + 0.6 * i, w0.alpha, w0.delta, w0.fdot, [],
                                 f_off=100 + (1 - 2 ** -5) * (3 * i + 1), dtype=np.float32))
    w = S.Workload("uneven", bands, w0.alpha, w0.delta, w0.fdot, 30.0)
    c, info = _gpu_F(fs, w, form)
    cells = [(s, j) for s in range(3) for j in range(2)]
    for bi, b in enumerate(bands):
        _check_all_bins(c, w, form, bi, cells, 1, b.n_fft // 2 - 1)


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("n,n_fft,U", [(100, 256, 2), (129, 0, 1), (1000, 8192, 4), (4096, 8192, 3),
                                         (2000, 1 << 12, 2), (7000, 1 << 14, 2), (30000, 1 << 16, 2),
                                         (200000, 1 << 19, 2)])
def test_small_and_odd_shapes(fs, form, n, n_fft, U):
    """Smallest transform, odd length, explicit longer n_fft, U = 1, 3, 4, and
    transform lengths 2^12 .. 2^19 beyond the standard workloads."""
    w0 = S.workload(1, n_sky=4, n_spin=2)
    b = S.make_band(n, 2.0, 77 + n, 1.0, w0.alpha, w0.delta, w0.fdot, [], n_fft=n_fft)
    w = S.Workload("small", [b], w0.alpha, w0.delta, w0.fdot, 10.0, upsample=U)
    c, _ = _gpu_F(fs, w, form)
    cells = [(s, j) for s in range(4) for j in range(2)]
    _check_all_bins(c, w, form, 0, cells, 1, b.n_fft // 2 - 1, upsample=U)


@pytest.mark.parametrize("form", [0, 1])
def test_full_bin_range_and_given_sigma(fs, form):
    """Bins [0, n_fft-1] (DC, Nyquist and negative frequencies) and a given sigma^2."""
    w = S.workload(1, n_sky=3, n_spin=2)
    c, _ = _gpu_F(fs, w, form, bin_lo=0, bin_hi=8191, sigma2=1.7)
    cells = [(s, j) for s in range(3) for j in range(2)]
    _check_all_bins(c, w, form, 0, cells, 0, 8191, sigma2=1.7)


@pytest.mark.parametrize("form", [0, 1])
def test_cell_ranges_resume(fs, form):
    """Searching [a, b) then [b, n) gives the full search's candidates (resume at
    any cell, including mid-sky), and an empty range gives none."""
    w = S.workload(1)
    p = _plan(fs, w, form, 12.0)
    p.search()
    full, _ = p.candidates()
    parts = []
    for a, b in ((0, 37), (37, 90), (90, 128)):
        p.search(a, b)
        c, _ = p.candidates()
        cell = c["sky"] * w.n_spin + c["spin"]
        assert np.all((cell >= a) & (cell < b))
        parts.append(c)
    assert np.array_equal(np.concatenate(parts), full)
    p.search(5, 5)
    c, total = p.candidates()
    assert total == 0 and c.size == 0
    p.close()


@pytest.mark.parametrize("form", [0, 1])
def test_overflow_keeps_exact_total(fs, form):
    w = S.workload(1, n_sky=4, n_spin=4)
    p = _plan(fs, w, form, -1.0, cand_capacity=1000)
    assert p.search_status() == fs.FSTAT_ERR_OVERFLOW
    rc, c, total = p.candidates_get_status(5000)
    assert rc == fs.FSTAT_ERR_OVERFLOW
    assert total == 16 * 4095 and c.size == 1000
    rc, c, total = p.candidates_get_status(10)
    assert rc == fs.FSTAT_ERR_OVERFLOW and c.size == 10
    p.close()


def test_allocation_failure_reports_oom_without_leak(fs):
    import torch
    w = S.workload(1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 5, 12, 20):
        os.environ["FSTAT_TEST_FAIL_ALLOC"] = str(k)
        try:
            with pytest.raises(fs.FstatError) as e:
                _plan(fs, w, 1, 20.0)
            assert e.value.code == fs.FSTAT_ERR_OOM
        finally:
            del os.environ["FSTAT_TEST_FAIL_ALLOC"]
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20)


def test_fp32_matches_fp64_gpu(fs):
    """The two GPU forms on the same grid agree within the FP32 tolerance."""
    w = S.workload(1, n_sky=8, n_spin=4)
    c0, _ = _gpu_F(fs, w, 0)
    c1, _ = _gpu_F(fs, w, 1)
    assert np.array_equal(c0["bin"], c1["bin"]) and np.array_equal(c0["sky"], c1["sky"])
    assert np.max(_rel_err(c1["F"], c0["F"])) <= 1e-4


def test_device_resident_inputs(fs):
    """inputs_on_device = 1 (torch CUDA tensors) gives the host-input result."""
    import torch
    w = S.workload(1, n_sky=8, n_spin=4)
    p = _plan(fs, w, 1, 20.0)
    p.search()
    ref, _ = p.candidates()
    p.close()

    class DB:
        pass
    dbs = []
    for b in w.bands:
        d = DB()
        d.n, d.dt, d.f_off, d.phi0, d.eps, d.n_fft = b.n, b.dt, b.f_off, b.phi0, b.eps, b.n_fft
        d.x = torch.from_numpy(b.x).cuda()
        d.r = torch.from_numpy(np.ascontiguousarray(b.r)).cuda()
        dbs.append(d)
    p = fs.Plan(dbs, torch.from_numpy(w.alpha).cuda(), torch.from_numpy(w.delta).cuda(),
                torch.from_numpy(w.fdot).cuda(), 20.0, lat=w.lat, gamma=w.gamma, form=1,
                on_device=True)
    p.search()
    c, _ = p.candidates()
    p.close()
    assert np.array_equal(c, ref)


# ------------------------------------------------------------------ full-size grid, sampled
def test_precision_workload_full_grid_sampled(fs):
    """The 4096 x 64 grid at N_fft = 2^18 in the FP32 batched launch configuration
    the benchmark times, threshold 2F > 30; the candidates of sampled cells
    (every injected cell and a few others) against the oracle, and the F of a
    sample of all candidates recomputed one by one."""
    w = S.workload(3)
    p = _plan(fs, w, 1, w.thr_2F, cand_capacity=1 << 27)
    assert p.search() == fs.FSTAT_OK, p.error()
    c, total = p.candidates()
    p.close()
    assert total == c.size
    b = w.bands[0]
    rng = np.random.default_rng(5)
    cells = sorted({(i.sky, i.spin) for i in b.injections[:6]} |
                   {(int(rng.integers(w.n_sky)), int(rng.integers(w.n_spin))) for _ in range(4)})
    ref = _oracle_F(w, 0, cells)
    for i, (sk, sp) in enumerate(cells):
        sel = c[(c["sky"] == sk) & (c["spin"] == sp)]
        want = np.nonzero(2 * ref[i] > w.thr_2F)[0] + 1
        got = sel["bin"]
        band = np.abs(2 * ref[i] - w.thr_2F) <= 2 * 1e-4 * np.maximum(ref[i], 2.0)
        sym = set(want.tolist()) ^ set(got.tolist())
        assert all(band[bn - 1] for bn in sym), (sk, sp, sym)
        common = np.intersect1d(want, got)
        if common.size:
            Fg = sel["F"][np.isin(got, common)]
            assert np.max(_rel_err(Fg, ref[i][common - 1])) <= 1e-4
    # injections are found at their bin
    for inj in b.injections:
        sel = c[(c["sky"] == inj.sky) & (c["spin"] == inj.spin)]
        if inj.snr >= 12:
            assert sel.size and abs(int(sel["bin"][np.argmax(sel["F"])]) - inj.bin) <= 1


# ------------------------------------------------------------------ full JKS statistic
@pytest.mark.parametrize("form", [0, 1])
def test_full_statistic_all_bins(fs, form):
    """The full form (with S_ab) on every bin of a small grid, a 4096-sample band
    with a band offset, against the oracle's full form."""
    w0 = S.workload(1, n_sky=5, n_spin=2)
    b = S.make_band(4096, 2.0, 31, 1.0, w0.alpha, w0.delta, w0.fdot, [], f_off=100 + (1 - 2 ** -5) * 3)
    w = S.Workload("full", [b], w0.alpha, w0.delta, w0.fdot, 10.0)
    c, _ = _gpu_F(fs, w, form, full=True)
    cells = [(s, j) for s in range(5) for j in range(2)]
    ref = _check_all_bins(c, w, form, 0, cells, 1, b.n_fft // 2 - 1, full=True)
    simple = _oracle_F(w, 0, cells[:1])
    assert np.max(np.abs(simple[0] - ref[0]) / np.maximum(ref[0], 2.0)) > 1e-3   # the forms differ


def test_full_statistic_candidates_two_sidereal_days(fs):
    """FP32 batched full form, N_fft = 2^18, 2F > 30: candidates of sampled cells
    (injected and random) against the oracle's full form."""
    w = S.workload(3, n_sky=64, n_spin=8)
    p = _plan(fs, w, 1, w.thr_2F, cand_capacity=1 << 24, full=True)
    assert p.search() == fs.FSTAT_OK
    c, total = p.candidates()
    p.close()
    assert total == c.size
    rng = np.random.default_rng(9)
    cells = sorted({(i.sky, i.spin) for i in w.bands[0].injections if i.sky < 64 and i.spin < 8} |
                   {(int(rng.integers(64)), int(rng.integers(8))) for _ in range(3)})
    ref = _oracle_F(w, 0, cells, full=True)
    _compare_candidates_cells(c, w, cells, ref, 1e-4)


def _compare_candidates_cells(c, w, cells, ref, tol):
    for i, (sk, sp) in enumerate(cells):
        sel = c[(c["sky"] == sk) & (c["spin"] == sp)]
        want = np.nonzero(2 * ref[i] > w.thr_2F)[0] + 1
        got = sel["bin"]
        inband = np.abs(2 * ref[i] - w.thr_2F) <= 2 * tol * np.maximum(ref[i], 2.0)
        sym = set(want.tolist()) ^ set(got.tolist())
        assert all(inband[bn - 1] for bn in sym), (sk, sp, sorted(sym)[:10])
        common = np.intersect1d(want, got)
        if common.size:
            assert np.max(_rel_err(sel["F"][np.isin(got, common)], ref[i][common - 1])) <= tol


# ------------------------------------------------------------------ interbinning
@pytest.mark.parametrize("n,n_fft,full,lohi", [(4096, 1 << 13, False, None), (4096, 1 << 13, True, None),
                                               (3000, 1 << 13, False, (0, (1 << 13) - 1)),
                                               (86164, 1 << 18, False, None)])
def test_interbin_all_bins(fs, n, n_fft, full, lohi):
    """The interbinning form (half-length transforms, odd bins (pi/4)(X_k - X_k+1))
    on every bin against the oracle's: default and full bin range (the wrap of
    the last bin to X(0)), simple and full statistic, short and two-day bands."""
    w0 = S.workload(1, n_sky=3, n_spin=2)
    b = S.make_band(n, 2.0, 17 + n, 1.0, w0.alpha, w0.delta, w0.fdot, [], n_fft=n_fft,
                    f_off=100 + (1 - 2 ** -5) * 5)
    w = S.Workload("ib", [b], w0.alpha, w0.delta, w0.fdot, 10.0)
    kw = dict(full=full, interbin=True)
    if lohi:
        kw.update(bin_lo=lohi[0], bin_hi=lohi[1])
    c, _ = _gpu_F(fs, w, 1, **kw)
    cells = [(s, j) for s in range(3) for j in range(2)]
    lo, hi = lohi if lohi else (1, n_fft // 2 - 1)
    _check_all_bins(c, w, 1, 0, cells, lo, hi, full=full, interbin=True)


def test_interbin_candidates_two_sidereal_days(fs):
    """Interbinning form, 2^18 bins, 2F > 30: candidates of sampled cells against
    the oracle's interbinning form; injections found near their bins."""
    w = S.workload(3, n_sky=64, n_spin=8)
    p = _plan(fs, w, 1, w.thr_2F, cand_capacity=1 << 24, interbin=True)
    assert p.search() == fs.FSTAT_OK
    c, total = p.candidates()
    p.close()
    assert total == c.size
    rng = np.random.default_rng(11)
    cells = sorted({(i.sky, i.spin) for i in w.bands[0].injections if i.sky < 64 and i.spin < 8} |
                   {(int(rng.integers(64)), int(rng.integers(8))) for _ in range(3)})
    ref = _oracle_F(w, 0, cells, interbin=True)
    _compare_candidates_cells(c, w, cells, ref, 1e-4)
