"""Seeded synthetic inputs shaped like the narrow-band segments of the all-sky search.

The search reads three inputs per (band, frame): a narrow-band real time series
sampled at a fixed interval, the detector-to-solar-system-barycentre vector for
every sample plus the sidereal phase at the first sample and the obliquity of the
ecliptic (Sect. 2), and a parameter grid.  No detector data ships here, so this
module draws stand-ins with the same structure:

* ephemeris: a circular 1 AU Earth orbit in the ecliptic, rotated to equatorial
  coordinates by the obliquity, plus the diurnal rotation of a detector at a given
  latitude (light-seconds, one 3-vector per sample);
* noise: white Gaussian noise of a given sigma from a seeded numpy PCG64 stream;
* sky grid: an equal-area Fibonacci sphere in equatorial (alpha, delta);
* spindown grid: uniform and inclusive of both ends;
* injected periodic signals placed exactly on sky and spindown grid points and on
  a zero-padded Fourier bin.

The injections model the detector response with the plus/cross polarisation
tensors contracted against the detector tensor of a right-angle interferometer.
That is the physics of the input, written with vectors; it does not use the
closed-form amplitude-modulation functions of the search.  This module holds none
of the search's own steps (no resampling, demodulation, transform or statistic):
it is imported by the tests, by the oracle's tests and by the benchmark alike.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

C_LIGHT = 299_792_458.0                  # m/s
AU_M = 149_597_870_700.0                 # m
AU_LIGHT_S = AU_M / C_LIGHT              # ~499.00478 s
R_EARTH_M = 6_378_137.0                  # m (equatorial radius)
R_EARTH_LIGHT_S = R_EARTH_M / C_LIGHT    # ~0.021275 s
SIDEREAL_DAY_S = 86_164.0905             # s
OMEGA_R = 2.0 * math.pi / SIDEREAL_DAY_S  # rad/s, Earth's rotation rate
YEAR_S = 365.25636 * 86_400.0            # sidereal year, s
EPS_ECLIPTIC = math.radians(23.439281)   # obliquity of the ecliptic
LAT_DEFAULT = math.radians(43.6)         # detector latitude used by the workloads
GAMMA_DEFAULT = math.radians(116.5)      # arm-bisector orientation, counter-clockwise from East


def n_fft_auto(n: int) -> int:
    """Smallest power of two >= 2n: the 'twice as long' transform of Sect. 2."""
    m = 1
    while m < 2 * n:
        m <<= 1
    return m


# --------------------------------------------------------------------------- ephemeris
def ephemeris(n: int, dt: float, seed: int, lat: float = LAT_DEFAULT,
              eps: float = EPS_ECLIPTIC):
    """Detector position relative to the SSB, per sample, in light-seconds.

    Returns (r[n,3] float64, phi0, eps).  phi0 is the sidereal phase of the
    detector's meridian at the first sample (drawn from the seed), the quantity the
    ephemeris file carries next to the vectors (Sect. 2)."""
    rng = np.random.default_rng(seed)
    orbit_phase0 = rng.uniform(0.0, 2.0 * math.pi)
    phi0 = rng.uniform(0.0, 2.0 * math.pi)
    t = np.arange(n, dtype=np.float64) * dt
    th = orbit_phase0 + 2.0 * math.pi * t / YEAR_S
    ex = AU_LIGHT_S * np.cos(th)
    ey = AU_LIGHT_S * np.sin(th)
    # ecliptic -> equatorial: rotate about x by eps (orbit has no z component)
    orb = np.stack([ex, ey * math.cos(eps), ey * math.sin(eps)], axis=1)
    lst = phi0 + OMEGA_R * t
    rot = R_EARTH_LIGHT_S * np.stack([math.cos(lat) * np.cos(lst),
                                      math.cos(lat) * np.sin(lst),
                                      np.full(n, math.sin(lat))], axis=1)
    return np.ascontiguousarray(orb + rot), phi0, eps


# --------------------------------------------------------------------------- grids
def fibonacci_sky(n_sky: int):
    """Equal-area Fibonacci sphere: (alpha[n], delta[n]) in radians, alpha in [0, 2pi)."""
    i = np.arange(n_sky, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n_sky
    delta = np.arcsin(z)
    golden = math.pi * (3.0 - math.sqrt(5.0))
    alpha = np.mod(i * golden, 2.0 * math.pi)
    return alpha, delta


def spindown_grid(n_spin: int, lo: float, hi: float):
    """Uniform spindown grid, inclusive of both ends (a single value is `lo`)."""
    if n_spin == 1:
        return np.array([lo], dtype=np.float64)
    return np.linspace(lo, hi, n_spin, dtype=np.float64)


# --------------------------------------------------------------------------- signal model
def detector_tensor(lat: float, gamma: float, lst):
    """Detector tensor D = (u u^T - v v^T)/2 in equatorial coordinates for each
    local sidereal time in `lst` (array).  Arms at gamma -/+ 45 degrees,
    counter-clockwise from local East."""
    lst = np.asarray(lst, dtype=np.float64)
    sl, cl = math.sin(lat), math.cos(lat)
    east = np.stack([-np.sin(lst), np.cos(lst), np.zeros_like(lst)], axis=-1)
    north = np.stack([-sl * np.cos(lst), -sl * np.sin(lst), np.full_like(lst, cl)], axis=-1)
    th_u, th_v = gamma - math.pi / 4.0, gamma + math.pi / 4.0
    u = math.cos(th_u) * east + math.sin(th_u) * north
    v = math.cos(th_v) * east + math.sin(th_v) * north
    return 0.5 * (u[..., :, None] * u[..., None, :] - v[..., :, None] * v[..., None, :])


def polarisation_tensors(alpha: float, delta: float, psi: float):
    """Plus/cross tensors for a source at (alpha, delta) with polarisation angle psi.
    p points along increasing alpha, q along decreasing delta (the orientation
    under which psi = 0 gives F_plus = a(t), F_cross = b(t) of the F-statistic)."""
    p = np.array([-math.sin(alpha), math.cos(alpha), 0.0])
    q = np.array([math.sin(delta) * math.cos(alpha), math.sin(delta) * math.sin(alpha),
                  -math.cos(delta)])
    ep = np.outer(p, p) - np.outer(q, q)
    ex = np.outer(p, q) + np.outer(q, p)
    c2, s2 = math.cos(2.0 * psi), math.sin(2.0 * psi)
    return c2 * ep + s2 * ex, -s2 * ep + c2 * ex


def antenna_response(lat, gamma, phi0, alpha, delta, psi, t):
    """(F_plus(t), F_cross(t)) by tensor contraction, t = detector time in s."""
    D = detector_tensor(lat, gamma, phi0 + OMEGA_R * np.asarray(t, dtype=np.float64))
    ep, ex = polarisation_tensors(alpha, delta, psi)
    return np.einsum('...ij,ij->...', D, ep), np.einsum('...ij,ij->...', D, ex)


@dataclasses.dataclass
class Injection:
    sky: int            # index into the sky grid
    spin: int           # index into the spindown grid
    bin: int            # zero-padded Fourier bin of the in-band frequency
    snr: float          # optimal SNR rho = sqrt(sum h^2) / sigma
    cos_iota: float
    psi: float
    phi0: float
    h0: float = 0.0     # filled in by inject()
    f: float = 0.0      # in-band frequency, Hz
    fdot: float = 0.0   # Hz/s
    sumsq: float = 0.0  # sum of h_k^2 over the samples


def signal(inj: Injection, alpha: float, delta: float, fdot: float, n: int, dt: float,
           r, phi0_sid: float, f_off: float, n_fft: int, lat: float, gamma: float,
           h0: float = 1.0):
    """Detector-frame strain of one periodic source at the sample times k*dt.

    Emission (SSB) time tau = t + nhat.r(t); the in-band phase is that of a source
    at f_off + f heterodyned at f_off in detector time:
    2 pi f tau + pi fdot tau^2 + 2 pi f_off (tau - t) + phi0."""
    t = np.arange(n, dtype=np.float64) * dt
    nhat = np.array([math.cos(delta) * math.cos(alpha), math.cos(delta) * math.sin(alpha),
                     math.sin(delta)])
    d = np.asarray(r, dtype=np.float64).reshape(n, 3) @ nhat
    tau = t + d
    f = inj.bin / (n_fft * dt)
    ph = 2.0 * math.pi * (f * tau + 0.5 * fdot * tau * tau + f_off * d) + inj.phi0
    fp, fx = antenna_response(lat, gamma, phi0_sid, alpha, delta, inj.psi, t)
    ci = inj.cos_iota
    return h0 * (fp * 0.5 * (1.0 + ci * ci) * np.cos(ph) + fx * ci * np.sin(ph)), f


# --------------------------------------------------------------------------- band / workload
@dataclasses.dataclass
class Band:
    n: int
    dt: float
    f_off: float
    x: np.ndarray           # float64 (or float32 for the batched multi-band workload)
    r: np.ndarray           # [n,3] float64, light-seconds
    phi0: float
    eps: float
    n_fft: int
    sigma: float
    injections: List[Injection] = dataclasses.field(default_factory=list)


@dataclasses.dataclass
class Workload:
    name: str
    bands: List[Band]
    alpha: np.ndarray
    delta: np.ndarray
    fdot: np.ndarray
    thr_2F: float
    lat: float = LAT_DEFAULT
    gamma: float = GAMMA_DEFAULT
    upsample: int = 2

    @property
    def n_sky(self):
        return int(self.alpha.size)

    @property
    def n_spin(self):
        return int(self.fdot.size)

    def f_evals(self, bin_lo: int = 0, bin_hi: int = 0):
        tot = 0
        for b in self.bands:
            lo, hi = (bin_lo, bin_hi) if (bin_lo or bin_hi) else (1, b.n_fft // 2 - 1)
            tot += self.n_sky * self.n_spin * (hi - lo + 1)
        return tot


def make_band(n: int, dt: float, seed: int, sigma: float, alpha, delta, fdot,
              injections: List[Injection], f_off: float = 0.0, n_fft: int = 0,
              lat: float = LAT_DEFAULT, gamma: float = GAMMA_DEFAULT,
              dtype=np.float64, noise: bool = True) -> Band:
    """One band: seeded noise plus the listed injections (h0 set from each SNR)."""
    if n_fft == 0:
        n_fft = n_fft_auto(n)
    r, phi0, eps = ephemeris(n, dt, seed, lat)
    rng = np.random.default_rng(seed + 7_919)
    x = sigma * rng.standard_normal(n) if noise else np.zeros(n)
    for inj in injections:
        h, f = signal(inj, float(alpha[inj.sky]), float(delta[inj.sky]), float(fdot[inj.spin]),
                      n, dt, r, phi0, f_off, n_fft, lat, gamma, 1.0)
        ss = float(np.dot(h, h))
        inj.h0 = inj.snr * sigma / math.sqrt(ss)
        inj.f, inj.fdot = f, float(fdot[inj.spin])
        inj.sumsq = ss * inj.h0 * inj.h0
        x = x + inj.h0 * h
    return Band(n=n, dt=dt, f_off=f_off, x=np.ascontiguousarray(x.astype(dtype)),
                r=r, phi0=phi0, eps=eps, n_fft=n_fft, sigma=sigma, injections=injections)


def draw_injections(rng, count, n_sky, n_spin, n_fft, dt, snr_lo, snr_hi,
                    f_lo=0.02, f_hi=0.23):
    out = []
    for _ in range(count):
        f = rng.uniform(f_lo, f_hi)
        out.append(Injection(sky=int(rng.integers(n_sky)), spin=int(rng.integers(n_spin)),
                             bin=int(round(f * n_fft * dt)), snr=float(rng.uniform(snr_lo, snr_hi)),
                             cos_iota=float(rng.uniform(-1, 1)),
                             psi=float(rng.uniform(-math.pi / 4, math.pi / 4)),
                             phi0=float(rng.uniform(0, 2 * math.pi))))
    return out


DT = 2.0
N_2SID = 86_164     # two sidereal days at 2 s


def workload(cfg: int, n_sky: Optional[int] = None, n_spin: Optional[int] = None,
             n_bands: Optional[int] = None) -> Workload:
    """The five workloads (seed = workload id * 1000 + band).  n_sky / n_spin /
    n_bands shrink a workload for tests while keeping its data."""
    rng = np.random.default_rng(cfg * 1000 + 999)
    if cfg == 1:
        # tiny: N=4096, N_fft=8192, 32 sky x 4 spindowns, one SNR-20 source at 0.1 Hz
        ns, nsp = n_sky or 32, n_spin or 4
        alpha, delta = fibonacci_sky(ns)
        fdot = spindown_grid(nsp, -3e-9, 0.0) if nsp == 4 else spindown_grid(nsp, -3e-9, 0.0)
        n, nfft = 4096, 8192
        spin_idx = int(np.argmin(np.abs(fdot - (-1e-9))))
        inj = Injection(sky=int(rng.integers(ns)), spin=spin_idx, bin=int(round(0.1 * nfft * DT)),
                        snr=20.0, cos_iota=float(rng.uniform(-1, 1)),
                        psi=float(rng.uniform(-math.pi / 4, math.pi / 4)),
                        phi0=float(rng.uniform(0, 2 * math.pi)))
        b = make_band(n, DT, cfg * 1000, 1.0, alpha, delta, fdot, [inj], n_fft=nfft)
        return Workload("tiny: N=4096 float64, N_fft=8192, 32 sky x 4 spindown", [b],
                        alpha, delta, fdot, 20.0)
    if cfg == 2:
        ns, nsp = n_sky or 1024, n_spin or 1
        alpha, delta = fibonacci_sky(ns)
        fdot = spindown_grid(nsp, -1e-9, -1e-9) if nsp == 1 else spindown_grid(nsp, -1e-8, 0.0)
        nfft = 1 << 18
        injs = draw_injections(rng, 3, ns, nsp, nfft, DT, 8.0, 15.0)
        b = make_band(N_2SID, DT, cfg * 1000, 1.0, alpha, delta, fdot, injs, n_fft=nfft)
        return Workload("segment: N=86164 float64, N_fft=2^18, 1024 sky x 1 spindown", [b],
                        alpha, delta, fdot, 20.0)
    if cfg == 3:
        ns, nsp = n_sky or 4096, n_spin or 64
        alpha, delta = fibonacci_sky(ns)
        fdot = spindown_grid(nsp, -1e-8, 0.0)
        nfft = 1 << 18
        injs = draw_injections(rng, 16, ns, nsp, nfft, DT, 6.0, 20.0)
        b = make_band(N_2SID, DT, cfg * 1000, 1.0, alpha, delta, fdot, injs, n_fft=nfft)
        return Workload("precision: N=86164, N_fft=2^18, 4096 sky x 64 spindown", [b],
                        alpha, delta, fdot, 30.0)
    if cfg == 4:
        ns, nsp, nb = n_sky or 512, n_spin or 16, n_bands or 16
        alpha, delta = fibonacci_sky(ns)
        fdot = spindown_grid(nsp, -1e-8, 0.0)
        bands = []
        for bi in range(nb):
            days = int(rng.integers(1, 5))               # 1..4 sidereal days
            n = 43_082 * days
            sigma = float(rng.uniform(0.5, 2.0))
            nfft = n_fft_auto(n)
            injs = draw_injections(rng, int(rng.integers(0, 5)), ns, nsp, nfft, DT, 6.0, 20.0)
            bands.append(make_band(n, DT, cfg * 1000 + bi, sigma, alpha, delta, fdot, injs,
                                   f_off=100.0 + (1.0 - 2.0 ** -5) * bi, n_fft=nfft,
                                   dtype=np.float32))
        return Workload("batched: 16 bands N=43082..172328 float32, 512 sky x 16 spindown",
                        bands, alpha, delta, fdot, 30.0)
    if cfg == 5:
        ns, nsp = n_sky or 65536, n_spin or 256
        alpha, delta = fibonacci_sky(ns)
        fdot = spindown_grid(nsp, -1e-8, 0.0)
        nfft = 1 << 18
        injs = draw_injections(rng, 64, ns, nsp, nfft, DT, 6.0, 25.0)
        b = make_band(N_2SID, DT, cfg * 1000, 1.0, alpha, delta, fdot, injs, n_fft=nfft)
        return Workload("large: N=86164, N_fft=2^18, 65536 sky x 256 spindown", [b],
                        alpha, delta, fdot, 30.0)
    raise ValueError(f"unknown workload {cfg}")
