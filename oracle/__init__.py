"""FP64 CPU oracle of the all-sky F-statistic search -- test infrastructure.

Only the tests, the package's smoke check and the benchmark's CPU-baseline leg may
import this package.  It wraps the plain C restatement in `fstat_oracle.c`
(compiled with gcc on first use, or by `build()`), which shares no code with the
CUDA path.  Parity: pinned by the `-m "not gpu"` tests in tests/test_oracle_*.py
against brute force, closed forms, the textbook periodogram and chi-square
statistics; no function here is parity-unpinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fstat_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

i64, f64, i32 = C.c_int64, C.c_double, C.c_int
P = C.POINTER


class OrcBand(C.Structure):
    _fields_ = [("n", i64), ("dt", f64), ("f_off", f64), ("x", P(f64)), ("r", P(f64)),
                ("phi0", f64), ("eps", f64), ("n_fft", i64)]


class OrcParams(C.Structure):
    _fields_ = [("lat", f64), ("gamma", f64), ("upsample", i32), ("sigma2", f64),
                ("full_form", i32), ("amp_mode", i32), ("interbin", i32)]


class OrcCandidate(C.Structure):
    _fields_ = [("band", C.c_int32), ("pad_", C.c_int32), ("sky", i64), ("spin", i64),
                ("bin", i64), ("F", f64)]


CAND_DTYPE = np.dtype([("band", np.int32), ("pad_", np.int32), ("sky", np.int64),
                       ("spin", np.int64), ("bin", np.int64), ("F", np.float64)])


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liborc.so with gcc (portable flags only)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "fstat_oracle.h"))):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                                   "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = P(f64)
        L.orc_fft_pow2.argtypes = [dp, i64, i32]
        L.orc_fft_any.argtypes = [dp, i64, i32]
        L.orc_dft_brute.argtypes = [dp, dp, i64, i32]
        L.orc_sigma2.argtypes = [dp, i64]
        L.orc_sigma2.restype = f64
        L.orc_upsample.argtypes = [dp, i64, i32, dp]
        L.orc_keys.argtypes = [dp, i64, f64]
        L.orc_keys.restype = f64
        L.orc_ab.argtypes = [f64, f64, f64, f64, f64, dp, dp]
        L.orc_ab.restype = None
        L.orc_delay_lin.argtypes = [dp, i64, f64]
        L.orc_delay_lin.restype = f64
        L.orc_sky_prepare.argtypes = [P(OrcBand), P(OrcParams), dp, f64, f64, dp, dp, dp,
                                      P(C.c_uint8), dp, dp]
        L.orc_cell_F.argtypes = [P(OrcBand), P(OrcParams), dp, dp, dp, dp, f64, f64, i64, i64,
                                 dp, dp]
        L.orc_exact_F.argtypes = [P(OrcBand), P(OrcParams), f64, f64, f64, f64, P(i64), i64, dp]
        L.orc_search.argtypes = [P(OrcBand), i32, P(OrcParams), i64, dp, dp, i64, dp, f64, i64,
                                 i64, i32, P(OrcCandidate), i64, P(i64)]
        L.orc_search.restype = i64
        L.orc_cells_F.argtypes = [P(OrcBand), P(OrcParams), dp, dp, dp, P(i64), P(i64), i64,
                                  i64, i64, i32, dp]
        L.orc_lattice_spin.argtypes = [dp, f64, i64, i64, dp]
        L.orc_lattice_sky.argtypes = [dp, f64, f64, i64, i64, i64, i64, i32, dp, dp, P(i64), i64,
                                      P(i64)]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(P(f64))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


# ----------------------------------------------------------------------- transforms
def fft(z, sign=-1):
    z = np.ascontiguousarray(z, dtype=np.complex128).copy()
    _check(lib().orc_fft_any(z.ctypes.data_as(P(f64)), z.size, sign), "fft")
    return z


def dft_brute(z, sign=-1):
    z = np.ascontiguousarray(z, dtype=np.complex128)
    out = np.empty_like(z)
    _check(lib().orc_dft_brute(z.ctypes.data_as(P(f64)), out.ctypes.data_as(P(f64)), z.size,
                               sign), "dft_brute")
    return out


# ----------------------------------------------------------------------- steps
def sigma2(x):
    x = _f64(x)
    return lib().orc_sigma2(_dp(x), x.size)


def upsample(x, U):
    x = _f64(x)
    out = np.empty(U * x.size)
    _check(lib().orc_upsample(_dp(x), x.size, U, _dp(out)), "upsample")
    return out


def keys(xu, p):
    xu = _f64(xu)
    return lib().orc_keys(_dp(xu), xu.size, float(p))


def ab(lat, gamma, alpha, delta, lst):
    a, b = f64(), f64()
    lib().orc_ab(lat, gamma, alpha, delta, lst, C.byref(a), C.byref(b))
    return a.value, b.value


def delay_lin(dk, u):
    dk = _f64(dk)
    return lib().orc_delay_lin(_dp(dk), dk.size, float(u))


class _BandRef:
    """Keeps the numpy buffers behind an OrcBand alive."""

    def __init__(self, band):
        self.x = _f64(band.x)
        self.r = _f64(np.asarray(band.r).reshape(-1))
        nfft = int(getattr(band, "n_fft", 0) or 0)
        self.s = OrcBand(int(self.x.size), float(band.dt), float(band.f_off), _dp(self.x),
                         _dp(self.r), float(band.phi0), float(getattr(band, "eps", 0.0)), nfft)


def params(lat, gamma, upsample=2, sigma2=0.0, full_form=False, amp_mode=0, interbin=False):
    return OrcParams(float(lat), float(gamma), int(upsample), float(sigma2), int(full_form),
                     int(amp_mode), int(interbin))


def sky_prepare(band, prm, xu, alpha, delta):
    """Returns dict(y complex[n], a, b, mask bool, u, S=[S_aa, S_bb, S_ab])."""
    br = _BandRef(band)
    n = br.x.size
    y = np.empty(n, np.complex128)
    a, b, u = np.empty(n), np.empty(n), np.empty(n)
    m = np.empty(n, np.uint8)
    S = np.empty(3)
    xu = _f64(xu)
    _check(lib().orc_sky_prepare(C.byref(br.s), C.byref(prm), _dp(xu), alpha, delta,
                                 y.ctypes.data_as(P(f64)), _dp(a), _dp(b),
                                 m.ctypes.data_as(P(C.c_uint8)), _dp(u), _dp(S)), "sky_prepare")
    return dict(y=y, a=a, b=b, mask=m.astype(bool), u=u, S=S)


def cell_F(band, prm, prep, sigma2, fdot, bin_lo, bin_hi):
    br = _BandRef(band)
    F = np.empty(bin_hi - bin_lo + 1)
    y = np.ascontiguousarray(prep["y"], np.complex128)
    _check(lib().orc_cell_F(C.byref(br.s), C.byref(prm), y.ctypes.data_as(P(f64)),
                            _dp(_f64(prep["a"])), _dp(_f64(prep["b"])), _dp(_f64(prep["S"])),
                            sigma2, fdot, bin_lo, bin_hi, _dp(F), None), "cell_F")
    return F


def exact_F(band, prm, alpha, delta, fdot, sigma2, bins):
    br = _BandRef(band)
    bins = np.ascontiguousarray(bins, np.int64)
    F = np.empty(bins.size)
    _check(lib().orc_exact_F(C.byref(br.s), C.byref(prm), alpha, delta, fdot, sigma2,
                             bins.ctypes.data_as(P(i64)), bins.size, _dp(F)), "exact_F")
    return F


def search(bands, prm, alpha, delta, fdot, thr_2F, bin_lo=0, bin_hi=0, nthreads=None,
           cap=None):
    """All cells of all bands; returns (candidates structured array, n_total)."""
    nthreads = nthreads or os.cpu_count() or 1
    refs = [_BandRef(b) for b in bands]
    arr = (OrcBand * len(refs))(*[r.s for r in refs])
    alpha, delta, fdot = _f64(alpha), _f64(delta), _f64(fdot)
    total = i64()
    cap = cap if cap is not None else 1 << 22
    out = np.zeros(cap, CAND_DTYPE)
    nw = lib().orc_search(arr, len(refs), C.byref(prm), alpha.size, _dp(alpha), _dp(delta),
                          fdot.size, _dp(fdot), float(thr_2F), bin_lo, bin_hi, nthreads,
                          out.ctypes.data_as(P(OrcCandidate)), cap, C.byref(total))
    if nw < 0:
        raise RuntimeError(f"oracle search failed with code {nw}")
    return out[:nw].copy(), total.value


def cells_F(band, prm, alpha, delta, fdot, cells_sky, cells_spin, bin_lo=0, bin_hi=0,
            nthreads=None):
    """F over [bin_lo, bin_hi] (default [1, n_fft/2-1]) of the listed cells: [n_cells, nb]."""
    nthreads = nthreads or os.cpu_count() or 1
    br = _BandRef(band)
    nfft = br.s.n_fft
    if nfft == 0:
        nfft = 1
        while nfft < 2 * br.x.size:
            nfft <<= 1
    lo, hi = (bin_lo, bin_hi) if (bin_lo or bin_hi) else (1, nfft // 2 - 1)
    cs = np.ascontiguousarray(cells_sky, np.int64)
    cp = np.ascontiguousarray(cells_spin, np.int64)
    F = np.empty((cs.size, hi - lo + 1))
    alpha, delta, fdot = _f64(alpha), _f64(delta), _f64(fdot)
    _check(lib().orc_cells_F(C.byref(br.s), C.byref(prm), _dp(alpha), _dp(delta), _dp(fdot),
                             cs.ctypes.data_as(P(i64)), cp.ctypes.data_as(P(i64)), cs.size, lo,
                             hi, nthreads, _dp(F)), "cells_F")
    return F


# ----------------------------------------------------------------------- grid from M
def lattice_spin(M, dt, s_lo, s_hi):
    """fdot of the spindown integers s_lo..s_hi (the spindown row of M)."""
    M = _f64(np.asarray(M).reshape(16))
    out = np.empty(s_hi - s_lo + 1)
    _check(lib().orc_lattice_spin(_dp(M), float(dt), s_lo, s_hi, _dp(out)), "lattice_spin")
    return out


def lattice_sky(M, f_ref, eps, n_lo, n_hi, m_lo, m_hi, hemispheres=1):
    """Sky points of the lattice on the sphere: (alpha, delta, nm[:, (hemisphere, n, m)])."""
    M = _f64(np.asarray(M).reshape(16))
    cnt = i64()
    _check(lib().orc_lattice_sky(_dp(M), float(f_ref), float(eps), n_lo, n_hi, m_lo, m_hi,
                                 hemispheres, None, None, None, 0, C.byref(cnt)), "lattice_sky")
    n = cnt.value
    a, d = np.empty(n), np.empty(n)
    nm = np.empty((n, 3), np.int64)
    _check(lib().orc_lattice_sky(_dp(M), float(f_ref), float(eps), n_lo, n_hi, m_lo, m_hi,
                                 hemispheres, _dp(a), _dp(d), nm.ctypes.data_as(P(i64)), n,
                                 C.byref(cnt)), "lattice_sky")
    return a, d, nm
