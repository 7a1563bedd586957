"""ctypes binding of libfstat.so (include/fstat.h): argument marshalling only.

Every step of the search runs in the library's CUDA kernels.  Importing this
module loads the in-tree libfstat.so and raises if it is missing; there is no
fallback of any kind.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfstat.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1410_3677_gb300.build`"
                      " (or __graft_entry__.build())")

_lib = C.CDLL(LIB_PATH)

i64, f64, i32 = C.c_int64, C.c_double, C.c_int
P = C.POINTER

FSTAT_OK, FSTAT_ERR_ARG, FSTAT_ERR_OOM, FSTAT_ERR_CUDA = 0, 1, 2, 3
FSTAT_ERR_OVERFLOW, FSTAT_ERR_TIMEOUT, FSTAT_ERR_STATE, FSTAT_ERR_INTERNAL = 4, 5, 6, 7
FP64_PLAIN, FP32_BATCHED = 0, 1
F_SIMPLE, F_FULL = 0, 1
INTERP_ZEROPAD, INTERP_INTERBIN = 0, 1


class fstat_band(C.Structure):
    _fields_ = [("n", i64), ("dt", f64), ("f_off", f64), ("x", P(f64)), ("x32", P(C.c_float)),
                ("r", P(f64)), ("phi0", f64), ("eps", f64), ("n_fft", i64)]


class fstat_plan_desc(C.Structure):
    _fields_ = [("n_bands", i32), ("bands", P(fstat_band)), ("n_sky", i64), ("alpha", P(f64)),
                ("delta", P(f64)), ("n_spin", i64), ("fdot", P(f64)), ("thr_2F", f64),
                ("bin_lo", i64), ("bin_hi", i64), ("lat", f64), ("gamma", f64),
                ("upsample", i32), ("statistic", i32), ("sigma2", f64), ("form", i32),
                ("interpolation", i32), ("cand_capacity", i64),
                ("cuda_stream", C.c_void_p), ("inputs_on_device", i32)]


class fstat_candidate(C.Structure):
    _fields_ = [("alpha", f64), ("delta", f64), ("freq", f64), ("fdot", f64), ("F", f64),
                ("band", C.c_int32), ("reserved", C.c_int32), ("sky", i64), ("spin", i64),
                ("bin", i64)]


class fstat_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", i64), ("timed_launches", i64),
                ("timed_ms", f64), ("flops_per_launch", f64), ("bytes_per_launch", f64)]


class fstat_tuning(C.Structure):
    _fields_ = [("engine", i32), ("pass2_threads", i32), ("pass2_bulk_copy", i32), ("fused", i32),
                ("cells_per_launch", i64), ("ms_per_cell", f64)]


class fstat_lattice(C.Structure):
    _fields_ = [("M", f64 * 16), ("dt", f64), ("f_ref", f64), ("eps", f64), ("s_lo", i64),
                ("s_hi", i64), ("n_lo", i64), ("n_hi", i64), ("m_lo", i64), ("m_hi", i64),
                ("hemispheres", i32), ("reserved_", i32)]


class fstat_plan_info(C.Structure):
    _fields_ = [("n_cells", i64), ("f_evals", i64), ("device_bytes", i64),
                ("kernel_launches", i64), ("n_fft_max", i64)]


CAND_DTYPE = np.dtype([("alpha", np.float64), ("delta", np.float64), ("freq", np.float64),
                       ("fdot", np.float64), ("F", np.float64), ("band", np.int32),
                       ("reserved", np.int32), ("sky", np.int64), ("spin", np.int64),
                       ("bin", np.int64)])
assert CAND_DTYPE.itemsize == C.sizeof(fstat_candidate)

_plan_p = C.c_void_p
_lib.fstat_plan_create.argtypes = [P(_plan_p), P(fstat_plan_desc)]
_lib.fstat_plan_create.restype = i32
_lib.fstat_plan_set_band.argtypes = [_plan_p, i32, P(fstat_band)]
_lib.fstat_plan_set_band.restype = i32
_lib.fstat_search.argtypes = [_plan_p, i64, i64]
_lib.fstat_search.restype = i32
_lib.fstat_candidates_get.argtypes = [_plan_p, P(fstat_candidate), i64, P(i64), P(i64)]
_lib.fstat_candidates_get.restype = i32
_lib.fstat_debug_sky.argtypes = [_plan_p, i32, i64, P(f64), P(f64), P(f64), P(C.c_uint8), P(f64)]
_lib.fstat_debug_sky.restype = i32
_lib.fstat_plan_get_info.argtypes = [_plan_p, P(fstat_plan_info)]
_lib.fstat_plan_get_info.restype = i32
_lib.fstat_plan_set_timing.argtypes = [_plan_p, i32]
_lib.fstat_plan_set_timing.restype = i32
_lib.fstat_plan_kernel_stats.argtypes = [_plan_p, P(fstat_kernel_stat), i32, P(i32)]
_lib.fstat_plan_kernel_stats.restype = i32
_lib.fstat_plan_autotune.argtypes = [_plan_p, i64, P(fstat_tuning)]
_lib.fstat_plan_autotune.restype = i32
_lib.fstat_cell_F_noalloc.argtypes = [C.c_void_p, i64, i64, f64, f64, f64, i64, i64,
                                       C.c_void_p, C.c_void_p]
_lib.fstat_cell_F_noalloc.restype = i32
_lib.fstat_lattice_grid.argtypes = [P(fstat_lattice), C.c_void_p, C.c_void_p, C.c_void_p, i64, P(i64),
                                    C.c_void_p, i64, P(i64), C.c_void_p]
_lib.fstat_lattice_grid.restype = i32
_lib.fstat_measure_fp32_fma.argtypes = [P(f64), C.c_void_p]
_lib.fstat_measure_fp32_fma.restype = i32
_lib.fstat_measure_l2_copy.argtypes = [i64, P(f64), C.c_void_p]
_lib.fstat_measure_l2_copy.restype = i32
_lib.fstat_plan_destroy.argtypes = [_plan_p]
_lib.fstat_plan_destroy.restype = None
_lib.fstat_status_string.argtypes = [i32]
_lib.fstat_status_string.restype = C.c_char_p
_lib.fstat_plan_error.argtypes = [_plan_p]
_lib.fstat_plan_error.restype = C.c_char_p

EXPORTED = ["fstat_plan_create", "fstat_plan_set_band", "fstat_search", "fstat_candidates_get", "fstat_debug_sky",
            "fstat_plan_get_info", "fstat_plan_set_timing", "fstat_plan_kernel_stats",
            "fstat_plan_autotune",
            "fstat_cell_F_noalloc", "fstat_measure_fp32_fma", "fstat_measure_l2_copy",
            "fstat_plan_destroy", "fstat_status_string",
            "fstat_plan_error"]


def measure_fp32_fma(stream: Optional[int] = None) -> float:
    """fstat_measure_fp32_fma: FP32 FMA throughput of the device, TFLOP/s."""
    v = f64()
    rc = _lib.fstat_measure_fp32_fma(C.byref(v), C.c_void_p(stream) if stream else None)
    if rc != FSTAT_OK:
        raise FstatError(rc, "fstat_measure_fp32_fma")
    return v.value


def measure_l2_copy(nbytes: int = 32 << 20, stream: Optional[int] = None) -> float:
    """fstat_measure_l2_copy: read + write GB/s of an L2-resident copy of nbytes."""
    v = f64()
    rc = _lib.fstat_measure_l2_copy(int(nbytes), C.byref(v), C.c_void_p(stream) if stream else None)
    if rc != FSTAT_OK:
        raise FstatError(rc, "fstat_measure_l2_copy")
    return v.value


def status_string(code: int) -> str:
    return _lib.fstat_status_string(code).decode()


class FstatError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{status_string(code)} ({code}): {msg}")
        self.code = code


def _ptr(a, ctype):
    return a.ctypes.data_as(P(ctype)) if a is not None else None


def _dev_ptr(t, ctype):
    return C.cast(C.c_void_p(t.data_ptr()), P(ctype))


def _fill_band(fb, b, on_device: bool) -> list:
    """Marshal one band (n, dt, f_off, phi0, eps, n_fft, x or float32 x, r) into
    an fstat_band; returns the arrays that must outlive the call."""
    fb.n = int(b.n)
    fb.dt, fb.f_off, fb.phi0 = float(b.dt), float(b.f_off), float(b.phi0)
    fb.eps = float(getattr(b, "eps", 0.0))
    fb.n_fft = int(getattr(b, "n_fft", 0) or 0)
    if on_device:
        if str(b.x.dtype) == "torch.float32":
            fb.x32 = _dev_ptr(b.x, C.c_float)
        else:
            fb.x = _dev_ptr(b.x, f64)
        fb.r = _dev_ptr(b.r, f64)
        return [b.x, b.r]
    x = np.ascontiguousarray(b.x)
    r = np.ascontiguousarray(np.asarray(b.r, dtype=np.float64).reshape(-1))
    if x.dtype == np.float32:
        fb.x32 = _ptr(x, C.c_float)
    else:
        x = x.astype(np.float64, copy=False)
        fb.x = _ptr(x, f64)
    fb.r = _ptr(r, f64)
    return [x, r]


class Plan:
    """One search plan: fstat_plan_create / fstat_search / fstat_candidates_get.

    bands: objects with n, dt, f_off, x (float64 or float32 array), r ([n,3]),
    phi0, eps, n_fft.  With on_device=True the arrays are torch CUDA tensors and
    their device pointers are passed (inputs_on_device = 1)."""

    def __init__(self, bands: Sequence, alpha, delta, fdot, thr_2F: float, *, lat: float,
                 gamma: float, upsample: int = 2, sigma2: float = 0.0, form: int = FP32_BATCHED,
                 bin_lo: int = 0, bin_hi: int = 0, cand_capacity: int = 1 << 20,
                 stream: Optional[int] = None, on_device: bool = False, full: bool = False,
                 interbin: bool = False):
        self._keep = []
        self._on_device = on_device
        nb = len(bands)
        arr = (fstat_band * nb)()
        for i, b in enumerate(bands):
            self._keep += _fill_band(arr[i], b, on_device)
        if on_device:
            pa, pd, pf = (_dev_ptr(alpha, f64), _dev_ptr(delta, f64), _dev_ptr(fdot, f64))
            n_sky, n_spin = int(alpha.numel()), int(fdot.numel())
            self._keep += [alpha, delta, fdot]
        else:
            alpha = np.ascontiguousarray(alpha, np.float64)
            delta = np.ascontiguousarray(delta, np.float64)
            fdot = np.ascontiguousarray(fdot, np.float64)
            self._keep += [alpha, delta, fdot]
            pa, pd, pf = _ptr(alpha, f64), _ptr(delta, f64), _ptr(fdot, f64)
            n_sky, n_spin = alpha.size, fdot.size
        d = fstat_plan_desc()
        d.n_bands, d.bands = nb, arr
        d.n_sky, d.alpha, d.delta = n_sky, pa, pd
        d.n_spin, d.fdot = n_spin, pf
        d.thr_2F, d.bin_lo, d.bin_hi = float(thr_2F), int(bin_lo), int(bin_hi)
        d.lat, d.gamma, d.upsample, d.sigma2 = float(lat), float(gamma), int(upsample), float(sigma2)
        d.form, d.cand_capacity = int(form), int(cand_capacity)
        d.statistic = F_FULL if full else F_SIMPLE
        d.interpolation = INTERP_INTERBIN if interbin else INTERP_ZEROPAD
        d.cuda_stream = C.c_void_p(stream) if stream else None
        d.inputs_on_device = 1 if on_device else 0
        self._desc = d
        self._arr = arr
        self._h = _plan_p()
        rc = _lib.fstat_plan_create(C.byref(self._h), C.byref(d))
        if rc != FSTAT_OK:
            raise FstatError(rc, "fstat_plan_create")
        self._keep = []   # the plan copied everything

    # ---------------------------------------------------------------- calls
    def _raise(self, rc, what):
        raise FstatError(rc, f"{what}: {_lib.fstat_plan_error(self._h).decode()}")

    def set_band(self, band: int, data) -> None:
        """fstat_plan_set_band: the next segment of band `band` (same n, dt, n_fft)."""
        fb = fstat_band()
        keep = _fill_band(fb, data, self._on_device)
        rc = _lib.fstat_plan_set_band(self._h, int(band), C.byref(fb))
        del keep
        if rc != FSTAT_OK:
            self._raise(rc, "fstat_plan_set_band")

    def search(self, cell_begin: int = 0, cell_end: int = -1, allow_overflow: bool = False) -> int:
        rc = _lib.fstat_search(self._h, cell_begin, cell_end)
        if rc not in (FSTAT_OK, FSTAT_ERR_OVERFLOW) or (rc == FSTAT_ERR_OVERFLOW and not allow_overflow):
            self._raise(rc, "fstat_search")
        return rc

    def search_status(self, cell_begin: int = 0, cell_end: int = -1) -> int:
        return _lib.fstat_search(self._h, cell_begin, cell_end)

    def candidates(self, cap: Optional[int] = None, out: Optional[np.ndarray] = None):
        """(structured array sorted by (band, sky, spin, bin), n_total).  With `out`
        (a CAND_DTYPE array, reused across calls) the records land there and a view
        of its first n_written entries is returned; it must hold every candidate
        unless cap limits the count."""
        nw, nt = i64(), i64()
        if cap is None:
            _lib.fstat_candidates_get(self._h, None, 0, C.byref(nw), C.byref(nt))
            cap = int(nt.value)
        if out is not None:
            if out.dtype != CAND_DTYPE or not out.flags.c_contiguous or out.size < cap:
                raise ValueError("out must be a contiguous CAND_DTYPE array of at least cap records")
            buf = out
        else:
            buf = np.empty(max(cap, 1), CAND_DTYPE)
        rc = _lib.fstat_candidates_get(self._h, buf.ctypes.data_as(P(fstat_candidate)), cap,
                                       C.byref(nw), C.byref(nt))
        if rc not in (FSTAT_OK, FSTAT_ERR_OVERFLOW):
            self._raise(rc, "fstat_candidates_get")
        if out is not None:
            return buf[:nw.value], int(nt.value)
        return (buf if nw.value == buf.size else buf[:nw.value].copy()), int(nt.value)

    def candidates_get_status(self, cap: int):
        nw, nt = i64(), i64()
        out = np.zeros(max(cap, 1), CAND_DTYPE)
        rc = _lib.fstat_candidates_get(self._h, out.ctypes.data_as(P(fstat_candidate)) if cap else None,
                                       cap, C.byref(nw), C.byref(nt))
        return rc, out[:nw.value].copy(), int(nt.value)

    def debug_sky(self, band: int, sky: int, n: int):
        y = np.zeros(2 * n)
        a, b = np.zeros(n), np.zeros(n)
        m = np.zeros(n, np.uint8)
        S = np.zeros(3)
        rc = _lib.fstat_debug_sky(self._h, band, sky, _ptr(y, f64), _ptr(a, f64), _ptr(b, f64),
                                  _ptr(m, C.c_uint8), _ptr(S, f64))
        if rc != FSTAT_OK:
            self._raise(rc, "fstat_debug_sky")
        return dict(y=y[0::2] + 1j * y[1::2], a=a, b=b, mask=m.astype(bool), S=S)

    def info(self):
        inf = fstat_plan_info()
        _lib.fstat_plan_get_info(self._h, C.byref(inf))
        return {k: getattr(inf, k) for k, _ in fstat_plan_info._fields_}

    def autotune(self, sample_cells: int):
        """Pick the launch shapes by timing searches over the first sample_cells
        cells; returns the chosen configuration."""
        t = fstat_tuning()
        rc = _lib.fstat_plan_autotune(self._h, int(sample_cells), C.byref(t))
        if rc != FSTAT_OK:
            self._raise(rc, "fstat_plan_autotune")
        return {k: getattr(t, k) for k, _ in fstat_tuning._fields_}

    def set_timing(self, sample_every: int):
        rc = _lib.fstat_plan_set_timing(self._h, int(sample_every))
        if rc != FSTAT_OK:
            self._raise(rc, "fstat_plan_set_timing")

    def kernel_stats(self):
        buf = (fstat_kernel_stat * 32)()
        n = i32()
        _lib.fstat_plan_kernel_stats(self._h, buf, 32, C.byref(n))
        out = {}
        for k in buf[:min(n.value, 32)]:
            out[k.name.decode()] = dict(launches=k.launches, timed_launches=k.timed_launches,
                                        timed_ms=k.timed_ms, flops_per_launch=k.flops_per_launch,
                                        bytes_per_launch=k.bytes_per_launch)
        return out

    def error(self) -> str:
        return _lib.fstat_plan_error(self._h).decode()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.fstat_plan_destroy(self._h)
            self._h = _plan_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def cell_F_noalloc(w_dev_ptr: int, n: int, n_fft: int, chirp_rate: float, norm_a: float,
                   norm_b: float, bin_lo: int, bin_hi: int, F_out_dev_ptr: int,
                   stream: Optional[int] = None) -> int:
    """fstat_cell_F_noalloc through the C ABI (device pointers as integers);
    returns the status code."""
    return _lib.fstat_cell_F_noalloc(C.c_void_p(w_dev_ptr), int(n), int(n_fft), float(chirp_rate),
                                     float(norm_a), float(norm_b), int(bin_lo), int(bin_hi),
                                     C.c_void_p(F_out_dev_ptr), C.c_void_p(stream) if stream else None)


def lattice_grid(M, dt: float, f_ref: float, eps: float, s_range, n_range, m_range,
                 hemispheres: int = 1, stream: Optional[int] = None):
    """fstat_lattice_grid: the search grid of a generating matrix M (4 x 4, rows
    frequency, spindown, sky n, sky m) over inclusive integer ranges, as torch CUDA
    tensors (alpha, delta, nm[:, (hemisphere, n, m)], fdot), ready for
    Plan(..., on_device=True)."""
    import torch
    L = fstat_lattice()
    Mf = np.ascontiguousarray(np.asarray(M, np.float64).reshape(16))
    for i in range(16):
        L.M[i] = float(Mf[i])
    L.dt, L.f_ref, L.eps = float(dt), float(f_ref), float(eps)
    L.s_lo, L.s_hi = int(s_range[0]), int(s_range[1])
    L.n_lo, L.n_hi = int(n_range[0]), int(n_range[1])
    L.m_lo, L.m_hi = int(m_range[0]), int(m_range[1])
    L.hemispheres = int(hemispheres)
    ns, nsp = i64(), i64()
    st = C.c_void_p(stream) if stream else None
    rc = _lib.fstat_lattice_grid(C.byref(L), None, None, None, 0, C.byref(ns), None, 0, C.byref(nsp), st)
    if rc != FSTAT_OK:
        raise FstatError(rc, "fstat_lattice_grid (count)")
    alpha = torch.empty(ns.value, dtype=torch.float64, device="cuda")
    delta = torch.empty(ns.value, dtype=torch.float64, device="cuda")
    nm = torch.empty((ns.value, 3), dtype=torch.int64, device="cuda")
    fdot = torch.empty(nsp.value, dtype=torch.float64, device="cuda")
    rc = _lib.fstat_lattice_grid(C.byref(L), C.c_void_p(alpha.data_ptr()), C.c_void_p(delta.data_ptr()),
                                 C.c_void_p(nm.data_ptr()), ns.value, C.byref(ns),
                                 C.c_void_p(fdot.data_ptr()), nsp.value, C.byref(nsp), st)
    if rc != FSTAT_OK:
        raise FstatError(rc, "fstat_lattice_grid")
    return alpha, delta, nm, fdot


def lattice_grid_status(M, **kw) -> int:
    """fstat_lattice_grid's status for arguments that may be invalid (count-only call)."""
    L = fstat_lattice()
    Mf = np.asarray(M, np.float64).reshape(16)
    for i in range(16):
        L.M[i] = float(Mf[i])
    for k, v in kw.items():
        setattr(L, k, v)
    ns, nsp = i64(), i64()
    return _lib.fstat_lattice_grid(C.byref(L), None, None, None, 0, C.byref(ns), None, 0, C.byref(nsp), None)


def plan_create_status(desc_kwargs_bands, **kw) -> int:
    """fstat_plan_create's status for arguments that may be invalid (for tests)."""
    try:
        p = Plan(desc_kwargs_bands, **kw)
        p.close()
        return FSTAT_OK
    except FstatError as e:
        return e.code
