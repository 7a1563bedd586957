"""C-ABI checks that need no GPU: the library loads, exports every function the
public header declares, and rejects invalid arguments before touching CUDA."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fs():
    from paper_1410_3677_gb300 import build
    build.build()
    from paper_1410_3677_gb300 import fstat
    return fstat


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(fstat_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("fstat_plan_create", "fstat_search", "fstat_candidates_get",
                 "fstat_plan_destroy", "fstat_status_string"):
        assert name in d


def test_library_exports_every_declared_symbol(fs):
    out = subprocess.run(["nm", "-D", "--defined-only", fs.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fstat_\w+)", out))
    for name in _declared():
        assert name in exported, name
        assert hasattr(fs._lib, name)


def test_library_leaves_no_internal_symbol_unresolved(fs):
    """Every function of the library's own namespace is defined in it (a missing
    definition would only show at the first call)."""
    out = subprocess.run(["nm", "-D", "--undefined-only", fs.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    missing = [ln.split()[-1] for ln in out.splitlines() if "_ZN5fstat" in ln]
    assert not missing, missing


def test_struct_layouts(fs):
    assert C.sizeof(fs.fstat_band) == 72
    assert C.sizeof(fs.fstat_candidate) == 72
    assert C.sizeof(fs.fstat_plan_desc) == 144
    assert C.sizeof(fs.fstat_plan_info) == 40
    assert C.sizeof(fs.fstat_tuning) == 32


def test_status_strings(fs):
    for code in range(8):
        assert fs.status_string(code)
    assert fs.status_string(99) == "unknown status"


class _B:
    def __init__(self, n=64, dt=2.0, x=True, x32=False, n_fft=0, r=True):
        self.n, self.dt, self.f_off, self.phi0, self.eps, self.n_fft = n, dt, 0.0, 0.1, 0.4, n_fft
        self.x = np.zeros(n, np.float32 if x32 else np.float64)
        self.r = np.zeros((n, 3))


def _status(fs, bands, **kw):
    args = dict(alpha=np.zeros(2), delta=np.zeros(2), fdot=np.zeros(1), thr_2F=10.0, lat=0.7,
                gamma=2.0)
    args.update(kw)
    try:
        p = fs.Plan(bands, **args)
        p.close()
        return fs.FSTAT_OK
    except fs.FstatError as e:
        return e.code


@pytest.mark.parametrize("case", [
    dict(bands=[_B(n=8)]),                                   # n < 16
    dict(bands=[_B(n=64, n_fft=100)]),                       # not a power of two
    dict(bands=[_B(n=64, n_fft=64)]),                        # n_fft < 2n
    dict(bands=[_B(n=64, n_fft=1 << 21)]),                   # beyond 2^20
    dict(bands=[_B(dt=0.0)]),
    dict(bands=[_B(dt=float("nan"))]),
    dict(bands=[_B()], upsample=0),
    dict(bands=[_B()], upsample=9),
    dict(bands=[_B()], cand_capacity=0),
    dict(bands=[_B()], thr_2F=float("inf")),
    dict(bands=[_B()], form=7),
    dict(bands=[_B()], bin_lo=5, bin_hi=3),
    dict(bands=[_B()], bin_lo=0, bin_hi=256),                 # >= n_fft (auto 128... 256)
    dict(bands=[_B()], fdot=np.zeros(0)),
    dict(bands=[_B(n=4096)], interbin=True, form=0),          # interbinning: FP32 form only
    dict(bands=[_B()], interbin=True, form=1),                # interbinning: n_fft >= 2^13
])
def test_invalid_arguments_rejected_without_gpu(fs, case):
    bands = case.pop("bands")
    assert _status(fs, bands, **case) == fs.FSTAT_ERR_ARG


def test_null_handles(fs):
    assert fs._lib.fstat_search(None, 0, -1) == fs.FSTAT_ERR_ARG
    assert fs._lib.fstat_candidates_get(None, None, 0, None, None) == fs.FSTAT_ERR_ARG
    assert fs._lib.fstat_plan_create(None, None) == fs.FSTAT_ERR_ARG
    h = fs._plan_p()
    assert fs._lib.fstat_plan_create(C.byref(h), None) == fs.FSTAT_ERR_ARG
    assert not h.value
    fs._lib.fstat_plan_destroy(None)
    assert fs._lib.fstat_plan_error(None) == b""
    assert fs._lib.fstat_plan_set_band(None, 0, None) == fs.FSTAT_ERR_ARG
    # measurement helpers check their arguments before touching a device
    assert fs._lib.fstat_measure_fp32_fma(None, None) == fs.FSTAT_ERR_ARG
    v = C.c_double(1.0)
    assert fs._lib.fstat_measure_l2_copy(1000, C.byref(v), None) == fs.FSTAT_ERR_ARG
    assert fs._lib.fstat_measure_l2_copy(1 << 24, None, None) == fs.FSTAT_ERR_ARG


def test_both_or_neither_series_rejected(fs):
    b = _B()
    d = fs.fstat_plan_desc()
    arr = (fs.fstat_band * 1)()
    arr[0].n, arr[0].dt, arr[0].n_fft = 64, 2.0, 0
    x = np.zeros(64)
    r = np.zeros(192)
    arr[0].r = r.ctypes.data_as(C.POINTER(C.c_double))
    al = np.zeros(1)
    d.n_bands, d.bands, d.n_sky, d.alpha, d.delta = 1, arr, 1, al.ctypes.data_as(C.POINTER(C.c_double)), al.ctypes.data_as(C.POINTER(C.c_double))
    d.n_spin, d.fdot, d.upsample, d.cand_capacity = 1, al.ctypes.data_as(C.POINTER(C.c_double)), 2, 10
    h = fs._plan_p()
    assert fs._lib.fstat_plan_create(C.byref(h), C.byref(d)) == fs.FSTAT_ERR_ARG   # neither
    x32 = np.zeros(64, np.float32)
    arr[0].x = x.ctypes.data_as(C.POINTER(C.c_double))
    arr[0].x32 = x32.ctypes.data_as(C.POINTER(C.c_float))
    assert fs._lib.fstat_plan_create(C.byref(h), C.byref(d)) == fs.FSTAT_ERR_ARG   # both
    del b


def test_lattice_struct_and_argument_checks(fs):
    """fstat_lattice_grid refuses invalid arguments on the host, before any CUDA
    call: coupled spindown and sky rows (not a product grid), a bad hemisphere
    count, empty ranges, non-finite entries."""
    assert C.sizeof(fs.fstat_lattice) == 16 * 8 + 3 * 8 + 6 * 8 + 8
    M = np.zeros((4, 4))
    M[1, 1], M[2, 2], M[3, 3] = 1e-14, 1e3, 1e3
    ok = dict(dt=2.0, f_ref=100.0, eps=0.4, s_lo=0, s_hi=3, n_lo=-2, n_hi=2, m_lo=-2, m_hi=2,
              hemispheres=1)
    for bad in ((1, 2), (1, 3), (2, 1), (3, 1)):
        Mc = M.copy()
        Mc[bad] = 1e-3
        assert fs.lattice_grid_status(Mc, **ok) == fs.FSTAT_ERR_ARG, bad
    for k, v in (("hemispheres", 3), ("dt", 0.0), ("f_ref", -1.0), ("s_hi", -1), ("n_hi", -3)):
        assert fs.lattice_grid_status(M, **dict(ok, **{k: v})) == fs.FSTAT_ERR_ARG, k
    Mn = M.copy()
    Mn[2, 2] = float("nan")
    assert fs.lattice_grid_status(Mn, **ok) == fs.FSTAT_ERR_ARG
