"""The device grid from a generating matrix (Sect. 2, grid.bin) against the
oracle's: the list of sky points (hemisphere, n, m) bit-exact, the spindowns
bit-exact, the angles within a few units in the last place (atan2 / asin of the
two math libraries), an overflow that keeps the counts exact, and a search on the
generated grid identical to a search on the oracle's arrays."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1410_3677_gb300 import synth as S

pytestmark = pytest.mark.gpu

EPS = 0.40909280422232897
TAU_E = 499.00478383615643


def _M(f_ref, step, hexagonal, spin):
    sc = f_ref * TAU_E * step
    M = np.zeros((4, 4))
    M[0, 0] = 2.0 ** -18
    M[1, 1] = spin
    M[0, 2], M[0, 3] = 0.3, -0.1          # frequency-row sky components: unused by the grid
    if hexagonal:
        M[2, 2:] = [sc, 0.0]
        M[3, 2:] = [0.5 * sc, 0.5 * math.sqrt(3.0) * sc]
    else:
        M[2, 2:] = [sc, 0.1 * sc]
        M[3, 2:] = [-0.2 * sc, 0.9 * sc]
    M[2, 0], M[3, 0] = 1e-7, 2e-7         # frequency components of the sky rows: the FFT's grid
    return M


def _ang(a, b):
    return np.abs(np.mod(a - b + math.pi, 2 * math.pi) - math.pi)


@pytest.mark.parametrize("hexagonal,hemi,step,rng", [(False, 1, 1 / 40.5, 45), (True, 2, 1 / 60.25, 80),
                                                    (False, 2, 1 / 3.3, 4)])
def test_grid_matches_oracle(hexagonal, hemi, step, rng):
    from paper_1410_3677_gb300 import fstat as fs
    f_ref, dt = 100.25, 2.0
    M = _M(f_ref, step, hexagonal, 7.5e-15)
    a, d, nm, fd = fs.lattice_grid(M, dt, f_ref, EPS, (-17, 30), (-rng, rng), (-rng, rng), hemi)
    ra, rd, rnm = O.lattice_sky(M, f_ref, EPS, -rng, rng, -rng, rng, hemi)
    rf = O.lattice_spin(M, dt, -17, 30)
    assert np.array_equal(nm.cpu().numpy(), rnm)
    assert np.array_equal(fd.cpu().numpy(), rf)
    ga, gd = a.cpu().numpy(), d.cpu().numpy()
    assert np.max(_ang(ga, ra)) <= 4e-15 and np.max(np.abs(gd - rd)) <= 4e-15
    assert np.all((ga >= 0) & (ga < 2 * math.pi))


def test_overflow_keeps_counts():
    import ctypes as C
    import torch
    from paper_1410_3677_gb300 import fstat as fs
    M = _M(100.25, 1 / 10.5, False, 1e-14)
    L = fs.fstat_lattice()
    for i, v in enumerate(M.reshape(16)):
        L.M[i] = float(v)
    L.dt, L.f_ref, L.eps = 2.0, 100.25, EPS
    L.s_lo, L.s_hi, L.n_lo, L.n_hi, L.m_lo, L.m_hi, L.hemispheres = 0, 9, -12, 12, -12, 12, 1
    a = torch.empty(50, dtype=torch.float64, device="cuda")
    d = torch.empty(50, dtype=torch.float64, device="cuda")
    f = torch.empty(4, dtype=torch.float64, device="cuda")
    ns, nsp = C.c_int64(), C.c_int64()
    rc = fs._lib.fstat_lattice_grid(C.byref(L), C.c_void_p(a.data_ptr()), C.c_void_p(d.data_ptr()), None,
                                    50, C.byref(ns), C.c_void_p(f.data_ptr()), 4, C.byref(nsp), None)
    ra, rd, _ = O.lattice_sky(M, 100.25, EPS, -12, 12, -12, 12, 1)
    assert rc == fs.FSTAT_ERR_OVERFLOW and ns.value == len(ra) > 50 and nsp.value == 10
    assert np.max(_ang(a.cpu().numpy(), ra[:50])) <= 4e-15
    assert np.array_equal(f.cpu().numpy(), O.lattice_spin(M, 2.0, 0, 3))


def test_search_on_generated_grid():
    """A plan fed the device-generated grid (inputs on the device) returns the
    candidates of a plan fed the oracle's grid arrays from the host: the grids
    are the same points, so the searches are the same."""
    import torch
    from paper_1410_3677_gb300 import fstat as fs
    w = S.workload(1, n_sky=4, n_spin=4)
    b = w.bands[0]
    f_ref = b.f_off + 1.0 / (2 * b.dt)
    M = _M(f_ref, 1 / 2.5, True, 2.5e-10 * b.dt * b.dt / 2)
    a, d, nm, fd = fs.lattice_grid(M, b.dt, f_ref, EPS, (-3, 0), (-2, 2), (-2, 2), 1)
    ra, rd, _ = O.lattice_sky(M, f_ref, EPS, -2, 2, -2, 2, 1)
    rf = O.lattice_spin(M, b.dt, -3, 0)
    p0 = fs.Plan(w.bands, ra, rd, rf, 12.0, lat=w.lat, gamma=w.gamma, form=fs.FP32_BATCHED)
    p0.search()
    ref, _ = p0.candidates()
    p0.close()

    class DB:
        pass
    db = DB()
    db.n, db.dt, db.f_off, db.phi0, db.eps, db.n_fft = b.n, b.dt, b.f_off, b.phi0, b.eps, b.n_fft
    db.x = torch.from_numpy(b.x).cuda()
    db.r = torch.from_numpy(np.ascontiguousarray(b.r)).cuda()
    p1 = fs.Plan([db], a, d, fd, 12.0, lat=w.lat, gamma=w.gamma, form=fs.FP32_BATCHED, on_device=True)
    p1.search()
    got, _ = p1.candidates()
    p1.close()
    assert got.size > 0
    assert np.array_equal(got[["sky", "spin", "bin"]], ref[["sky", "spin", "bin"]])
    # angles differ in the last bits between the libraries: F within the FP32 tolerance
    assert np.max(np.abs(got["F"] - ref["F"]) / np.maximum(ref["F"], 2.0)) <= 1e-4
