"""Pins of the oracle's grid from the generating matrix M (Sect. 2: the integer
multiples of M's rows are the grid points; a sky position is a pair of integers
(n, m), a spindown an integer s), each against something other than the oracle:
positions a reader can name by hand (the ecliptic poles, the equinox, the
solstice points), the lattice-point count of a disk by integer arithmetic, and
exact integer round trips through an independent inversion of M."""
import math

import numpy as np
import pytest

import oracle as O

EPS = 0.40909280422232897     # obliquity of the ecliptic, rad (23.439281 deg)
TAU_E = 499.00478383615643    # 1 AU / c, s
F_REF = 100.25


def _M(step=1.0, hexagonal=False, spin=1e-14):
    """Sky rows spanning steps of `step` in the ecliptic-plane components beta;
    the spindown row (0, spin, 0, 0); the frequency row (1/2^18, 0, 0, 0)."""
    sc = F_REF * TAU_E * step
    M = np.zeros((4, 4))
    M[0, 0] = 2.0 ** -18
    M[1, 1] = spin
    if hexagonal:                 # rows (1, 0) and (1/2, sqrt(3)/2): the A2 lattice
        M[2, 2:] = [sc, 0.0]
        M[3, 2:] = [0.5 * sc, 0.5 * math.sqrt(3.0) * sc]
    else:
        M[2, 2] = sc
        M[3, 3] = sc
    return M


def _ang(a, b):
    return abs((a - b + math.pi) % (2 * math.pi) - math.pi)


def test_named_sky_points():
    """Unit steps in beta: the centre is the north ecliptic pole (alpha = 18 h,
    delta = 90 deg - eps), beta = (1, 0) the vernal equinox (0, 0), beta = (0, 1)
    the summer-solstice point (6 h, +eps), (-1, 0) and (0, -1) their opposites;
    the south hemisphere's centre is the south ecliptic pole (6 h, eps - 90 deg)."""
    a, d, nm = O.lattice_sky(_M(), F_REF, EPS, -1, 1, -1, 1, hemispheres=2)
    got = {tuple(k): (x, y) for k, x, y in zip(nm.tolist(), a, d)}
    want = {(0, 0, 0): (1.5 * math.pi, 0.5 * math.pi - EPS),
            (0, 1, 0): (0.0, 0.0),
            (0, 0, 1): (0.5 * math.pi, EPS),
            (0, -1, 0): (math.pi, 0.0),
            (0, 0, -1): (1.5 * math.pi, -EPS),
            (1, 0, 0): (0.5 * math.pi, EPS - 0.5 * math.pi)}
    assert set(got) == set(want)          # corners (|beta| = sqrt 2) are off the sphere
    for k, (wa, wd) in want.items():
        ga, gd = got[k]
        assert _ang(ga, wa) < 1e-12 and abs(gd - wd) < 1e-12, (k, ga, gd)
    # the order: north hemisphere first, then n, then m ascending
    assert nm.tolist() == [[0, -1, 0], [0, 0, -1], [0, 0, 0], [0, 0, 1], [0, 1, 0], [1, 0, 0]]


@pytest.mark.parametrize("R", [3.7, 10.3, 25.9])
def test_disk_point_count(R):
    """With sky steps of 1/R in beta the points on the sphere are the integer
    pairs with n^2 + m^2 <= R^2 (counted by integer arithmetic; R is chosen so
    that no integer n^2 + m^2 lies near R^2)."""
    k = int(math.ceil(R)) + 1
    nn, mm = np.meshgrid(np.arange(-k, k + 1), np.arange(-k, k + 1), indexing="ij")
    want = int(np.sum(nn * nn + mm * mm <= math.floor(R * R)))
    a, d, nm = O.lattice_sky(_M(1.0 / R), F_REF, EPS, -k, k, -k, k, hemispheres=1)
    assert len(a) == want
    a2, _, nm2 = O.lattice_sky(_M(1.0 / R), F_REF, EPS, -k, k, -k, k, hemispheres=2)
    assert len(a2) == 2 * want and np.array_equal(nm2[:want], nm)


@pytest.mark.parametrize("hexagonal", [False, True])
def test_round_trip_to_integers(hexagonal):
    """(alpha, delta) -> unit vector -> ecliptic components -> lattice
    coordinates through the inverse of M's sky block: the integers (n, m) come
    back exactly, and the hemisphere is the sign of the ecliptic latitude."""
    M = _M(1.0 / 12.5, hexagonal=hexagonal)
    a, d, nm = O.lattice_sky(M, F_REF, EPS, -15, 15, -15, 15, hemispheres=2)
    assert len(a) > 500
    x = np.cos(d) * np.cos(a)
    y = np.cos(d) * np.sin(a)
    z = np.sin(d)
    b1 = x
    b2 = y * math.cos(EPS) + z * math.sin(EPS)
    ze = -y * math.sin(EPS) + z * math.cos(EPS)
    w = np.stack([b1, b2], 1) * (F_REF * TAU_E)
    nmf = np.linalg.solve(M[2:, 2:].T, w.T).T
    assert np.max(np.abs(nmf - np.rint(nmf))) < 1e-6
    assert np.array_equal(np.rint(nmf).astype(np.int64), nm[:, 1:])
    north = nm[:, 0] == 0
    assert np.all(ze[north] >= -1e-12) and np.all(ze[~north] < 0)


def test_spindown_row():
    """fdot = 2 w1 / dt^2 with w1 = s M[1][1]: back to the integers exactly, and
    zero at s = 0."""
    M = _M(spin=3.0e-14)
    f = O.lattice_spin(M, 2.0, -5, 7)
    s = f * 4.0 / (2 * 3.0e-14)
    assert np.array_equal(np.rint(s).astype(int), np.arange(-5, 8))
    assert np.max(np.abs(s - np.rint(s))) < 1e-9 and f[5] == 0.0
