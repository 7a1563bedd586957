"""GPU parity at the full sizes of the remaining standard workloads, in the launch
configuration of the default search, on sampled outputs the oracle computes one
by one:

- the plain FP64 form on the 1024-position grid at N_fft = 2^18;
- the FP32 batched form on 16 uneven float32 bands (1-4 sidereal days, N_fft
  2^17 .. 2^19, band offsets f_off = 100 + (1 - 2^-5) b, sigma per band);
- the FP32 batched form on the 65536 x 256 grid, searched as resumable cell
  ranges (the candidate stream is drained range by range).

Candidate indices must be identical except inside the tolerance band
|2F_ref - thr| <= 2 tol max(F_ref, 2); F within tol max(F_ref, 2).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1410_3677_gb300 import synth as S

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def fs():
    from paper_1410_3677_gb300 import fstat
    return fstat


def _plan(fs, w, form, cap):
    return fs.Plan(w.bands, w.alpha, w.delta, w.fdot, w.thr_2F, lat=w.lat, gamma=w.gamma,
                   upsample=w.upsample, form=form, cand_capacity=cap)


def _oracle(w, band_idx, cells):
    prm = O.params(w.lat, w.gamma, w.upsample, 0.0, False, 0)
    cs = np.array([c[0] for c in cells])
    cp = np.array([c[1] for c in cells])
    return O.cells_F(w.bands[band_idx], prm, w.alpha, w.delta, w.fdot, cs, cp, 0, 0, NTHREADS)


def _compare(c, w, band_idx, cells, ref, tol):
    """Candidates of the listed cells of one band against the oracle's F."""
    for i, (sk, sp) in enumerate(cells):
        sel = c[(c["band"] == band_idx) & (c["sky"] == sk) & (c["spin"] == sp)]
        want = np.nonzero(2 * ref[i] > w.thr_2F)[0] + 1
        got = sel["bin"]
        inband = np.abs(2 * ref[i] - w.thr_2F) <= 2 * tol * np.maximum(ref[i], 2.0)
        sym = set(want.tolist()) ^ set(got.tolist())
        assert all(inband[bn - 1] for bn in sym), (band_idx, sk, sp, sorted(sym)[:10])
        common = np.intersect1d(want, got)
        if common.size:
            Fg = sel["F"][np.isin(got, common)]
            err = np.abs(Fg - ref[i][common - 1]) / np.maximum(ref[i][common - 1], 2.0)
            assert err.max() <= tol, (band_idx, sk, sp, err.max())


def test_plain_fp64_form_1024_positions(fs):
    """The 1024 x 1 grid, N = 86164, N_fft = 2^18, FP64 plain form, 2F > 20: the
    injected cells and three others, every bin, at 1e-10."""
    w = S.workload(2)
    p = _plan(fs, w, fs.FP64_PLAIN, 1 << 24)
    assert p.search() == fs.FSTAT_OK, p.error()
    c, total = p.candidates()
    p.close()
    assert total == c.size > 0
    rng = np.random.default_rng(2)
    cells = sorted({(i.sky, i.spin) for i in w.bands[0].injections} |
                   {(int(rng.integers(w.n_sky)), 0) for _ in range(3)})
    ref = _oracle(w, 0, cells)
    _compare(c, w, 0, cells, ref, 1e-10)
    for inj in w.bands[0].injections:
        sel = c[(c["sky"] == inj.sky) & (c["spin"] == inj.spin)]
        assert sel.size and abs(int(sel["bin"][np.argmax(sel["F"])]) - inj.bin) <= 1


def test_banded_float32_16_bands(fs):
    """16 uneven float32 bands, 512 x 16 cells each, FP32 batched form, 2F > 30:
    per band an injected cell (where the band has one) and a random cell."""
    w = S.workload(4)
    p = _plan(fs, w, fs.FP32_BATCHED, 1 << 27)
    assert p.search() == fs.FSTAT_OK, p.error()
    c, total = p.candidates()
    info = p.info()
    p.close()
    assert total == c.size
    assert info["f_evals"] == sum(w.n_sky * w.n_spin * (b.n_fft // 2 - 1) for b in w.bands)
    rng = np.random.default_rng(4)
    for bi, b in enumerate(w.bands):
        cells = {(int(rng.integers(w.n_sky)), int(rng.integers(w.n_spin)))}
        if b.injections:
            cells.add((b.injections[0].sky, b.injections[0].spin))
        cells = sorted(cells)
        _compare(c, w, bi, cells, _oracle(w, bi, cells), 1e-4)
    # frequencies carry each band's offset
    for bi, b in enumerate(w.bands):
        sel = c[c["band"] == bi][:100]
        assert np.allclose(sel["freq"], b.f_off + sel["bin"] / (b.n_fft * b.dt), rtol=0, atol=1e-12)


def test_large_grid_streamed_by_cell_ranges(fs):
    """The 65536 x 256 grid (N_fft = 2^18, 2F > 30) searched as cell ranges, each
    range's candidates drained before the next search: three ranges of whole sky
    positions around injected ones; their sampled cells against the oracle and
    the injections found at their bins."""
    w = S.workload(5)
    b = w.bands[0]
    p = _plan(fs, w, fs.FP32_BATCHED, 1 << 25)
    rng = np.random.default_rng(5)
    injs = [b.injections[k] for k in rng.choice(len(b.injections), 3, replace=False)]
    for inj in injs:
        s0 = max(0, inj.sky - 2)
        lo, hi = s0 * w.n_spin, (s0 + 5) * w.n_spin
        assert p.search(lo, hi) == fs.FSTAT_OK, p.error()
        c, total = p.candidates()
        assert total == c.size
        cell = c["sky"] * w.n_spin + c["spin"]
        assert np.all((cell >= lo) & (cell < hi))
        cells = sorted({(inj.sky, inj.spin), (s0, int(rng.integers(w.n_spin))),
                        (s0 + 4, int(rng.integers(w.n_spin)))})
        _compare(c, w, 0, cells, _oracle(w, 0, cells), 1e-4)
        if inj.snr >= 12:
            sel = c[(c["sky"] == inj.sky) & (c["spin"] == inj.spin)]
            assert sel.size and abs(int(sel["bin"][np.argmax(sel["F"])]) - inj.bin) <= 1
    p.close()
