"""A stream of data segments through one plan (fstat_plan_set_band): the search
of a replaced segment must return exactly the candidates of a plan created on
that segment, whether or not the previous searches were replayed from a CUDA
graph, for float64 and float32 series, and when the band offset changes with
the segment (a kernel argument of the captured launches)."""
import numpy as np
import pytest

from paper_1410_3677_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    from paper_1410_3677_gb300 import fstat
    return fstat


def _segment(w, seed, dtype=np.float64, f_off=0.0):
    """Another segment of the tiny workload's band: same n, dt and n_fft, new noise,
    ephemeris phase and source."""
    b = w.bands[0]
    rng = np.random.default_rng(seed)
    inj = S.draw_injections(rng, 1, w.n_sky, w.n_spin, b.n_fft, b.dt, 20.0, 20.0)
    return S.make_band(b.n, b.dt, seed, 1.0, w.alpha, w.delta, w.fdot, inj, f_off=f_off,
                       n_fft=b.n_fft, lat=w.lat, gamma=w.gamma, dtype=dtype)


def _plan(fs, w, band, form):
    return fs.Plan([band], w.alpha, w.delta, w.fdot, w.thr_2F, lat=w.lat, gamma=w.gamma,
                   upsample=w.upsample, form=form, cand_capacity=1 << 20)


def _cands(p):
    assert p.search() == 0, p.error()
    c, total = p.candidates()
    assert total == c.size
    return c


@pytest.mark.parametrize("form", ["FP32_BATCHED", "FP64_PLAIN"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_replaced_segment_equals_fresh_plan(fs, form, dtype):
    w = S.workload(1)
    fm = getattr(fs, form)
    segs = [_segment(w, 11, dtype), _segment(w, 12, dtype), _segment(w, 13, dtype, f_off=100.0)]
    p = _plan(fs, w, segs[0], fm)
    first = _cands(p)
    _cands(p)          # a repeated search: captured as a graph, replayed from now on
    for seg in segs[1:]:
        p.set_band(0, seg)
        got = _cands(p)
        q = _plan(fs, w, seg, fm)
        want = _cands(q)
        q.close()
        assert got.size == want.size > 0
        assert np.array_equal(got, want)
        assert not np.array_equal(got["bin"][:10], first["bin"][:10]) or got.size != first.size
    # back to the first segment: the first candidates again
    p.set_band(0, segs[0])
    again = _cands(p)
    p.close()
    assert np.array_equal(again, first)


def test_set_band_rejects_another_shape(fs):
    w = S.workload(1)
    b = w.bands[0]
    p = _plan(fs, w, b, fs.FP32_BATCHED)
    short = S.make_band(b.n - 16, b.dt, 5, 1.0, w.alpha, w.delta, w.fdot, [], n_fft=b.n_fft)
    with pytest.raises(fs.FstatError) as e:
        p.set_band(0, short)
    assert e.value.code == fs.FSTAT_ERR_ARG
    other_dt = S.make_band(b.n, 2 * b.dt, 5, 1.0, w.alpha, w.delta, w.fdot, [], n_fft=b.n_fft)
    with pytest.raises(fs.FstatError) as e:
        p.set_band(0, other_dt)
    assert e.value.code == fs.FSTAT_ERR_ARG
    with pytest.raises(fs.FstatError) as e:
        p.set_band(1, b)
    assert e.value.code == fs.FSTAT_ERR_ARG
    # the plan is still usable after the refusals
    assert p.search() == 0
    p.close()


def test_replaced_segment_from_device_memory(fs):
    """inputs_on_device = 1: the segments are torch CUDA tensors (float32 series)."""
    import torch
    w = S.workload(1)
    segs = [_segment(w, 21, np.float32), _segment(w, 22, np.float32)]

    def dev(b):
        class D:
            pass
        d = D()
        d.n, d.dt, d.f_off, d.phi0, d.eps, d.n_fft = b.n, b.dt, b.f_off, b.phi0, b.eps, b.n_fft
        d.x = torch.from_numpy(np.ascontiguousarray(b.x)).cuda()
        d.r = torch.from_numpy(np.ascontiguousarray(b.r).reshape(-1)).cuda()
        return d

    grid = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (w.alpha, w.delta, w.fdot)]
    p = fs.Plan([dev(segs[0])], *grid, w.thr_2F, lat=w.lat, gamma=w.gamma, upsample=w.upsample,
                form=fs.FP32_BATCHED, cand_capacity=1 << 20, on_device=True)
    _cands(p)
    p.set_band(0, dev(segs[1]))
    got = _cands(p)
    p.close()
    q = _plan(fs, w, segs[1], fs.FP32_BATCHED)
    want = _cands(q)
    q.close()
    assert got.size == want.size > 0 and np.array_equal(got, want)
