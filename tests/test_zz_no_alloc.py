"""The allocation-free single-cell entry point, for callers that cannot allocate
device memory (they hold the device memory budget themselves and pass views).

It must reproduce, through the C ABI, the F of every bin that the plan-based
search computes for the same cell, on two calls in a row (two different cells),
within the FP32 tolerance of the other GPU tests, and refuse lengths beyond its
maximum.  This file is collected last."""
import math

import numpy as np
import pytest

from paper_1410_3677_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _case(fs, w, cells):
    import torch
    band = w.bands[0]
    p = fs.Plan(w.bands, w.alpha, w.delta, w.fdot, -1.0, lat=w.lat, gamma=w.gamma,
                upsample=w.upsample, form=fs.FP32_BATCHED, cand_capacity=1 << 20)
    nb = band.n_fft // 2 - 1
    sigma2 = math.fsum(np.asarray(band.x, np.float64) ** 2) / band.n
    stream = torch.cuda.current_stream()
    out = torch.empty(nb, dtype=torch.float32, device="cuda")
    for sky, spin in cells:          # two calls in a row, different cells
        cell = sky * w.n_spin + spin
        assert p.search(cell, cell + 1) == fs.FSTAT_OK
        c, total = p.candidates()
        assert total == nb and np.array_equal(c["bin"], np.arange(1, nb + 1))
        g = p.debug_sky(0, sky, band.n)
        y = g["y"]
        a = g["a"].astype(np.float32)
        b = g["b"].astype(np.float32)
        yr, yi = y.real.astype(np.float32), y.imag.astype(np.float32)
        w4 = np.ascontiguousarray(np.stack([yr * a, yi * a, yr * b, yi * b], 1), np.float32)
        wt = torch.from_numpy(w4).cuda()
        out.fill_(float("nan"))
        rate = 0.5 * float(w.fdot[spin]) * band.dt * band.dt
        rc = fs.cell_F_noalloc(wt.data_ptr(), band.n, band.n_fft, rate, 1.0 / (sigma2 * g["S"][0]),
                               1.0 / (sigma2 * g["S"][1]), 1, nb, out.data_ptr(),
                               stream.cuda_stream)
        assert rc == fs.FSTAT_OK
        F = out.cpu().numpy().astype(np.float64)
        err = np.abs(F - c["F"]) / np.maximum(c["F"], 2.0)
        assert np.all(np.isfinite(F)) and err.max() <= 1e-4, (sky, spin, err.max())
    p.close()


def test_noalloc_matches_plan_two_calls():
    from paper_1410_3677_gb300 import fstat as fs
    _case(fs, S.workload(1, n_sky=6, n_spin=4), [(1, 2), (4, 0)])          # N_fft = 2^13
    w = S.workload(2, n_sky=1024, n_spin=1)
    inj = w.bands[0].injections[0]
    w2 = S.Workload(w.name, w.bands, w.alpha[[3, inj.sky]], w.delta[[3, inj.sky]], w.fdot, w.thr_2F)
    _case(fs, w2, [(1, 0), (0, 0)])                                          # N_fft = 2^18


def test_noalloc_rejects_beyond_maximum():
    import torch
    from paper_1410_3677_gb300 import fstat as fs
    buf = torch.zeros(4 * 8, dtype=torch.float32, device="cuda")
    out = torch.zeros(8, dtype=torch.float32, device="cuda")
    assert fs.cell_F_noalloc(buf.data_ptr(), 8, 1 << 19, 0.0, 1.0, 1.0, 1, 7, out.data_ptr()) == fs.FSTAT_ERR_ARG
    assert fs.cell_F_noalloc(buf.data_ptr(), 8, 1 << 11, 0.0, 1.0, 1.0, 1, 7, out.data_ptr()) == fs.FSTAT_ERR_ARG
    assert fs.cell_F_noalloc(0, 8, 1 << 12, 0.0, 1.0, 1.0, 1, 7, out.data_ptr()) == fs.FSTAT_ERR_ARG
    # views that start off the 16-byte (series) or 4-byte (output) boundary are
    # refused on the host, before anything is launched
    assert fs.cell_F_noalloc(buf.data_ptr() + 4, 8, 1 << 12, 0.0, 1.0, 1.0, 1, 7,
                             out.data_ptr()) == fs.FSTAT_ERR_ARG
    assert fs.cell_F_noalloc(buf.data_ptr(), 8, 1 << 12, 0.0, 1.0, 1.0, 1, 7,
                             out.data_ptr() + 2) == fs.FSTAT_ERR_ARG


def test_noalloc_allocates_no_device_memory():
    """The property the entry point exists for: once the kernels of a length are
    loaded (first call), further calls leave the device's free memory unchanged."""
    import torch
    from paper_1410_3677_gb300 import fstat as fs
    n, n_fft = 3000, 1 << 13
    rng = np.random.default_rng(7)
    w = torch.from_numpy(rng.standard_normal((n, 4)).astype(np.float32)).cuda()
    out = torch.empty(n_fft // 2 - 1, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    args = (w.data_ptr(), n, n_fft, 1e-7, 1.0, 1.0, 1, n_fft // 2 - 1, out.data_ptr(), stream)
    assert fs.cell_F_noalloc(*args) == fs.FSTAT_OK     # first call: set-up and module load
    first = out.clone()                                 # torch's own allocation, outside the window
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert fs.cell_F_noalloc(*args) == fs.FSTAT_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(out, first)                      # the shared scratch keeps no state
    del first
