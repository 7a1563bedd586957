"""Per-result error of the FP32 batched form against the FP64 oracle on a
256-cell sample of the precision workload (4096 x 64 cells, N = 86164,
N_fft = 2^18, 2F > 30), every searched bin of every sampled cell.

The sample: the sky position of each of the 16 injected signals with 16
consecutive spindowns around the injected one (signal-bearing and noise bins
alike).  Reported: the max, p50, p99 and p99.9 of |F_gpu - F_ref| / max(F_ref, 2)
over all 256 x 131071 bins; the same above F_ref = 10; and the symmetric
difference of the candidate sets at 2F > 30 with each differing candidate's
distance from the threshold in units of the tolerance band 2 tol max(F_ref, 2).
The report is printed in the terminal summary (section "F error vs the FP64
oracle").  Bounds: max error <= 1e-4; every differing candidate inside the band.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1410_3677_gb300 import synth as S

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 4
TOL = 1e-4


def test_error_report_precision_workload_256_cells(report_lines):
    from paper_1410_3677_gb300 import fstat as fs
    w = S.workload(3)
    b = w.bands[0]
    nb = b.n_fft // 2 - 1
    sample = []                                  # (sky, first spindown) of 16-cell runs
    for inj in b.injections:
        s0 = min(max(inj.spin - 8, 0), w.n_spin - 16)
        sample.append((inj.sky, s0))
    assert len(sample) == 16
    p = fs.Plan(w.bands, w.alpha, w.delta, w.fdot, -1.0, lat=w.lat, gamma=w.gamma,
                upsample=w.upsample, form=fs.FP32_BATCHED, cand_capacity=16 * nb)
    F_gpu = np.empty((256, nb))
    cells = []
    for i, (sky, s0) in enumerate(sample):
        lo = sky * w.n_spin + s0
        assert p.search(lo, lo + 16) == fs.FSTAT_OK, p.error()
        c, total = p.candidates()
        assert total == 16 * nb
        F_gpu[16 * i:16 * i + 16] = c["F"].reshape(16, nb)
        assert np.array_equal(c["spin"].reshape(16, nb)[:, 0], np.arange(s0, s0 + 16))
        cells += [(sky, s0 + j) for j in range(16)]
    p.close()
    prm = O.params(w.lat, w.gamma, w.upsample, 0.0, False, 0)
    cs = np.array([c[0] for c in cells])
    cp = np.array([c[1] for c in cells])
    F_ref = O.cells_F(b, prm, w.alpha, w.delta, w.fdot, cs, cp, 0, 0, NTHREADS)
    assert F_ref.shape == F_gpu.shape
    err = np.abs(F_gpu - F_ref) / np.maximum(F_ref, 2.0)
    strong = F_ref > 10.0
    thr = w.thr_2F
    want, got = 2 * F_ref > thr, 2 * F_gpu > thr   # the kernel's F > thr/2 in float, stored exactly
    diff = np.nonzero(want != got)
    dist = np.abs(2 * F_ref[diff] - thr) / (2 * TOL * np.maximum(F_ref[diff], 2.0))
    rep = {"workload": "precision 4096x64, N_fft=2^18; sample: 16 sky positions (one per injection) "
                       "x 16 consecutive spindowns = 256 cells, all 131071 bins",
           "bins": int(err.size),
           "rel_err": {"max": float(err.max()), "p50": float(np.percentile(err, 50)),
                       "p99": float(np.percentile(err, 99)), "p99.9": float(np.percentile(err, 99.9))},
           "rel_err_F_ref_above_10": {"bins": int(strong.sum()),
                                      "max": float(err[strong].max()) if strong.any() else None},
           "candidates_2F_gt_30": {"oracle": int(want.sum()), "gpu": int(got.sum()),
                                   "symmetric_difference": int(diff[0].size),
                                   "max_distance_in_band_units": float(dist.max()) if dist.size else None}}
    report_lines.append("F error vs the FP64 oracle (FP32 batched form): " + json.dumps(rep))
    assert err.max() <= TOL, rep
    assert np.all(dist <= 1.0), rep
    assert want.sum() > 0
