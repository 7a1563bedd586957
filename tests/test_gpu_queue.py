"""The persistent FP32 search kernel and its device work queue.

Its per-element arithmetic is the same as the two-launches-per-batch form, so the
candidates must agree bit for bit, whatever the batch size and the number of
scratch slots.  A withheld completion (test hook) must end the search with
FSTAT_ERR_TIMEOUT after the bounded waits run out, leaving the GPU usable.
"""
import os
import time

import numpy as np
import pytest

from paper_1410_3677_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fs():
    from paper_1410_3677_gb300 import fstat
    return fstat


def _run(fs, w, thr, env=None, **kw):
    old = {}
    for k, v in (env or {}).items():
        old[k] = os.environ.get(k)
        os.environ[k] = v
    try:
        p = fs.Plan(w.bands, w.alpha, w.delta, w.fdot, thr, lat=w.lat, gamma=w.gamma,
                    upsample=w.upsample, form=fs.FP32_BATCHED, cand_capacity=1 << 22, **kw)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v
    rc = p.search_status()
    c, total = p.candidates() if rc in (fs.FSTAT_OK, fs.FSTAT_ERR_OVERFLOW) else (None, None)
    return p, rc, c, total


R8 = {"FSTAT_PERSISTENT": "0", "FSTAT_ENGINE": "1"}     # radix-8 engine, two launches per batch
# two-stage engine, two launches per batch, scalar FP32 (the fused launch's arithmetic)
TWO = {"FSTAT_PERSISTENT": "0", "FSTAT_FUSED": "0", "FSTAT_PACKED": "0"}
DEFAULT = {"FSTAT_PERSISTENT": "0"}                       # the default (pass 2 paired at 2^18)
FUSED = {"FSTAT_PERSISTENT": "0", "FSTAT_FUSED": "1"}    # two-stage engine, one ticket-ordered launch
PK1 = {"FSTAT_PERSISTENT": "0", "FSTAT_FUSED": "0", "FSTAT_PACKED": "1"}   # pass 2 paired at 2^18
PK2 = {"FSTAT_PERSISTENT": "0", "FSTAT_FUSED": "0", "FSTAT_PACKED": "2"}   # both passes paired
PK3 = {"FSTAT_PERSISTENT": "0", "FSTAT_FUSED": "0", "FSTAT_PACKED": "3"}   # pass 2 and pass-1 stage 1


@pytest.mark.parametrize("base,env", [
    (R8, {"FSTAT_PERSISTENT": "1", "FSTAT_PERSIST_BATCH": "1", "FSTAT_PERSIST_SLOTS": "2"}),
    (R8, {"FSTAT_PERSISTENT": "1", "FSTAT_PERSIST_BATCH": "3", "FSTAT_PERSIST_SLOTS": "3"}),
    (R8, {"FSTAT_PERSISTENT": "1", "FSTAT_PERSIST_BATCH": "5", "FSTAT_PERSIST_SLOTS": "8"}),
    (R8, {"FSTAT_ENGINE": "1", "FSTAT_ELEMS_PER_THREAD": "8"}),
    (R8, {"FSTAT_ENGINE": "1", "FSTAT_ELEMS_PER_THREAD": "8", "FSTAT_CELL_BATCH": "7", "FSTAT_STREAMS": "2"}),
    (TWO, {"FSTAT_FUSED": "0", "FSTAT_PACKED": "0", "FSTAT_CELL_BATCH": "7", "FSTAT_STREAMS": "2"}),
    (TWO, {"FSTAT_FUSED": "0", "FSTAT_PACKED": "0", "FSTAT_CELL_BATCH": "1", "FSTAT_STREAMS": "3"}),
    (PK1, DEFAULT),
    (PK1, {"FSTAT_CELL_BATCH": "2"}),
    (PK1, {"FSTAT_CELL_BATCH": "7", "FSTAT_STREAMS": "2"}),
    (PK1, {"FSTAT_PF_DIST": "0", "FSTAT_CELL_BATCH": "9"}),
    (PK2, {"FSTAT_PACKED": "2", "FSTAT_CELL_BATCH": "5", "FSTAT_STREAMS": "2"}),
    (PK3, {"FSTAT_PACKED": "3", "FSTAT_CELL_BATCH": "6"}),
    (PK1, {"FSTAT_P2_TS": "128"}),                            # paired pass 2: four rows per CTA
    (PK1, {"FSTAT_P2_TS": "64", "FSTAT_CELL_BATCH": "7"}),    # two rows per CTA
    (TWO, {"FSTAT_PACKED": "0", "FSTAT_SHARE_CHIRP": "0"}),   # each lane its own spindown phases
    (TWO, {"FSTAT_TMA": "0"}),
    (TWO, {"FSTAT_P2_THREADS": "256"}),
    (TWO, {"FSTAT_PACKED": "0", "FSTAT_CELL_BATCH": "5", "FSTAT_STREAMS": "2"}),
    (TWO, FUSED),
    (TWO, {"FSTAT_FUSED": "1", "FSTAT_FUSED_BATCH": "3"}),
    (TWO, {"FSTAT_FUSED": "1", "FSTAT_FUSED_BATCH": "11", "FSTAT_STREAMS": "2"}),
    (TWO, {"FSTAT_FUSED": "1", "FSTAT_FUSED_TPI": "2", "FSTAT_FUSED_SLOTS": "3", "FSTAT_FUSED_AHEAD": "2"}),
    (TWO, {"FSTAT_FUSED": "1", "FSTAT_FUSED_TPI": "4", "FSTAT_FUSED_BATCH": "5"}),
])
def test_launch_shapes_match_bitwise(fs, base, env):
    """The queue-fed persistent kernel, the fused ticket-ordered launch and other
    tile / batch shapes against the two-launches-per-batch form of the same FFT
    engine.  Tiny workload (N_fft =
    2^13) and a two-sidereal-day band (2^18) with cell counts that leave a partial
    last batch."""
    for w in (S.workload(1, n_sky=9, n_spin=3), S.workload(3, n_sky=5, n_spin=3)):
        p0, rc0, ref, t0 = _run(fs, w, 8.0, base)
        p0.close()
        p1, rc1, got, t1 = _run(fs, w, 8.0, env)
        p1.close()
        assert rc0 == rc1 == fs.FSTAT_OK
        assert t0 == t1 and np.array_equal(ref, got)


@pytest.mark.parametrize("n,n_fft", [(2000, 1 << 12), (4096, 1 << 13), (7000, 1 << 14), (16000, 1 << 15),
                                     (30000, 1 << 16), (60000, 1 << 17), (86164, 1 << 18), (200000, 1 << 19)])
def test_engines_agree_on_every_bin(fs, n, n_fft):
    """The two-stage and the radix-8 FFT engines, every bin of every cell, at each
    transform length the two-stage engine serves: each is within 1e-4 max(F, 2)
    of the oracle, so they agree within twice that."""
    w0 = S.workload(1, n_sky=3, n_spin=2)
    b = S.make_band(n, 2.0, 5 + n, 1.0, w0.alpha, w0.delta, w0.fdot, [], n_fft=n_fft)
    w = S.Workload("engines", [b], w0.alpha, w0.delta, w0.fdot, 10.0, upsample=2)
    out = []
    for env in (R8, DEFAULT):
        p, rc, c, total = _run(fs, w, -1.0, env)
        p.close()
        assert rc == fs.FSTAT_OK and total == 6 * (n_fft // 2 - 1)
        out.append(c)
    a, b = out
    for key in ("band", "sky", "spin", "bin"):
        assert np.array_equal(a[key], b[key])
    assert np.all(np.abs(a["F"] - b["F"]) <= 2e-4 * np.maximum(np.maximum(a["F"], b["F"]), 2.0))


@pytest.mark.parametrize("n,n_fft,full,rows", [(30000, 1 << 16, False, "1"), (60000, 1 << 17, False, "1"),
                                               (43082, 1 << 17, True, "1"), (60000, 1 << 17, False, "0")])
def test_row_pairs_against_oracle_every_bin(fs, n, n_fft, full, rows):
    """The 256-point rows (N_fft = 2^16, 2^17) two per warp in packed arithmetic (the
    default) and in the scalar two-stage pass: every bin of every cell against the
    FP64 oracle at the FP32 tolerance, with the simple and the full (cross-term)
    statistic."""
    import oracle as O
    w0 = S.workload(1, n_sky=3, n_spin=2)
    b = S.make_band(n, 2.0, 77 + n, 1.0, w0.alpha, w0.delta, w0.fdot, [], n_fft=n_fft,
                    f_off=100 + (1 - 2 ** -5) * 3)
    w = S.Workload("row-pairs", [b], w0.alpha, w0.delta, w0.fdot, 10.0, upsample=2)
    env = {"FSTAT_PERSISTENT": "0", "FSTAT_P2_ROWS": rows}
    p, rc, c, total = _run(fs, w, -1.0, env, full=full)
    p.close()
    nb = n_fft // 2 - 1
    assert rc == fs.FSTAT_OK and total == 6 * nb
    prm = O.params(w.lat, w.gamma, w.upsample, 0.0, full, 0)
    cells = [(s, j) for s in range(3) for j in range(2)]
    ref = O.cells_F(b, prm, w.alpha, w.delta, w.fdot, np.array([x[0] for x in cells]),
                    np.array([x[1] for x in cells]), 0, 0, os.cpu_count() or 4)
    for i, (sk, sp) in enumerate(cells):
        sel = c[(c["sky"] == sk) & (c["spin"] == sp)]
        assert np.array_equal(sel["bin"], np.arange(1, nb + 1))
        err = np.abs(sel["F"] - ref[i]) / np.maximum(ref[i], 2.0)
        assert err.max() <= 1e-4, (n_fft, full, sk, sp, err.max())


def test_two_plans_in_two_threads(fs):
    """Two plans on two streams searched from two host threads at once (the way the
    benchmark overlaps one range's candidate drain with the next range's search):
    each returns bit for bit what one plan returns for its cell range."""
    import threading
    import torch
    w = S.workload(3, n_sky=12, n_spin=8)
    cells = w.n_sky * w.n_spin
    half = cells // 2
    p0, rc0, _, _ = _run(fs, w, w.thr_2F, DEFAULT)
    ref = []
    for lo, hi in ((0, half), (half, cells)):
        p0.search(lo, hi)
        ref.append(p0.candidates()[0])
    p0.close()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    plans = [fs.Plan(w.bands, w.alpha, w.delta, w.fdot, w.thr_2F, lat=w.lat, gamma=w.gamma,
                     upsample=w.upsample, form=fs.FP32_BATCHED, cand_capacity=1 << 22,
                     stream=st.cuda_stream) for st in streams]
    device = torch.cuda.current_device()
    errors = []

    def run(i, lo, hi):
        try:
            torch.cuda.set_device(device)
            for _ in range(3):               # plain, captured, replayed
                plans[i].search(lo, hi)
        except Exception as e:               # reported to the main thread
            errors.append(e)
    th = [threading.Thread(target=run, args=(0, 0, half)), threading.Thread(target=run, args=(1, half, cells))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors
    got = [pl.candidates()[0] for pl in plans]
    for pl in plans:
        pl.close()
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


def test_queue_cell_ranges(fs):
    """Ranges that start and end inside a sky position and a batch."""
    w = S.workload(1, n_sky=7, n_spin=5)
    p, rc, full, _ = _run(fs, w, 6.0, {"FSTAT_PERSISTENT": "1", "FSTAT_PERSIST_BATCH": "4"})
    parts = []
    for a, b in ((0, 3), (3, 17), (17, 35)):
        p.search(a, b)
        parts.append(p.candidates()[0])
    p.close()
    assert np.array_equal(np.concatenate(parts), full)


def test_withheld_completion_times_out_and_gpu_stays_usable(fs):
    w = S.workload(1, n_sky=8, n_spin=4)
    t0 = time.time()
    p, rc, _, _ = _run(fs, w, 20.0, {"FSTAT_PERSISTENT": "1", "FSTAT_TEST_WITHHOLD_ITEM": "0"})
    elapsed = time.time() - t0
    assert rc == fs.FSTAT_ERR_TIMEOUT
    assert elapsed < 30.0
    assert "wait" in p.error()
    assert p.search_status() == fs.FSTAT_ERR_STATE      # poisoned
    p.close()
    p, rc, c, total = _run(fs, w, 20.0)                 # a fresh plan works
    p.close()
    assert rc == fs.FSTAT_OK and total > 0


def test_fused_launch_withheld_completion_times_out(fs):
    """The fused launch with the pass-1 completion of cell 0 withheld (test hook):
    its pass-2 tiles give up after the bounded wait, every later wait sees the
    error flag, the search returns FSTAT_ERR_TIMEOUT and the GPU stays usable."""
    w = S.workload(1, n_sky=8, n_spin=4)
    t0 = time.time()
    p, rc, _, _ = _run(fs, w, 20.0, {"FSTAT_FUSED": "1", "FSTAT_TEST_WITHHOLD_ITEM": "0"})
    elapsed = time.time() - t0
    assert rc == fs.FSTAT_ERR_TIMEOUT
    assert elapsed < 30.0
    assert p.search_status() == fs.FSTAT_ERR_STATE
    p.close()
    p, rc, c, total = _run(fs, w, 20.0)
    p.close()
    assert rc == fs.FSTAT_OK and total > 0


def test_graph_replay_repeats_the_search(fs):
    """A search repeated over the same cell range is captured into a CUDA graph
    on its second run and replayed after that: identical candidates, the same
    kernel count per search, and a recapture when the range changes."""
    w = S.workload(3, n_sky=70, n_spin=8)
    p = fs.Plan(w.bands, w.alpha, w.delta, w.fdot, 25.0, lat=w.lat, gamma=w.gamma,
                upsample=w.upsample, form=fs.FP32_BATCHED, cand_capacity=1 << 22)
    p.set_timing(2)
    ref = None
    launches = []
    for rng in [(0, -1)] * 4 + [(8, 300)] * 3 + [(0, -1)] * 3:
        k0 = p.info()["kernel_launches"]
        assert p.search(*rng) == fs.FSTAT_OK
        launches.append((rng, p.info()["kernel_launches"] - k0))
        c, total = p.candidates()
        if rng == (0, -1):
            if ref is None:
                ref = c
            assert np.array_equal(c, ref)
        else:
            cell = c["sky"] * w.n_spin + c["spin"]
            assert np.all((cell >= 8) & (cell < 300))
            sel = ref[(ref["sky"] * w.n_spin + ref["spin"] >= 8) & (ref["sky"] * w.n_spin + ref["spin"] < 300)]
            assert np.array_equal(c, sel)
    full = {n for r, n in launches if r == (0, -1)}
    part = {n for r, n in launches if r == (8, 300)}
    assert len(full) == 1 and len(part) == 1
    stats = p.kernel_stats()
    assert any(v["timed_launches"] > 0 for v in stats.values())
    p.close()
    os.environ["FSTAT_GRAPH"] = "0"
    try:
        q = fs.Plan(w.bands, w.alpha, w.delta, w.fdot, 25.0, lat=w.lat, gamma=w.gamma,
                    upsample=w.upsample, form=fs.FP32_BATCHED, cand_capacity=1 << 22)
    finally:
        del os.environ["FSTAT_GRAPH"]
    for _ in range(3):
        q.search()
        assert np.array_equal(q.candidates()[0], ref)
    q.close()


def test_autotune_keeps_results(fs):
    """The autotuner times searches over a sample of cells and leaves the plan on
    its best launch shapes; the candidates stay within FP32 rounding of the
    default shapes' (exactly equal for the shapes that share the engine)."""
    w = S.workload(3, n_sky=40, n_spin=8)
    def plan():
        return fs.Plan(w.bands, w.alpha, w.delta, w.fdot, 25.0, lat=w.lat, gamma=w.gamma,
                       upsample=w.upsample, form=fs.FP32_BATCHED, cand_capacity=1 << 22)
    p0 = plan()
    p0.search()
    ref, _ = p0.candidates()
    p0.close()
    p = plan()
    t = p.autotune(64)
    assert t["engine"] in (1, 2, 3, 4) and t["pass2_threads"] in (32, 128, 256)
    assert t["cells_per_launch"] >= 1 and t["ms_per_cell"] > 0
    assert p.candidates()[1] == 0                      # tuning searches are discarded
    p.search()
    c, _ = p.candidates()
    p.close()
    # the default kernels (the paired rows in one- or four-row CTAs compute the same): bit for bit
    default = t["engine"] == 3 and t["pass2_threads"] in (32, 128) and t["pass2_bulk_copy"] == 1 and t["fused"] == 0
    if default:
        assert np.array_equal(c, ref)
    else:
        keys = ("sky", "spin", "bin")
        common = {tuple(x) for x in np.stack([ref[k] for k in keys], 1).tolist()} & \
                 {tuple(x) for x in np.stack([c[k] for k in keys], 1).tolist()}
        assert len(common) >= 0.99 * min(len(ref), len(c))


@pytest.mark.parametrize("env", [
    {"FSTAT_PERSISTENT": "1", "FSTAT_PERSIST_BATCH": "3"},     # warp-specialised persistent kernel
    {"FSTAT_FUSED": "1", "FSTAT_FUSED_BATCH": "4"},             # queue-fed persistent launch
    PK2,                                                        # both passes paired
    PK3,                                                        # pass 2 and pass-1 stage 1 paired
    {"FSTAT_P2_TS": "128"},                                     # paired pass 2, four rows per CTA
    TWO,                                                        # scalar two-stage passes
])
def test_queue_kernels_against_oracle_every_bin(fs, env):
    """Every bin of a few cells of a two-sidereal-day band (N = 86164, N_fft =
    2^18, with a band offset) in each non-default launch form, directly against
    the FP64 oracle at the FP32 tolerance (not only bitwise against the default)."""
    import oracle as O
    w0 = S.workload(1, n_sky=2, n_spin=2)
    b = S.make_band(86164, 2.0, 404, 1.0, w0.alpha, w0.delta, w0.fdot, [], n_fft=1 << 18,
                    f_off=100 + (1 - 2 ** -5) * 7)
    w = S.Workload("queue-oracle", [b], w0.alpha, w0.delta, w0.fdot, 10.0, upsample=2)
    p, rc, c, total = _run(fs, w, -1.0, env)
    p.close()
    nb = (1 << 17) - 1
    assert rc == fs.FSTAT_OK and total == 4 * nb
    prm = O.params(w.lat, w.gamma, w.upsample, 0.0, False, 0)
    cells = [(s, j) for s in range(2) for j in range(2)]
    ref = O.cells_F(b, prm, w.alpha, w.delta, w.fdot, np.array([x[0] for x in cells]),
                    np.array([x[1] for x in cells]), 0, 0, os.cpu_count() or 4)
    for i, (sk, sp) in enumerate(cells):
        sel = c[(c["sky"] == sk) & (c["spin"] == sp)]
        assert np.array_equal(sel["bin"], np.arange(1, nb + 1))
        err = np.abs(sel["F"] - ref[i]) / np.maximum(ref[i], 2.0)
        assert err.max() <= 1e-4, (env, sk, sp, err.max())
