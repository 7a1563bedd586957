"""The multi-rank output of Sect. 3.2 on the CPU: two gloo ranks each search their
round-robin share of the sky grid (the FP64 oracle stands in for each rank's GPU
search here: only the exchange is under test), all-gather their candidate counts,
write their records into disjoint slices of one joint file at the exclusive-scan
offsets, and the joint file equals a single-rank search of the whole grid,
record for record once both are put in grid order."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1410_3677_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _search_records(w, skies):
    """Candidates of the listed sky positions, as the paper's five doubles, with
    the global sky index for ordering."""
    import oracle as O
    prm = O.params(w.lat, w.gamma, w.upsample, 0.0, False, 0)
    c, _ = O.search(w.bands, prm, w.alpha[skies], w.delta[skies], w.fdot, w.thr_2F, nthreads=2)
    b = w.bands[0]
    r = np.empty(c.size, shard.RECORD_DTYPE)
    gsky = skies[c["sky"]]
    r["alpha"], r["delta"] = w.alpha[gsky], w.delta[gsky]
    r["freq"] = b.f_off + c["bin"] / (b.n_fft * b.dt)
    r["fdot"] = w.fdot[c["spin"]]
    r["F"] = c["F"]
    return r, gsky, c["spin"], c["bin"]


def _rank_main(rank, world, port, path, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    from paper_1410_3677_gb300 import synth as S
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = S.workload(1, n_sky=10, n_spin=4)
        skies = shard.sky_share(w.n_sky, world, rank)
        rec, gsky, spin, bins = _search_records(w, skies)
        off, total = shard.write_joint(path, rec)
        out[rank] = (off, total, rec.size, np.stack([gsky, spin, bins], 1).tolist())
    finally:
        dist.destroy_process_group()


def test_offsets_are_the_exclusive_scan():
    off, total = shard.exclusive_offsets([3, 0, 5, 2])
    assert off.tolist() == [0, 3, 3, 8] and total == 10
    with pytest.raises(ValueError):
        shard.exclusive_offsets([1, -1])


def test_sky_shares_cover_the_grid_once():
    for mode in ("round_robin", "block"):
        parts = [shard.sky_share(37, 4, r, mode) for r in range(4)]
        allv = np.sort(np.concatenate(parts))
        assert np.array_equal(allv, np.arange(37))
        assert max(p.size for p in parts) == -(-37 // 4)     # P_size = ceil(N_sky / N_tasks)


def test_two_gloo_ranks_write_one_joint_file(tmp_path):
    world = 2
    port = _free_port()
    path = str(tmp_path / "candidates_joint.bin")
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, path, out), nprocs=world, join=True)
        res = dict(out)
    from paper_1410_3677_gb300 import synth as S
    w = S.workload(1, n_sky=10, n_spin=4)
    ref, gsky, spin, bins = _search_records(w, np.arange(w.n_sky))
    got = shard.read_joint(path)
    (o0, t0, n0, k0), (o1, t1, n1, k1) = res[0], res[1]
    assert t0 == t1 == got.size == ref.size > 0
    assert (o0, o1) == (0, n0) and n0 + n1 == t0          # disjoint slices in rank order
    # rank slices in grid order equal the single-rank search record for record
    keys = np.array(k0 + k1, dtype=np.int64)
    order = np.lexsort((keys[:, 2], keys[:, 1], keys[:, 0]))
    ref_keys = np.stack([gsky, spin, bins], 1)
    assert np.array_equal(keys[order], ref_keys)
    assert got[order].tobytes() == ref.tobytes()


def test_eq2_interpolation_by_hand():
    """Eq. 2 on a three-row table: S(150) between (100, 200) and (200, 600) is
    200 + 4 * 50 = 400; at a table frequency it is that row's S; beyond the table
    the end segment continues (S(350) = 600 + 1 * 50 = 650)."""
    tf, ts = [100.0, 200.0, 300.0], [200.0, 600.0, 700.0]
    got = shard.eq2_tasks([150.0, 200.0, 300.0, 350.0, 50.0], tf, ts)
    assert np.allclose(got, [400.0, 600.0, 700.0, 750.0, 0.0], rtol=0, atol=1e-9)
    with pytest.raises(ValueError):
        shard.eq2_tasks(1.0, [1.0, 1.0], [2.0, 3.0])


def _queue_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import time
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        store = dist.distributed_c10d._get_default_store()
        # 16 uneven bands (1..4 sidereal days: n_fft 2^17..2^19) of 64 sky x 16 spindowns
        days = [1, 3, 2, 4, 1, 2, 4, 3, 2, 1, 4, 2, 3, 1, 2, 4]
        nfft = {1: 1 << 17, 2: 1 << 18, 3: 1 << 19, 4: 1 << 19}
        items, costs = shard.CostQueue.band_items([(64, nfft[d], 16) for d in days], 16)
        q = shard.CostQueue(items, costs)
        dist.barrier()
        mine = []
        while True:
            got = q.claim(store)
            if got is None:
                break
            mine.append(got)
            time.sleep(0.001 * (1 + rank))   # uneven speed: the faster rank takes more
        out[rank] = (mine, q.items, q.costs)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_cost_queue_hands_out_every_item_once_most_expensive_first():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_queue_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    mine0, items, costs = res[0]
    mine1 = res[1][0]
    assert res[1][1] == items
    pos = sorted([p for p, _ in mine0] + [p for p, _ in mine1])
    assert pos == list(range(len(items)))                     # each item exactly once
    assert sorted([it for _, it in mine0] + [it for _, it in mine1]) == sorted(items)
    assert all(costs[i] >= costs[i + 1] for i in range(len(costs) - 1))   # decreasing cost
    assert all(p0 < p1 for (p0, _), (p1, _) in zip(mine0, mine0[1:]))     # each rank in queue order
