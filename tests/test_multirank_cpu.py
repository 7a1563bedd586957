"""The N > 1 path of the benchmark on CPU: two gloo ranks, each taking its own
block of sky positions of an N-times larger grid (weak scaling, no data-path
collective), and the max-over-ranks timing reduction."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = bench.make_workload(world, rank)
        skies = list(zip(w.alpha.tolist(), w.delta.tolist()))
        gathered = [None] * world
        dist.all_gather_object(gathered, skies)
        t = bench.max_over_ranks(1.0 + rank, dist)
        out[rank] = (gathered, t, w.n_spin, len(w.bands))
        # the reference arm: only rank 0 works, the others return 0 at once
        if rank != 0:
            assert bench.run_reference(None, rank, world) == 0
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_sky_grid():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    from paper_1410_3677_gb300 import synth as S
    a, d = S.fibonacci_sky(4096 * world)
    gathered, t0, n_spin, n_bands = res[0]
    assert res[1][0] == gathered                      # every rank saw the same exchange
    assert t0 == res[1][1] == 2.0                     # max over ranks
    assert n_spin == 64 and n_bands == 1
    blocks = [np.array(g) for g in gathered]
    assert all(b.shape == (4096, 2) for b in blocks)  # fixed work per rank
    union = np.concatenate(blocks)
    ref = np.stack([a, d], axis=1)
    key = lambda x: np.lexsort((x[:, 1], x[:, 0]))
    assert np.array_equal(union[key(union)], ref[key(ref)])   # disjoint cover of the grid
