"""Sharding of a search over several GPUs (one process per GPU) and the joint
candidate output of Sect. 3.2.

Sky positions are independent (Sect. 3: the sky loops are the parallelised
dimension), so each rank searches its own share of the sky grid with its own plan
and no data-path collective.  The only exchange is the one the paper's parallel
output uses: every rank's candidate count is all-gathered, each rank's offset is
the exclusive prefix sum of the counts of the lower ranks, and every rank writes
its records into its own slice of one joint file (or one global array) -- the
MPI_Allgather-then-collective-write pattern of Sect. 3.2.  The collective runs
through torch.distributed (NCCL between GPUs, gloo on the CPU); no rank reads
another GPU's memory.
"""
from __future__ import annotations

import os
from typing import Optional, Tuple

import numpy as np

# The paper's candidate: five doubles (sky position, frequency, spindown, F), Sect. 2.
RECORD_DTYPE = np.dtype([("alpha", "<f8"), ("delta", "<f8"), ("freq", "<f8"), ("fdot", "<f8"),
                         ("F", "<f8")])
HEADER_BYTES = 16            # magic + total record count (int64 each)
MAGIC = 0x4653544154433031   # "FSTATC01"


def sky_share(n_sky: int, world: int, rank: int, mode: str = "round_robin") -> np.ndarray:
    """Indices of the sky positions of `rank`: round-robin as the paper's farm
    distributes them (Sect. 3, P_size = ceil(N_sky / N_tasks) each), or one
    contiguous block per rank (`mode="block"`)."""
    if not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    if mode == "round_robin":
        return np.arange(rank, n_sky, world, dtype=np.int64)
    if mode == "block":
        per = -(-n_sky // world)
        return np.arange(rank * per, min(n_sky, (rank + 1) * per), dtype=np.int64)
    raise ValueError(f"unknown mode {mode!r}")


def exclusive_offsets(counts) -> Tuple[np.ndarray, int]:
    """Offsets of every rank's slice: the exclusive prefix sum of the counts."""
    c = np.asarray(counts, dtype=np.int64)
    if np.any(c < 0):
        raise ValueError("negative count")
    off = np.zeros_like(c)
    if c.size > 1:
        np.cumsum(c[:-1], out=off[1:])
    return off, int(c.sum())


def candidate_offsets(n_local: int, group=None, device: str = "cpu") -> Tuple[int, int, np.ndarray]:
    """All-gather of the ranks' candidate counts (one int64 each) and this rank's
    offset: returns (offset, total, counts)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mine = torch.tensor([int(n_local)], dtype=torch.int64, device=device)
    out = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(world)]
    dist.all_gather(out, mine, group=group)
    counts = np.array([int(t.item()) for t in out], dtype=np.int64)
    off, total = exclusive_offsets(counts)
    return int(off[rank]), total, counts


def to_records(c: np.ndarray) -> np.ndarray:
    """The five doubles of the paper's candidate from the library's candidate array."""
    r = np.empty(c.size, RECORD_DTYPE)
    for k in RECORD_DTYPE.names:
        r[k] = c[k]
    return r


def write_joint(path: str, records: np.ndarray, group=None, device: str = "cpu") -> Tuple[int, int]:
    """Every rank writes its records into its slice of one joint file: a 16-byte
    header (magic, total count) written by rank 0, then the records of rank 0,
    rank 1, ... in rank order.  Returns (offset, total) in records."""
    import torch.distributed as dist
    records = np.ascontiguousarray(records, dtype=RECORD_DTYPE)
    off, total, _ = candidate_offsets(records.size, group, device)
    rank = dist.get_rank(group)
    if rank == 0:                 # create the file at its final size
        with open(path, "wb") as fh:
            fh.write(np.array([MAGIC, total], dtype=np.int64).tobytes())
            fh.truncate(HEADER_BYTES + total * RECORD_DTYPE.itemsize)
    dist.barrier(group)
    if records.size:
        fd = os.open(path, os.O_WRONLY)
        try:
            buf = records.tobytes()
            pos = HEADER_BYTES + off * RECORD_DTYPE.itemsize
            done = 0
            while done < len(buf):
                done += os.pwrite(fd, buf[done:], pos + done)
        finally:
            os.close(fd)
    dist.barrier(group)
    return off, total


def read_joint(path: str) -> np.ndarray:
    """The records of a joint candidate file."""
    with open(path, "rb") as fh:
        head = np.frombuffer(fh.read(HEADER_BYTES), dtype=np.int64)
        if head.size != 2 or int(head[0]) != MAGIC:
            raise ValueError(f"{path}: not a joint candidate file")
        data = np.frombuffer(fh.read(), dtype=RECORD_DTYPE)
    if data.size != int(head[1]):
        raise ValueError(f"{path}: {data.size} records, header says {int(head[1])}")
    return data.copy()


def gather_global(records: np.ndarray, out: Optional[np.ndarray], group=None,
                  device: str = "cpu") -> Tuple[int, int]:
    """The same exchange for an in-memory global array that every rank can
    address (e.g. one array in shared host memory): writes this rank's records at
    its offset; returns (offset, total)."""
    off, total, _ = candidate_offsets(records.size, group, device)
    if out is not None and records.size:
        if out.size < total:
            raise ValueError("global array smaller than the total")
        out[off:off + records.size] = records
    return off, total


# --------------------------------------------------------------------------- cost model
def eq2_tasks(f, table_f, table_S) -> np.ndarray:
    """Eq. 2 (Sect. 3.1.1): the number of parallel tasks S(f) of a band at frequency
    f, by first-order spline interpolation S(f) = a f + b between the two table
    frequencies f1 < f2 that enclose f, a = (S2 - S1)/(f2 - f1), b = S1 - a f1
    (the table is the paper's cpuperband.dat: frequencies and task counts).  Beyond
    the table the end segment is extended."""
    tf = np.asarray(table_f, dtype=np.float64)
    ts = np.asarray(table_S, dtype=np.float64)
    if tf.ndim != 1 or tf.size < 2 or tf.size != ts.size or np.any(np.diff(tf) <= 0):
        raise ValueError("need >= 2 strictly increasing table frequencies with one S each")
    fv = np.atleast_1d(np.asarray(f, dtype=np.float64))
    j = np.clip(np.searchsorted(tf, fv, side="right") - 1, 0, tf.size - 2)
    f1, f2, s1, s2 = tf[j], tf[j + 1], ts[j], ts[j + 1]
    a = (s2 - s1) / (f2 - f1)
    b = s1 - a * f1
    return a * fv + b


def search_cost(n_cells: int, n_fft: int) -> float:
    """Relative GPU cost of searching n_cells cells of a band with transforms of
    n_fft points: the FFT work, cells x n_fft log2 n_fft."""
    return float(n_cells) * float(n_fft) * float(np.log2(n_fft))


class CostQueue:
    """Work items (band, first sky, last sky + 1) ordered by decreasing estimated
    cost and handed out to the ranks through an atomic counter in the
    torch.distributed store (the device-side work queue's role, across
    processes): the most expensive items start first, every item is claimed by
    exactly one rank, and a rank that finishes early takes the next one.  Costs
    come from Eq. 2 (a cpuperband-style table) or from search_cost."""

    def __init__(self, items, costs, key: str = "fstat_cost_queue"):
        if len(items) != len(costs):
            raise ValueError("one cost per item")
        order = sorted(range(len(items)), key=lambda i: (-float(costs[i]), i))
        self.items = [tuple(items[i]) for i in order]
        self.costs = [float(costs[i]) for i in order]
        self.key = key

    @staticmethod
    def band_items(bands_cells, sky_block: int):
        """(band, s0, s1) items of sky blocks for bands of (n_sky, n_fft, n_spin)."""
        items, costs = [], []
        for bi, (n_sky, n_fft, n_spin) in enumerate(bands_cells):
            for s0 in range(0, n_sky, sky_block):
                s1 = min(n_sky, s0 + sky_block)
                items.append((bi, s0, s1))
                costs.append(search_cost((s1 - s0) * n_spin, n_fft))
        return items, costs

    def claim(self, store) -> Optional[Tuple[int, tuple]]:
        """The next unclaimed item as (queue position, item), or None when the queue
        is drained.  `store` is a torch.distributed Store shared by the ranks."""
        t = int(store.add(self.key, 1)) - 1
        if t >= len(self.items):
            return None
        return t, self.items[t]
