#!/usr/bin/env python3
"""Throughput of the all-sky F-statistic search on GB300: F-statistic evaluations
per second (sky x spindown x searched bin), FP32 batched form, with the plain
FP64 form, the roofline fraction of the dominant kernel, an end-to-end number
through the C ABI with host buffers, and the FP64 CPU oracle as a baseline.

One step = one fstat_search over the whole grid: per band the noise variance and
the FFT upsample, per sky position the geometry / resampling / phase
demodulation, per cell the spindown demodulation, two zero-padded FFTs, F per
bin, threshold and candidate compaction.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank searches its own block of sky positions of an N-times
larger grid (weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "F-stat evals/s (sky×spindown×bin) on 1 GB300: FP32-batched vs FP64 plain, % roofline"
UNIT = "F-evals/s"
SMS, FP32_LANES = 152, 128          # GB300: SMs, FP32 lanes per SM
L2_BYTES = 129 << 20


def fp32_peak_tflops(mhz: float) -> float:
    return SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# ----------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# ----------------------------------------------------------------------------- workload
def make_workload(world: int, rank: int, n_sky: int = 0):
    """The precision workload: one band of N = 86164 samples (two sidereal days at
    2 s), 4096 sky positions x 64 spindowns in [-1e-8, 0] Hz/s, N_fft = 2^18,
    16 injected signals, 2F > 30.  Under N ranks, rank r takes sky block r of a
    4096*N-point Fibonacci grid."""
    from paper_1410_3677_gb300 import synth as S
    w = S.workload(3)
    if n_sky:                               # a smaller grid of the same data (profiling)
        w.alpha, w.delta = w.alpha[:n_sky].copy(), w.delta[:n_sky].copy()
        for b in w.bands:
            b.injections = [i for i in b.injections if i.sky < n_sky]
    if world > 1:
        a, d = S.fibonacci_sky(4096 * world)
        w.alpha, w.delta = a[rank::world].copy(), d[rank::world].copy()
    return w


def max_over_ranks(x: float, dist, device: str = "cpu") -> float:
    """The slowest rank's time (the job's time under weak scaling)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sample_cells(w, n_cells):
    """A bounded, deterministic sample of cells: whole sky positions (all
    spindowns) spread over the grid."""
    n_sky = max(1, math.ceil(n_cells / w.n_spin))
    skies = np.linspace(0, w.n_sky - 1, n_sky).astype(np.int64)
    cs = np.repeat(skies, w.n_spin)[:n_cells]
    cp = np.tile(np.arange(w.n_spin), n_sky)[:n_cells]
    return cs, cp


def oracle_rate(w, target_s=30.0):
    """FP64 CPU oracle F-evals/s on a bounded sample of the workload's cells: the
    sample grows (whole sky positions, all host threads) until one run takes at
    least a third of target_s; that run is the number reported."""
    import oracle as O
    prm = O.params(w.lat, w.gamma, w.upsample, 0.0, False, 0)
    threads = os.cpu_count() or 1
    b = w.bands[0]
    nb = b.n_fft // 2 - 1
    n = threads
    while True:
        cs, cp = sample_cells(w, n)
        t0 = time.perf_counter()
        O.cells_F(b, prm, w.alpha, w.delta, w.fdot, cs, cp, nthreads=threads)
        el = time.perf_counter() - t0
        if el >= target_s / 3 or n >= w.n_sky * w.n_spin:
            break
        grow = min(8.0, max(2.0, target_s / max(el, 1e-3)))
        n = min(w.n_sky * w.n_spin, int(math.ceil(n * grow / threads)) * threads)
    # one thread: the first sky position's cells, about a second
    cs1, cp1 = sample_cells(w, w.n_spin)
    t0 = time.perf_counter()
    O.cells_F(b, prm, w.alpha, w.delta, w.fdot, cs1, cp1, nthreads=1)
    el1 = time.perf_counter() - t0
    return {"value": cs.size * nb / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{cs.size} cells ({len(set(cs.tolist()))} sky positions x up to "
                      f"{w.n_spin} spindowns) of the {w.n_sky}x{w.n_spin} grid, N_fft=2^18, "
                      f"all {nb} bins, one run of {el:.1f} s",
            "one_thread": {"value": cs1.size * nb / el1, "unit": UNIT,
                           "sample": f"{cs1.size} cells of one sky position, one run of {el1:.2f} s"}}


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_1410_3677_gb300 import synth as S
    w = make_workload(1, 0)
    import oracle as O
    prm = O.params(w.lat, w.gamma, w.upsample, 0.0, False, 0)
    threads = os.cpu_count() or 1
    nb = w.bands[0].n_fft // 2 - 1
    # size each step to a few seconds of CPU work
    cs, cp = sample_cells(w, threads)
    t0 = time.perf_counter()
    O.cells_F(w.bands[0], prm, w.alpha, w.delta, w.fdot, cs, cp, nthreads=threads)
    per_cell = (time.perf_counter() - t0) / cs.size
    budget = 150.0 / max(args.steps + args.warmup, 1)
    n = max(threads, int(budget / per_cell) // threads * threads)
    cs, cp = sample_cells(w, n)
    for _ in range(args.warmup):
        O.cells_F(w.bands[0], prm, w.alpha, w.delta, w.fdot, cs[:threads], cp[:threads],
                  nthreads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.cells_F(w.bands[0], prm, w.alpha, w.delta, w.fdot, cs, cp, nthreads=threads)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = cs.size * nb * args.steps / tot
    sample = (f"{cs.size} cells per step ({cs.size // w.n_spin} sky positions x {w.n_spin} "
              f"spindowns) of the 4096x64 grid, all {nb} bins")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "precision: N=86164, N_fft=2^18, 4096 sky x 64 spindown",
                       "form": "fp64 cpu oracle", "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
# Files that define the FFT/F-statistic kernels (host orchestration excluded): a
# change to any of them voids the recorded DRAM traffic.
KERNEL_SOURCES = ("fft_engine.cuh", "fft_engine2.cuh", "passes.cuh", "passes2.cuh", "packed.cuh",
                  "passes3.cuh", "search_launch.cuh", "search_f32.cu", "search_f64.cu", "geometry.cu",
                  "search_persistent.cu", "sync_ptx.cuh", "fstat_internal.h")


def traffic_record(kernel_name, flops_per_launch):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the
    current kernel source and on launches of the same size (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except OSError:
        return None
    k = rec.get(kernel_name)
    if not k or k.get("source_hash") != source_hash() or k.get("flops_per_launch") != flops_per_launch:
        return None
    return k.get("dram_bytes_per_launch")


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1410_3677_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _timed(stream, fn, flush=None):
    """Milliseconds of fn() on the plan's stream, CUDA events, L2 flushed first."""
    import torch
    if flush is not None:
        with torch.cuda.stream(stream):
            flush.add_(1.0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def run_banded(args, stream, flush, peak):
    """The batching workload: 16 float32 bands of 1-4 sidereal days (N = 43082 ..
    172328, N_fft 2^17 .. 2^19, sigma per band, f_off = 100 + (1 - 2^-5) b), 512 sky
    x 16 spindowns per band, 2F > 30, one plan.  Aggregate: whole searches; per
    band: searches of the band's cell range.  Roofline: the bands' FFT FLOP
    (2 x 5 N log2 N per cell) over the time, against the FP32 peak."""
    from paper_1410_3677_gb300 import fstat
    from paper_1410_3677_gb300 import synth as S
    w = S.workload(4)
    plan = fstat.Plan(w.bands, w.alpha, w.delta, w.fdot, w.thr_2F, lat=w.lat, gamma=w.gamma,
                      upsample=w.upsample, form=fstat.FP32_BATCHED, cand_capacity=1 << 26,
                      stream=stream.cuda_stream)
    per_band_cells = w.n_sky * w.n_spin
    flop = [per_band_cells * 2 * 5 * b.n_fft * math.log2(b.n_fft) for b in w.bands]
    evals = [per_band_cells * (b.n_fft // 2 - 1) for b in w.bands]
    tuning = None if args.no_autotune else plan.autotune(4096)   # launch shapes on the first cells
    for _ in range(2):
        plan.search()                        # the second search captures the graph
    ms = [_timed(stream, plan.search, flush) for _ in range(max(2, min(args.steps, 5)))]
    agg_ms = statistics.mean(ms)
    bands = []
    for bi, b in enumerate(w.bands):
        lo, hi = bi * per_band_cells, (bi + 1) * per_band_cells
        plan.search(lo, hi)
        bms = min(_timed(stream, lambda: plan.search(lo, hi), flush) for _ in range(2))
        bands.append({"band": bi, "n": int(b.n), "n_fft": int(b.n_fft), "cells": per_band_cells,
                      "ms": round(bms, 4), "f_evals_per_s": evals[bi] / (bms / 1e3),
                      "roofline_frac": round(flop[bi] / (bms / 1e3) / 1e12 / peak, 4)})
    _, n_total = plan.candidates(cap=0)
    plan.close()
    return {"workload": w.name, "n_bands": len(w.bands), "n_cells": per_band_cells * len(w.bands),
            "value": sum(evals) / (agg_ms / 1e3), "unit": UNIT, "ms_per_search": round(agg_ms, 3),
            "searches": len(ms), "candidates": int(n_total), "tuning": tuning,
            "roofline": {"bound": "alu", "achieved": round(sum(flop) / (agg_ms / 1e3) / 1e12, 3),
                         "peak": round(peak, 2), "unit": "TFLOP/s",
                         "frac": round(sum(flop) / (agg_ms / 1e3) / 1e12 / peak, 4),
                         "basis": "2 x 5 N log2 N FLOP per cell over the bands' transform lengths"},
            "per_band": bands,
            "note": "one plan over all bands, launch shapes autotuned on the first 4096 cells; bands "
                    "run one after another, each as launch pairs over sky batches, the search replayed "
                    "as a CUDA graph (L2 flushed before each timed search)"}


def run_large(args, stream, flush, peak):
    """The large grid: one band of N = 86164, N_fft = 2^18, 65536 sky x 256 spindown
    (16.8 M cells), 64 injections, 2F > 30, searched once as 256 resumable cell
    ranges of 256 sky positions, every range's candidates drained to the host
    (device sort, copy, expansion).  Two plans on two streams take the ranges in
    turn, so that the drain of one range runs on the host (and its sort and copy
    on the other stream) while the next range is searched: the sustained rate is
    the wall time of all searches and all drains.  Beside it the plain FP64 form
    on a 1024 x 16 subgrid."""
    from paper_1410_3677_gb300 import fstat
    from paper_1410_3677_gb300 import synth as S
    import torch
    w = S.workload(5)
    b = w.bands[0]
    streams = [stream, torch.cuda.Stream()]
    plans = [fstat.Plan(w.bands, w.alpha, w.delta, w.fdot, w.thr_2F, lat=w.lat, gamma=w.gamma,
                        upsample=w.upsample, form=fstat.FP32_BATCHED, cand_capacity=1 << 27,
                        stream=st.cuda_stream) for st in streams]
    cells = w.n_sky * w.n_spin
    ranges = 256
    step = cells // ranges
    for pl in plans:
        pl.search(0, w.n_spin)               # warm-up on one sky position
    out = None
    n_cand = 0
    dev_ms = [0.0]
    drain_s = 0.0
    max_range = 0

    def drain(pl):
        nonlocal out, n_cand, max_range
        _, nt = pl.candidates(cap=0)
        if out is None or out.size < nt:
            out = np.empty(nt + nt // 4 + 1024, fstat.CAND_DTYPE)
        c, nt = pl.candidates(out=out)
        n_cand += int(nt)
        max_range = max(max_range, int(nt))

    device = torch.cuda.current_device()

    def search(i, lo, hi):
        torch.cuda.set_device(device)        # the CUDA device is per host thread
        dev_ms[0] += _timed(streams[i], lambda: plans[i].search(lo, hi))

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in range(ranges):
        lo, hi = r * step, cells if r == ranges - 1 else (r + 1) * step
        th = threading.Thread(target=search, args=(r % 2, lo, hi))
        th.start()
        if r > 0:                            # the previous range, while this one runs
            td = time.perf_counter()
            drain(plans[(r - 1) % 2])
            drain_s += time.perf_counter() - td
        th.join()
    td = time.perf_counter()
    drain(plans[(ranges - 1) % 2])
    drain_s += time.perf_counter() - td
    wall = time.perf_counter() - t0
    for pl in plans:
        pl.close()
    dev_ms = dev_ms[0]
    nb = b.n_fft // 2 - 1
    flop_cell = 2 * 5 * b.n_fft * math.log2(b.n_fft)
    sub_sky, sub_spin = 1024, 16
    spins = np.linspace(0, w.n_spin - 1, sub_spin).round().astype(np.int64)
    p64 = fstat.Plan(w.bands, w.alpha[:sub_sky], w.delta[:sub_sky], w.fdot[spins], w.thr_2F,
                     lat=w.lat, gamma=w.gamma, upsample=w.upsample, form=fstat.FP64_PLAIN,
                     cand_capacity=1 << 24, stream=stream.cuda_stream)
    p64.search(0, sub_spin)
    ms64 = _timed(stream, p64.search)
    ev64 = p64.info()["f_evals"]
    p64.close()
    fp64 = ev64 / (ms64 / 1e3)
    sustained = cells * nb / wall
    return {"workload": w.name, "n_cells": cells, "value": sustained, "unit": UNIT,
            "wall_s": round(wall, 3), "device_s": round(dev_ms / 1e3, 3), "ranges": ranges,
            "drain_s": round(drain_s, 3), "candidates_streamed": n_cand,
            "max_candidates_per_range": max_range,
            "device_rate": cells * nb / (dev_ms / 1e3),
            "roofline": {"bound": "alu", "achieved": round(cells * flop_cell / wall / 1e12, 3),
                         "peak": round(peak, 2), "unit": "TFLOP/s",
                         "frac": round(cells * flop_cell / wall / 1e12 / peak, 4),
                         "basis": "2 x 5 N log2 N FLOP per cell over the sustained wall time"},
            "fp64_plain": {"value": fp64, "unit": UNIT, "dtype": "f64",
                           "sample": f"{sub_sky} sky x {sub_spin} spindown subgrid (spindowns spread "
                                     f"over the range), one cell per launch pair",
                           "roofline_frac": round(flop_cell * ev64 / nb / (ms64 / 1e3) / 1e12 / peak, 6)},
            "speedup_vs_fp64_plain": sustained / fp64,
            "note": "wall time of the 256 range searches and their candidate drains to the host "
                    "(72-byte candidates: sky, frequency, spindown, F and indices); two plans take "
                    "the ranges in turn, each range drained while the next is searched"}


def run_ours(args, rank, world, dist):
    import torch
    from paper_1410_3677_gb300 import fstat
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    w = make_workload(world, rank, args.n_sky)
    stream = torch.cuda.Stream()
    nb_total = w.f_evals()

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---------------------------------------------------------------- device-resident value
    plan = fstat.Plan(w.bands, w.alpha, w.delta, w.fdot, w.thr_2F, lat=w.lat, gamma=w.gamma,
                      upsample=w.upsample, form=fstat.FP32_BATCHED, cand_capacity=args.cand_capacity,
                      stream=stream.cuda_stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    tuning = None
    if not args.no_autotune:                 # launch shapes picked on one sky batch of cells
        tuning = plan.autotune(min(64 * w.n_spin, w.n_sky * w.n_spin))
    plan.set_timing(args.sample_every)       # the warm-up searches capture the launch graph
    for _ in range(args.warmup):
        plan.search()
    plan.set_timing(args.sample_every)       # statistics of the timed steps only
    launches0 = plan.info()["kernel_launches"]
    clocks = Clocks(dev)
    torch.cuda.synchronize()
    barrier()
    clocks.start()
    t_wall0 = time.perf_counter()
    step_ms = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.add_(1.0)                       # evict L2 between steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.search()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier()
    clk = clocks.stop()
    launches = plan.info()["kernel_launches"] - launches0
    kstats = plan.kernel_stats()
    cands, n_total = plan.candidates()
    plan.close()
    tot_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    value = nb_total * world * args.steps / (tot_ms / 1e3)

    # ---------------------------------------------------------------- roofline of the dominant kernel
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    dom = max(((k, v) for k, v in kstats.items() if v["timed_launches"] > 0),
              key=lambda kv: kv[1]["timed_ms"] / kv[1]["timed_launches"] * kv[1]["launches"])
    dname, dv = dom
    avg_ms = dv["timed_ms"] / dv["timed_launches"]
    achieved = dv["flops_per_launch"] / (avg_ms / 1e3) / 1e12
    peak = fp32_peak_tflops(sm_max)
    tot_local = sum(step_ms)
    shares = {k: round(v["timed_ms"] / v["timed_launches"] * v["launches"] / tot_local, 4)
              if v["timed_launches"] else None for k, v in kstats.items()}
    roofline = {"bound": "alu", "kernel": dname, "achieved": round(achieved, 3),
                "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "traffic": traffic_record(dname, dv["flops_per_launch"]),
                "peak_basis": f"{SMS} SMs x {FP32_LANES} FP32 lanes x 2 flop/FMA x {sm_max:.0f} MHz (max SM clock)",
                "flops_per_launch": dv["flops_per_launch"], "avg_launch_ms": round(avg_ms, 5),
                "timed_launches": dv["timed_launches"], "kernel_time_share": shares}
    if clk and clk.get("sm_mhz"):
        roofline["frac_at_measured_clock"] = round(achieved / fp32_peak_tflops(clk["sm_mhz"]), 4)
    # the path's roofline per cell: the slower of its FFT FLOP at the measured FP32
    # FMA rate, its inter-pass scratch bytes at the measured L2 copy rate and its
    # algorithmic HBM bytes at the measured HBM copy rate
    fma_tf = fstat.measure_fp32_fma(stream.cuda_stream)
    l2_gbs = fstat.measure_l2_copy(32 << 20, stream.cuda_stream)
    # the same fraction against the FFMA rate measured on this device (the derived
    # peak above rests on the SM count and lanes per SM)
    roofline["frac_vs_measured_fma"] = round(achieved / fma_tf, 4)
    roofline["measured_fma_tflops"] = round(fma_tf, 2)
    hbm_gbs = float(peaks.get("hbm_gbs", 6800.0))
    cells = w.n_sky * w.n_spin * len(w.bands)
    nfft = w.bands[0].n_fft
    flop_cell = 2 * 5 * nfft * math.log2(nfft)
    l2_cell = 2 * 2 * nfft * 8
    hbm_cell = 16.0 * w.bands[0].n / w.n_spin + 16.0 * n_total / cells
    terms = {"fft_flop_us": flop_cell / (fma_tf * 1e12) * 1e6,
             "l2_scratch_us": l2_cell / (l2_gbs * 1e9) * 1e6,
             "hbm_inputs_us": hbm_cell / (hbm_gbs * 1e9) * 1e6}
    t_cell = tot_ms / 1e3 / args.steps / cells * 1e6
    roof_us = max(terms.values())
    logn = int(round(math.log2(nfft)))
    cells_per_launch = dv["flops_per_launch"] / (2 * 5 * nfft * (logn - logn // 2))
    tr1 = traffic_record("fft_pass1_f32", dv["flops_per_launch"])
    tr2 = traffic_record("fft_pass2_fstat_f32", dv["flops_per_launch"])
    dram_us = ((tr1 + tr2) / cells_per_launch) / (hbm_gbs * 1e9) * 1e6 if tr1 and tr2 else None
    roofline["path"] = {"per_cell_us": round(t_cell, 4), "roofline_us": round(roof_us, 4),
                        "frac": round(roof_us / t_cell, 4),
                        "terms_us": {k: round(v, 4) for k, v in terms.items()},
                        "fp32_fma_measured_tflops": round(fma_tf, 2), "l2_copy_measured_gbs": round(l2_gbs, 1),
                        "hbm_gbs": hbm_gbs,
                        "scratch_dram_us_as_run": round(dram_us, 4) if dram_us else None,
                        "basis": "2 transforms x 5 N log2 N FLOP; scratch written and read once (2 x 2 x N x 8 B) "
                                 "through L2; HBM: the sky's w (16 B per sample) shared by its spindowns + 16 B "
                                 "per candidate; the as-run DRAM term uses the measured traffic of both passes "
                                 "(the scratch of a launch is larger than L2 and reaches DRAM)"}

    # ---------------------------------------------------------------- plain FP64 form on a subgrid
    fp64 = None
    if not args.skip_fp64:
        sub = 64
        p64 = fstat.Plan(w.bands, w.alpha[:sub], w.delta[:sub], w.fdot, w.thr_2F, lat=w.lat,
                         gamma=w.gamma, upsample=w.upsample, form=fstat.FP64_PLAIN,
                         cand_capacity=1 << 22, stream=stream.cuda_stream)
        p64.search(0, w.n_spin)           # warm-up on one sky position
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p64.search()
        e1.record(stream)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1)
        ev64 = p64.info()["f_evals"]
        p64.close()
        fp64 = {"value": ev64 / (ms64 / 1e3), "unit": UNIT, "dtype": "f64",
                "sample": f"{sub} sky x {w.n_spin} spindown subgrid of the same workload, "
                          f"one cell per launch pair"}

    # ---------------------------------------------------------------- interbinning form, same grid
    interbin = None
    if not args.skip_interbin:
        pib = fstat.Plan(w.bands, w.alpha, w.delta, w.fdot, w.thr_2F, lat=w.lat, gamma=w.gamma,
                         upsample=w.upsample, form=fstat.FP32_BATCHED,
                         cand_capacity=args.cand_capacity, stream=stream.cuda_stream, interbin=True)
        for _ in range(2):
            pib.search()                      # the second run captures the graph
        ib_ms = []
        for _ in range(max(1, min(args.steps, 3))):
            with torch.cuda.stream(stream):
                flush.add_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pib.search()
            e1.record(stream)
            e1.synchronize()
            ib_ms.append(e0.elapsed_time(e1))
        pib.close()
        interbin = {"value": nb_total / (statistics.mean(ib_ms) / 1e3), "unit": UNIT,
                    "ms_per_step": statistics.mean(ib_ms),
                    "form": "interbinning: transforms of n_fft/2, odd bins (pi/4)(X_k - X_k+1) "
                            "(the paper's Fourier-transform interpolation; approximate odd bins)"}

    # ---------------------------------------------------------------- end to end through the C ABI
    e2e = None
    if not args.skip_e2e:
        def pinned(a):
            t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
            t.numpy()[...] = a
            return t.numpy()

        class HB:
            pass
        hbs = []
        h2d = 0
        for b in w.bands:
            hb = HB()
            hb.n, hb.dt, hb.f_off, hb.phi0, hb.eps, hb.n_fft = b.n, b.dt, b.f_off, b.phi0, b.eps, b.n_fft
            hb.x = pinned(np.ascontiguousarray(b.x))
            hb.r = pinned(np.ascontiguousarray(b.r))
            h2d += hb.x.nbytes + hb.r.nbytes
            hbs.append(hb)
        al, de, fd = pinned(w.alpha), pinned(w.delta), pinned(w.fdot)
        n_e2e = max(3, min(args.steps, 5))
        w_e2e = 2     # per plan: the first search runs plainly, the second is captured as a CUDA graph
        streams = [stream, torch.cuda.Stream()]

        def make_plan(st=None):
            return fstat.Plan(hbs, al, de, fd, w.thr_2F, lat=w.lat, gamma=w.gamma,
                              upsample=w.upsample, form=fstat.FP32_BATCHED,
                              cand_capacity=args.cand_capacity,
                              stream=(st or stream).cuda_stream)
        # a stream of segments through two plans that take the segments in turn: per
        # step the segment's series and ephemeris go host -> device and the search
        # runs (a host thread) while the previous segment's candidates come back
        # (sort, device -> host copy, expansion into the caller's array)
        plans = [make_plan(st) for st in streams]
        outs = [None, None]   # the caller's candidate arrays, reused across segments
        d2h = 0
        device = torch.cuda.current_device()

        def upload_and_search(pl):
            torch.cuda.set_device(device)
            for bi, hb in enumerate(hbs):
                pl.set_band(bi, hb)
            pl.search()

        def drain(i):
            nonlocal d2h
            if outs[i] is not None:
                c, nt = plans[i].candidates(out=outs[i])
            else:
                c, nt = plans[i].candidates()
                outs[i] = np.empty(c.size + c.size // 4 + 1024, fstat.CAND_DTYPE)
                outs[i].view(np.uint8)[:] = 0     # resident before the timed steps
            d2h = int(c.size) * 16 + 8
        for it in range(w_e2e):               # untimed: both plans, plain then captured
            for i in range(2):
                upload_and_search(plans[i])
                drain(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(n_e2e):
            th = threading.Thread(target=upload_and_search, args=(plans[k % 2],))
            th.start()
            if k > 0:
                drain((k - 1) % 2)
            th.join()
        drain((n_e2e - 1) % 2)
        torch.cuda.synchronize()
        times = [(time.perf_counter() - t0) / n_e2e]
        for pl in plans:
            pl.close()
        # the same with a plan created (allocations, tables, grid upload) and destroyed per step
        h2d_grid = al.nbytes + de.nbytes + fd.nbytes
        times_pc = []
        for it in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p = make_plan()
            p.search()
            c, nt = p.candidates()
            p.close()
            torch.cuda.synchronize()
            if it > 0:
                times_pc.append(time.perf_counter() - t0)
        e2e = {"value": nb_total * world / statistics.mean(times), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "steps": n_e2e, "warmup": w_e2e,
               "with_plan_create": {"value": nb_total * world / statistics.mean(times_pc),
                                    "ms_per_step": 1e3 * statistics.mean(times_pc),
                                    "h2d_bytes_per_step": int(h2d + h2d_grid)},
               "includes": "fstat_plan_set_band per band (host->device copy of the segment's series "
                           "and ephemeris from pinned memory; sigma^2 and the upsample are redone by "
                           "the search) + fstat_search + fstat_candidates_get (device->host + sort) "
                           "for every step; two plans created before the timed steps take the "
                           "segments in turn, a segment's candidates drained while the next is "
                           "searched"}

    banded = large = None
    if rank == 0 and world == 1 and not args.skip_banded:
        banded = run_banded(args, stream, flush, peak)
    if rank == 0 and world == 1 and not args.skip_large:
        large = run_large(args, stream, flush, peak)

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        cpu = oracle_rate(w)

    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "precision: N=86164 float64 samples (2 sidereal days at 2 s), "
                                   "N_fft=2^18, 4096 sky x 64 spindown, 16 injections, 2F>30",
                       "form": "fp32_batched", "n_cells": int(w.n_sky * w.n_spin),
                       "bins_per_cell": int(w.bands[0].n_fft // 2 - 1),
                       "l2": "a 258 MB buffer is rewritten between timed steps (L2 flushed)",
                       "tuning": tuning,
                       "wall_s": round(t_wall, 3)},
            "candidates": int(n_total), "gpu_launches": int(launches),
            "roofline": roofline, "fp64_plain": fp64, "interbin": interbin,
            "speedup_vs_fp64_plain": (value / world / fp64["value"]) if fp64 else None,
            "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
            "banded_16_bands": banded, "large_65536x256": large}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sample-every", type=int, default=16)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-interbin", action="store_true")
    ap.add_argument("--skip-banded", action="store_true", help="no 16-band batching workload leg")
    ap.add_argument("--skip-large", action="store_true", help="no 65536 x 256 large-grid leg")
    ap.add_argument("--n-sky", type=int, default=0, help="first n sky positions only (profiling)")
    ap.add_argument("--cand-capacity", type=int, default=1 << 27)
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        td.init_process_group(backend)
        dist = td
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        return run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
