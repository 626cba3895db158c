"""Sharding of independent realizations across ranks (one process per GPU).

Realizations never exchange data, so a batch shards with no collective on
the data path: rank r advances its own subset and the host gathers results.
Subsets are balanced by cell count with the longest-processing-time rule
(largest realization first, each to the currently lightest rank), which is
within 4/3 of the optimal makespan (Graham, 1969).

run_shard advances one rank's subset in one batched launch (lem.Batch, shape
picked by the autotuner); gather_surfaces brings every rank's final surfaces
to rank 0 over the host-side process group (gloo or NCCL's object gather),
indexed by realization.
"""
from __future__ import annotations

import heapq


def lpt_partition(sizes, nranks):
    """Indices of `sizes` per rank; deterministic (ties by index, then rank)."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    heap = [(0, r) for r in range(nranks)]
    parts = [[] for _ in range(nranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + sizes[i], r))
    return [sorted(p) for p in parts]


def shard_loads(sizes, parts):
    return [sum(sizes[i] for i in p) for p in parts]


def run_shard(lem, bw, mine, steps, tune=True, advance=None):
    """Advance realizations `mine` of the batch workload `bw` by `steps` time
    steps; returns {"surfaces": {r: (ny, nx) float32 array}, "ms": device time
    of the batched launch, "shape": kernel shape, "tune_ms": autotuner table}.

    The batch is one lem.Batch of the shard's grids (FP32), its kernel shape
    picked by the autotuner on a copy of the initial state; one untimed
    warm-up launch runs on that copy too, so the returned surfaces are those
    after exactly `steps` steps.  `advance`, if given, replaces the GPU: it is
    called as advance(list of float32 surfaces, list of parameter dicts,
    steps) and returns the advanced surfaces (a host-side stand-in for runs
    without a GPU)."""
    import numpy as np
    init = [bw.initial(r).astype(np.float32) for r in mine]
    pars = [dict(dx=bw.dx, K=bw.K[r], m=bw.m[r], U=bw.U, dt=bw.dt) for r in mine]
    if advance is not None:
        out = advance(init, pars, steps)
        return {"surfaces": dict(zip(mine, out)), "ms": None, "shape": None, "tune_ms": {}}
    import torch
    from . import autotune
    B = lem.Batch(init, dx=bw.dx, K=[p["K"] for p in pars], m=[p["m"] for p in pars],
                  U=bw.U, dt=bw.dt)
    try:
        shape, tune_ms = autotune.tune_batch(B, steps=1) if tune else ((1024, 4), {})
        h0 = B.h.clone()
        B.step(1)  # warm-up launch, then back to the initial state
        B.h.copy_(h0)
        del h0
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        B.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        B.sync()
        ms = e0.elapsed_time(e1)
        surf = {r: B.surface(i).cpu().numpy() for i, r in enumerate(mine)}
    finally:
        B.close()
    return {"surfaces": surf, "ms": ms, "shape": shape, "tune_ms": tune_ms}


def gather_surfaces(local, count, rank, world):
    """Every rank's {realization: surface} to rank 0 as a list indexed by
    realization (None on other ranks).  world == 1 needs no process group."""
    if world == 1:
        return [local[r] for r in range(count)]
    import torch.distributed as dist
    got = [None] * world if rank == 0 else None
    dist.gather_object(local, got, dst=0)
    if rank != 0:
        return None
    merged = {}
    for part in got:
        for r, s in part.items():
            if r in merged:
                raise ValueError(f"realization {r} advanced by two ranks")
            merged[r] = s
    missing = [r for r in range(count) if r not in merged]
    if missing:
        raise ValueError(f"realizations {missing[:8]} advanced by no rank")
    return [merged[r] for r in range(count)]
