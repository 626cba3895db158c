"""Autotuner for the kernels' work decomposition.

tune_batch times every supported (threads per block, entries per thread)
shape of the batched form on a copy of the batch's own elevations; tune_step
times the single-grid step's tilings (lem_set_tiling: rows per strip of the
codes pass, whole or half-height warp tiles).  Each keeps the
fastest and caches the choice in a JSON file keyed by GPU name and the
problem (the batch's size profile -- number of realizations and a log2
histogram of their cell counts -- or the grid's size and types), so later
runs of the same problem skip the timing.  All choices compute identical
results; only speed differs.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import lem


def cache_path() -> str:
    p = os.environ.get("LEM_AUTOTUNE_CACHE")
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "lem_autotune.json")


def profile_key(batch: "lem.Batch") -> str:
    hist = {}
    for ny, nx in batch.shapes:
        b = int(math.log2(max(nx * ny, 1)))
        hist[b] = hist.get(b, 0) + 1
    name = torch.cuda.get_device_name(batch.h.device)
    return f"{name}|f32|R={batch.R}|" + ",".join(f"{k}:{hist[k]}" for k in sorted(hist))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict) -> None:
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def tune_batch(batch: "lem.Batch", steps: int = 2, use_cache: bool = True):
    """Pick and set the fastest kernel shape; returns (shape, {shape: ms})."""
    key = profile_key(batch)
    cache = _load() if use_cache else {}
    if key in cache:
        bd, pi = cache[key]["shape"]
        batch.set_config(bd, pi)
        return (bd, pi), cache[key].get("ms", {})
    saved = batch.h.clone()
    stream = torch.cuda.current_stream()
    timings = {}
    for bd, pi in lem.BATCH_CONFIGS:
        batch.h.copy_(saved)
        batch.set_config(bd, pi)
        batch.step(1)  # warm-up
        batch.h.copy_(saved)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        timings[f"{bd}x{pi}"] = e0.elapsed_time(e1) / steps
    best = min(timings, key=timings.get)
    bd, pi = (int(v) for v in best.split("x"))
    batch.h.copy_(saved)
    batch.set_config(bd, pi)
    torch.cuda.synchronize()
    if use_cache:
        cache[key] = {"shape": [bd, pi], "ms": timings}
        _store(cache)
    return (bd, pi), timings


# ---- the single-grid step (lem_set_tiling) ------------------------------------

def step_strip_rows(model: "lem.Model"):
    """Rows per strip of the codes pass that the step accepts for this grid."""
    return (8, 16, 32) if model.dtype == lem.LEM_F32 else (8, 16)


def step_key(model: "lem.Model") -> str:
    name = torch.cuda.get_device_name(model.h.device)
    dt = "f64" if model.dtype == lem.LEM_F64 else "f32"
    return f"{name}|step|{dt}|c{model.count_bits}|{model.nx}x{model.ny}"


def tune_step(model: "lem.Model", steps: int = 3, use_cache: bool = True):
    """Pick and set the fastest work decomposition of lem_step for this grid
    (lem_set_tiling: rows per strip of the codes pass, whole or half-height
    warp tiles), timed on copies of the model's own elevations; returns
    ((strip_rows, half_tiles), {"<rows>x<half>": ms per step}).  Every choice
    computes the same receivers, masks and (while no tree needs the
    pointer-jumping device tier) the same elevations."""
    key = step_key(model)
    cache = _load() if use_cache else {}
    if key in cache:
        k, hf = cache[key]["shape"]
        lem.lem_set_tiling(model.ctx, k, hf)
        return (k, hf), cache[key].get("ms", {})
    saved = model.h.clone()
    stream = torch.cuda.current_stream()
    timings = {}
    for k in step_strip_rows(model):
        for hf in (0, 1):
            model.h.copy_(saved)
            lem.lem_set_tiling(model.ctx, k, hf)
            model.step(1)  # warm-up
            model.h.copy_(saved)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                model.step(1)
            e1.record(stream)
            torch.cuda.synchronize()
            timings[f"{k}x{hf}"] = e0.elapsed_time(e1) / steps
    best = min(timings, key=timings.get)
    k, hf = (int(v) for v in best.split("x"))
    model.h.copy_(saved)
    lem.lem_set_tiling(model.ctx, k, hf)
    model.sync()
    if use_cache:
        cache[key] = {"shape": [k, hf], "ms": timings}
        _store(cache)
    return (k, hf), timings
