"""Autotuner for the batched form's kernel shape.

Times every supported (threads per block, entries per thread) shape on a
copy of the batch's own elevations for a few steps, keeps the fastest, and
caches the choice in a JSON file keyed by GPU name and the batch's size
profile (number of realizations and a log2 histogram of their cell counts),
so later batches of the same profile skip the timing.  All shapes compute
identical results; only speed differs.
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
