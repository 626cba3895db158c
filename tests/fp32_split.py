"""Separating the two error sources of an FP32 trajectory against the FP64
oracle (test helper; no method arithmetic beyond reading the oracle's graphs).

A cell's new elevation depends on its own elevation, its receiver's new
elevation, its receiver direction and its count (Alg 6).  So if, over a whole
run, a cell's receiver and count were the same in both runs at every step and
its receiver was itself such a cell at every step, its error is rounding of
the FP32 arithmetic alone.  Every other cell is downstream of, or drains
through, a receiver decision that went the other way in the FP32 state (a
near tie), and its difference is a different flow path, not arithmetic.
"""
from __future__ import annotations

import numpy as np


def clean_update(clean, rec64, cnt64, rec32, cnt32, queue, levels):
    """One step of the clean set.

    clean       bool[N], cells clean before this step (updated copy returned)
    rec64/cnt64 the FP64 run's receivers (self = none) and counts this step
    rec32/cnt32 the FP32 run's, computed from its own state
    queue/levels the FP64 run's breadth-first levels (receivers first)
    A cell stays clean if it was clean, its receiver and count agree, and its
    receiver (already visited, one level lower) is clean after this step."""
    out = clean & (rec64 == rec32) & (cnt64 == cnt32)
    for lv in range(1, levels.size - 1):
        cs = queue[levels[lv]:levels[lv + 1]]
        out[cs] &= out[rec64[cs]]
    return out
