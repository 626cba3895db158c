"""Host logic of the scaling sweep (bench.py --sweep): the per-region fit of
the wall-time exponent x in O(N^x), against timings built with known
exponents (continuous across the region bounds, as measured curves are)."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _piecewise(edges, xs, bounds, t0=1.0):
    # t(N) continuous, slope xs[i] in log-log on region i
    out = []
    for e in edges:
        logt, lo = np.log(t0), 100.0
        for x, hi in zip(xs, bounds):
            a, b = np.log(lo * lo), np.log(min(e, hi) ** 2)
            if b > a:
                logt += x * (b - a)
            if e <= hi:
                break
            lo = hi
        out.append(np.exp(logt))
    return out


def test_fit_recovers_known_exponents():
    xs = [0.33, 0.16, 0.42, 0.92]
    bounds = [hi for _, hi, _ in bench.SWEEP_REGIONS]
    t = _piecewise(bench.SWEEP_EDGES, xs, bounds)
    fit = bench.fit_exponents(bench.SWEEP_EDGES, t)
    for (name, _, _), x in zip(bench.SWEEP_REGIONS, xs):
        assert fit[name] == pytest.approx(x, abs=1e-9)


def test_fit_constant_time_is_flat_and_linear_time_is_one():
    e = bench.SWEEP_EDGES
    assert all(abs(v) < 1e-12 for v in bench.fit_exponents(e, [3.0] * len(e)).values())
    lin = [1e-6 * x * x for x in e]
    assert all(v == pytest.approx(1.0) for v in bench.fit_exponents(e, lin).values())


def test_fit_reports_none_for_a_region_without_two_points():
    fit = bench.fit_exponents([100, 200], [1.0, 2.0])
    assert fit["A"] == pytest.approx(0.5)
    assert fit["B"] is None and fit["C"] is None and fit["D"] is None


def test_sweep_spans_the_papers_regions():
    edges = bench.SWEEP_EDGES
    assert edges[0] == 100 and edges[-1] == 16000
    for _, hi, _ in bench.SWEEP_REGIONS:
        assert hi in edges
