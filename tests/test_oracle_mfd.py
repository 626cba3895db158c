"""Pins the oracle's multiple-flow-direction accumulation (Eq. 2 with a
slope-weighted split): a dense linear solve of A = w + M^T A on tiny grids, a
hand-computed 3x3 cone, a channel where every cell has one receiver (D8
counts), mass balance, linearity in w, and the level order."""
import math

import numpy as np
import pytest

import oracle
from brute import NBR
from paper_1803_02977_gb300 import synth


def _perim(nx, ny, x, y):
    return x == 0 or y == 0 or x == nx - 1 or y == ny - 1


def _split(h, p):
    """M[d, c] = share of d's flow sent to c, from the definition: every
    strictly lower neighbour of an interior cell, weights slope^p."""
    ny, nx = h.shape
    N = nx * ny
    M = np.zeros((N, N))
    for y in range(ny):
        for x in range(nx):
            if _perim(nx, ny, x, y):
                continue
            d = y * nx + x
            ws = {}
            for ox, oy in NBR:
                xn, yn = x + ox, y + oy
                if h[yn, xn] < h[y, x]:
                    dist = math.sqrt(2.0) if ox and oy else 1.0
                    ws[yn * nx + xn] = ((h[y, x] - h[yn, xn]) / dist) ** p
            tot = sum(ws.values())
            for c, v in ws.items():
                M[d, c] = v / tot
    return M


@pytest.mark.parametrize("seed,p", [(1, 1.0), (2, 1.0), (3, 1.1), (4, 2.0)])
def test_equals_dense_linear_solve(seed, p):
    nx, ny = 7, 6
    h = synth.noise_surface(nx, ny, seed)
    w = 0.5 + synth.uniform01(seed + 10, nx * ny)
    A, _, _ = oracle.accumulate_mfd(h, p, w.reshape(ny, nx))
    M = _split(h, p)
    want = np.linalg.solve(np.eye(nx * ny) - M.T, w)
    assert np.abs(A.ravel() - want).max() <= 1e-12 * np.abs(want).max()


def test_cone_by_hand():
    # the centre of a 3x3 grid sends its unit of flow to its eight lower
    # neighbours in proportion to slope: 1 for the cardinal, 1/sqrt2 diagonal
    h = np.zeros((3, 3))
    h[1, 1] = 1.0
    A, lev, L = oracle.accumulate_mfd(h, 1.0)
    D = 4.0 + 4.0 / math.sqrt(2.0)
    assert A[1, 1] == 1.0
    for (y, x) in [(0, 1), (1, 0), (1, 2), (2, 1)]:
        assert abs(A[y, x] - (1.0 + 1.0 / D)) <= 1e-15
    for (y, x) in [(0, 0), (0, 2), (2, 0), (2, 2)]:
        assert abs(A[y, x] - (1.0 + (1.0 / math.sqrt(2.0)) / D)) <= 1e-15
    assert L == 2 and lev[1, 1] == 0 and lev[0, 0] == 1


def test_single_receivers_give_d8_counts():
    # a channel along row 1 rising eastward between walls of 1000: each cell
    # has exactly one lower neighbour, its west one
    nx = 20
    h = np.full((3, nx), 1000.0)
    h[1, :] = np.arange(nx, dtype=np.float64)
    h[1, 0] = 0.0
    h[1, -1] = 1000.0
    A, _, _ = oracle.accumulate_mfd(h, 1.3)
    for x in range(1, nx - 1):
        assert A[1, x] == float(nx - 1 - x)
    assert A[1, 0] == float(nx - 1)  # the outlet gathers the whole channel


@pytest.mark.parametrize("p", [1.0, 1.1])
def test_mass_balance_and_linearity(p):
    nx, ny = 40, 33
    h = synth.noise_surface(nx, ny, 5)
    w1 = synth.uniform01(6, nx * ny).reshape(ny, nx)
    w2 = synth.uniform01(7, nx * ny).reshape(ny, nx)
    A1, _, _ = oracle.accumulate_mfd(h, p, w1)
    A2, _, _ = oracle.accumulate_mfd(h, p, w2)
    A12, _, _ = oracle.accumulate_mfd(h, p, w1 + w2)
    assert np.abs(A12 - (A1 + A2)).max() <= 1e-12 * np.abs(A12).max()
    # every unit of flow ends in a cell without receivers
    rec = np.zeros((ny, nx), bool)
    for y in range(1, ny - 1):
        for x in range(1, nx - 1):
            rec[y, x] = any(h[y + oy, x + ox] < h[y, x] for ox, oy in NBR)
    assert abs(A1[~rec].sum() - w1.sum()) <= 1e-11 * w1.sum()
    assert np.all(A1 >= w1)


def test_levels_follow_the_deepest_donor():
    nx, ny = 30, 25
    h = synth.noise_surface(nx, ny, 8)
    _, lev, L = oracle.accumulate_mfd(h, 1.0)
    for y in range(ny):
        for x in range(nx):
            donors = [lev[y + oy, x + ox] for ox, oy in NBR
                      if 0 <= x + ox < nx and 0 <= y + oy < ny
                      and not _perim(nx, ny, x + ox, y + oy) and h[y + oy, x + ox] > h[y, x]]
            assert lev[y, x] == (1 + max(donors) if donors else 0)
    assert L == lev.max() + 1
