"""Pins Alg 1 of the oracle (receivers) and Algs 2-4 on real grids, by brute
force from the definitions (tests/brute.py), not by retyping the oracle."""
import numpy as np
import pytest

import oracle
from brute import exact_receivers, exact_slope, path_counts, walk_to_sink, NBR
from paper_1803_02977_gb300 import synth


def _int_grid(nx, ny, seed, levels=6):
    u = synth.uniform01(seed, nx * ny).reshape(ny, nx)
    return np.floor(u * levels).astype(np.float64)


@pytest.mark.parametrize("nx,ny,seed", [(3, 3, 1), (5, 4, 2), (8, 8, 3), (7, 9, 4),
                                        (8, 8, 5), (6, 6, 6), (9, 5, 7)])
def test_receivers_exact_on_integer_grids(nx, ny, seed):
    # integer heights: many exact ties and flats; exact rational argmax with
    # lowest-k tie-break must equal the oracle bit for bit
    h = _int_grid(nx, ny, seed)
    assert np.array_equal(oracle.receivers(h), exact_receivers(h))


def test_receivers_plateau_and_pit():
    h = np.full((6, 6), 5.0)
    h[2, 3] = 1.0  # an interior pit inside a plateau
    rec = oracle.receivers(h)
    nx = 6
    # plateau cells adjacent to the pit drain into it; other plateau cells
    # have no strictly lower neighbour and are sinks (self)
    pit = 2 * nx + 3
    assert rec[pit] == pit
    for y in range(1, 5):
        for x in range(1, 5):
            c = y * nx + x
            if c == pit:
                continue
            if abs(x - 3) <= 1 and abs(y - 2) <= 1:
                assert rec[c] == pit
            else:
                assert rec[c] == c


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_receivers_near_argmax_on_real_grids(seed):
    h = synth.noise_surface(12, 10, seed)
    h[1:-1, 1:-1] += 0.5  # make the perimeter a drain for most cells
    rec = oracle.receivers(h)
    exact = exact_receivers(h)
    ny, nx = h.shape
    for c in range(nx * ny):
        if exact[c] == c:
            assert rec[c] == c
            continue
        assert rec[c] != c
        s_best = exact_slope(h, c, exact[c])
        s_got = exact_slope(h, c, rec[c])
        assert s_got > 0
        assert s_got >= s_best * (1 - 1e-12)


def test_perimeter_is_noflow():
    h = synth.noise_surface(9, 7, 3) + 1.0
    rec = oracle.receivers(h)
    ny, nx = h.shape
    for c in range(nx * ny):
        x, y = c % nx, c // nx
        if x in (0, nx - 1) or y in (0, ny - 1):
            assert rec[c] == c


def test_receivers_f32_promotes():
    h32 = synth.noise_surface(16, 16, 9).astype(np.float32)
    assert np.array_equal(oracle.receivers(h32), oracle.receivers(h32.astype(np.float64)))


@pytest.mark.parametrize("nx,ny,seed,ints", [(8, 8, 21, False), (10, 7, 22, True),
                                             (16, 16, 23, False), (12, 12, 24, True)])
def test_graph_invariants(nx, ny, seed, ints):
    h = _int_grid(nx, ny, seed) if ints else synth.noise_surface(nx, ny, seed)
    rec = oracle.receivers(h)
    n = nx * ny
    # every receiver is a neighbour (or self) and strictly lower
    for c in range(n):
        r = rec[c]
        if r != c:
            assert abs(r % nx - c % nx) <= 1 and abs(r // nx - c // nx) <= 1
            assert h.flat[r] < h.flat[c]
    # donors: exact inverse of rec, in ascending address order
    dnum, donor = oracle.donors_grid(nx, ny, rec)
    for c in range(n):
        want = sorted(v for v in range(n) if v != c and rec[v] == c)
        assert donor[c, :dnum[c]].tolist() == want
    # acyclic: every path reaches a sink within n hops
    for c in range(n):
        walk_to_sink(rec, c, n + 1)
    q, lev, depth = oracle.queue(rec, dnum, donor)
    assert lev[0] == 0 and lev[-1] == n
    assert np.array_equal(np.sort(q), np.arange(n))
    sinks = [c for c in range(n) if rec[c] == c]
    assert q[:lev[1]].tolist() == sinks  # level 0: sinks, ascending
    for c in range(n):
        assert depth[c] == len(walk_to_sink(rec, c, n + 1)) - 1
    for l in range(lev.size - 1):
        assert set(depth[q[lev[l]:lev[l + 1]]].tolist()) == {l}
    # accumulation = brute-force path counting; totals equal the cell count
    cnt = oracle.accumulate(q, lev, dnum, donor)
    assert np.array_equal(cnt, path_counts(rec))
    assert cnt[sinks].sum() == n


def test_donor_order_follows_neighbour_code():
    # a cell with donors on all 8 sides: donors listed NW, N, NE, W, E, SW, S, SE
    h = np.full((5, 5), 10.0)
    h[2, 2] = 0.0
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 20.0
    rec = oracle.receivers(h)
    dnum, donor = oracle.donors_grid(5, 5, rec)
    c = 12
    assert dnum[c] == 8
    assert donor[c].tolist() == [(2 + oy) * 5 + (2 + ox) for ox, oy in NBR]
