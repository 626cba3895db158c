"""Pins the oracle's depression filling (Section "Local Minima": depressions
filled to their outlets by Priority-Flood, the flats resolved with epsilon
increments): the fixed-point equation that defines the least such surface,
Bellman-Ford relaxation on tiny grids, hand-computed nested basins, no interior
sink left for Alg 1, and no change to a surface that already drains."""
import numpy as np
import pytest

import oracle
from brute import NBR
from paper_1803_02977_gb300 import synth


def _int_grid(nx, ny, seed, levels=4):
    u = synth.uniform01(seed, nx * ny).reshape(ny, nx)
    h = np.floor(u * levels)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


def _succ(v, dtype):
    return dtype(np.nextafter(dtype(v), dtype(np.inf)))


def _fixed_point_violations(h, w):
    """Cells where w differs from max(h, next value above the lowest
    neighbouring w) (interior) or from h (perimeter)."""
    ny, nx = h.shape
    dt = h.dtype.type
    bad = []
    for y in range(ny):
        for x in range(nx):
            if x in (0, nx - 1) or y in (0, ny - 1):
                if w[y, x] != h[y, x]:
                    bad.append((x, y))
                continue
            lo = min(w[y + oy, x + ox] for ox, oy in NBR)
            want = max(h[y, x], _succ(lo, dt))
            if w[y, x] != want:
                bad.append((x, y))
    return bad


CASES = [
    ("noise_9x7", lambda: synth.noise_surface(9, 7, 1)),
    ("noise_40x33", lambda: synth.noise_surface(40, 33, 2)),
    ("int_flats_30x30", lambda: _int_grid(30, 30, 3)),
    ("plateau_20x20", lambda: np.pad(np.full((18, 18), 7.0), 1)),
    ("all_flat_12x9", lambda: np.zeros((9, 12))),
    ("tilt_25x20", lambda: synth.noise_surface(25, 20, 4, south_tilt=1e-1)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_fixed_point_equation_every_cell(name, make, dtype):
    h = make().astype(dtype)
    w = oracle.fill(h)
    assert w.dtype == h.dtype
    assert _fixed_point_violations(h, w) == []
    assert np.all(w >= h)


def _bellman_ford(h):
    """Relaxation from +inf in the interior until nothing changes: the least
    fixed point, reached by a different route than the priority queue."""
    ny, nx = h.shape
    dt = h.dtype.type
    w = np.full_like(h, np.inf)
    w[0, :], w[-1, :], w[:, 0], w[:, -1] = h[0, :], h[-1, :], h[:, 0], h[:, -1]
    changed = True
    while changed:
        changed = False
        for y in range(1, ny - 1):
            for x in range(1, nx - 1):
                lo = min(w[y + oy, x + ox] for ox, oy in NBR)
                v = max(h[y, x], _succ(lo, dt))
                if v < w[y, x]:
                    w[y, x] = v
                    changed = True
    return w


@pytest.mark.parametrize("seed", [5, 6, 7])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_equals_bellman_ford_on_tiny_grids(seed, dtype):
    for h in (synth.noise_surface(8, 7, seed).astype(dtype), _int_grid(9, 8, seed).astype(dtype)):
        assert np.array_equal(oracle.fill(h), _bellman_ford(h))


def test_nested_basins_by_hand():
    # perimeter at 2; a ring of 5s encloses an inner ring of 1s around a pit
    # of 0 at the centre, with one gap in the outer ring at height 3
    h = np.full((7, 7), 5.0)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 2.0
    h[2:5, 2:5] = 1.0
    h[3, 3] = 0.0
    h[1, 3] = 3.0  # the outlet of the basin, next to the perimeter
    w = oracle.fill(h)
    s = lambda v, k=1: v if k == 0 else s(np.nextafter(v, np.inf), k - 1)  # noqa: E731
    assert w[1, 3] == 3.0                 # outlet: above its perimeter neighbour
    # the row just inside touches the outlet (diagonally at its ends)
    assert w[2, 2] == w[2, 3] == w[2, 4] == s(3.0)
    assert w[3, 2] == w[3, 3] == w[3, 4] == s(3.0, 2)  # the pit row, two steps in
    assert w[4, 2] == w[4, 3] == w[4, 4] == s(3.0, 3)
    assert w[1, 1] == 5.0                 # the outer ring keeps its height
    assert w[5, 3] == 5.0


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_no_interior_sink_after_filling(dtype):
    h = synth.noise_surface(60, 45, 8).astype(dtype)
    w = oracle.fill(h)
    rec = oracle.receivers(w)
    ny, nx = h.shape
    for c in range(nx * ny):
        x, y = c % nx, c // nx
        interior = 0 < x < nx - 1 and 0 < y < ny - 1
        assert (rec[c] != c) == interior
    # and every path of receivers ends on the perimeter
    for c in range(nx * ny):
        s, hops = c, 0
        while rec[s] != s:
            s = rec[s]
            hops += 1
            assert hops <= nx * ny
        assert s % nx in (0, nx - 1) or s // nx in (0, ny - 1)


def test_draining_surface_unchanged_and_small_grids():
    # a plane falling toward the west edge: every cell already drains
    ny, nx = 20, 30
    h = np.tile(np.arange(nx, dtype=np.float64) * 0.5 + 1.0, (ny, 1))
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    assert np.array_equal(oracle.fill(h), h)
    # grids with no interior cell are their own fill
    for shape in [(1, 1), (2, 5), (7, 2)]:
        g = synth.uniform01(9, shape[0] * shape[1]).reshape(shape)
        assert np.array_equal(oracle.fill(g), g)
