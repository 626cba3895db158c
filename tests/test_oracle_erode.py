"""Pins Algs 5-6 of the oracle (uplift + implicit n = 1 erosion): dense linear
solve, closed-form steady state, special cases and invariants."""
import numpy as np
import pytest

import oracle
from brute import implicit_solve, is_perimeter
from paper_1803_02977_gb300 import synth


@pytest.mark.parametrize("nx,ny,seed,area_scale", [(6, 6, 1, None), (8, 7, 2, None),
                                                   (10, 10, 3, 1.0), (12, 9, 4, None)])
def test_erode_equals_dense_implicit_solve(nx, ny, seed, area_scale):
    h = synth.noise_surface(nx, ny, seed)
    p = oracle.params(dx=100.0, K=1e-4, m=0.5, U=1e-3, dt=1000.0, area_scale=area_scale)
    hn, g = oracle.step(h, p)
    want = implicit_solve(h, g.rec, g.cnt, 100.0, 1e-4, 0.5, 1e-3, 1000.0, p.area_scale)
    scale = max(np.abs(want).max(), 1.0)
    assert np.abs(hn - want).max() <= 1e-12 * scale


def test_erode_equals_dense_solve_with_uplift_field():
    nx, ny = 9, 8
    h = synth.noise_surface(nx, ny, 7)
    Uf = 1e-3 * (1.0 + 0.5 * synth.signed_field(nx, ny, 8))
    p = oracle.params(K=3e-5, Ufield=Uf)
    hn, g = oracle.step(h, p)
    want = implicit_solve(h, g.rec, g.cnt, 100.0, 3e-5, 0.5, None, 1000.0, p.area_scale, Uf)
    assert np.abs(hn - want).max() <= 1e-12 * max(np.abs(want).max(), 1.0)


def _channel(nx):
    """A 1-D channel along row 1 of a 3-row grid: cell (x,1) drains west."""
    rec = np.arange(3 * nx, dtype=np.int32)
    for x in range(1, nx - 1):
        rec[nx + x] = nx + x - 1
    return rec


def _channel_profile(nx, dx, K, m, U, area_scale):
    # steady state: (h_x - h_{x-1}) / dx = U / (K A_x^m), A_x = (nx-1-x) cells
    h = np.zeros((3, nx))
    for x in range(1, nx - 1):
        A = (nx - 1 - x) * area_scale
        h[1, x] = h[1, x - 1] + dx * U / (K * A ** m)
    return h


def test_channel_steady_state_is_fixed_point():
    nx, dx, K, m, U, dt = 40, 100.0, 1e-5, 0.5, 1e-3, 1000.0
    p = oracle.params(dx=dx, K=K, m=m, U=U, dt=dt)
    h = _channel_profile(nx, dx, K, m, U, p.area_scale)
    hn, g = oracle.step(h, p, frozen_rec=_channel(nx))
    assert np.array_equal(g.cnt[nx + 1:2 * nx - 1], np.arange(nx - 2, 0, -1))
    assert np.abs(hn - h).max() <= 1e-12 * np.abs(h).max()


def test_channel_converges_to_closed_form():
    nx, dx, K, m, U, dt = 24, 100.0, 1e-3, 0.45, 2e-3, 5000.0
    p = oracle.params(dx=dx, K=K, m=m, U=U, dt=dt)
    want = _channel_profile(nx, dx, K, m, U, p.area_scale)
    h = np.zeros((3, nx))
    h = oracle.run(h, p, 400, frozen_rec=_channel(nx))
    assert np.abs(h - want).max() <= 1e-9 * np.abs(want).max()


def test_free_grid_steady_state_relation():
    # uniform uplift on a free grid, run to steady state: every eroding cell
    # satisfies (h_c - h_r)/d_c = U / (K A_c^m)
    nx = ny = 14
    dx, K, m, U, dt = 100.0, 2e-4, 0.5, 1e-3, 2000.0
    p = oracle.params(dx=dx, K=K, m=m, U=U, dt=dt)
    h = synth.noise_surface(nx, ny, 5)
    prev_rec = None
    for it in range(400):
        hn, g = oracle.step(h, p)
        done = prev_rec is not None and np.array_equal(g.rec, prev_rec) and \
            np.abs(hn - h).max() < 1e-10
        prev_rec = g.rec
        h = hn
        if done:
            break
    assert done, "did not reach steady state"
    g = oracle.StepGraph(h)
    assert np.array_equal(g.rec, prev_rec)
    n_checked = 0
    for c in range(nx * ny):
        r = g.rec[c]
        if r == c or is_perimeter(nx, ny, c):
            continue
        diag = (c % nx != r % nx) and (c // nx != r // nx)
        d = dx * (2 ** 0.5 if diag else 1.0)
        slope = (h.flat[c] - h.flat[r]) / d
        want = U / (K * (g.cnt[c] * p.area_scale) ** m)
        assert abs(slope - want) <= 1e-9 * want
        n_checked += 1
    assert n_checked > 100


def test_K_zero_is_pure_uplift():
    nx, ny, T = 10, 9, 7
    h0 = synth.noise_surface(nx, ny, 9)
    p = oracle.params(K=0.0, U=2e-3, dt=500.0)
    h = oracle.run(h0, p, T)
    inner = (slice(1, -1), slice(1, -1))
    assert np.allclose(h[inner], h0[inner] + T * 2e-3 * 500.0, rtol=0, atol=1e-12)
    assert np.all(h[0, :] == 0) and np.all(h[-1, :] == 0)


def test_no_uplift_large_erosion_flattens_to_base_level():
    nx, ny = 12, 12
    h0 = synth.noise_surface(nx, ny, 10) + 0.0
    p = oracle.params(K=1e6, U=0.0, dt=1e6)
    h1, g = oracle.step(h0, p)
    for c in range(nx * ny):
        s = c
        while g.rec[s] != s:
            s = g.rec[s]
        if is_perimeter(nx, ny, s):
            assert abs(h1.flat[c]) < 1e-9
        elif s == c:
            assert h1.flat[c] == h0.flat[c]  # pits keep their height (U = 0)


def test_uniform_uplift_keeps_strict_descent():
    nx = ny = 32
    h = synth.noise_surface(nx, ny, 12)
    p = oracle.params()
    for _ in range(20):
        hn, g = oracle.step(h, p)
        for l in range(1, g.nlevels):
            cs = g.queue[g.levels[l]:g.levels[l + 1]]
            assert np.all(hn.flat[cs] > hn.flat[g.rec[cs]])
        h = hn


def test_newton_n1_matches_closed_form_and_n2_residual():
    nx, ny = 16, 12
    h0 = synth.noise_surface(nx, ny, 13)
    p = oracle.params(K=2e-5)
    g = oracle.StepGraph(h0)
    a = h0.copy()
    oracle.uplift(a, p)
    h_cf = a.copy()
    oracle.erode(h_cf, g.rec, g.queue, g.levels, g.cnt, p)
    h_nr = a.copy()
    oracle.erode_newton(h_nr, g.rec, g.queue, g.levels, g.cnt, p, 1.0, 1e-14, 50)
    assert np.abs(h_nr - h_cf).max() <= 1e-12 * np.abs(h_cf).max()
    # n = 2: residual h - h0 + F (h - h_r)^2 = 0 at every eroding cell
    h2 = a.copy()
    oracle.erode_newton(h2, g.rec, g.queue, g.levels, g.cnt, p, 2.0, 1e-13, 100)
    for l in range(1, g.nlevels):
        for c in g.queue[g.levels[l]:g.levels[l + 1]]:
            r = g.rec[c]
            diag = (c % nx != r % nx) and (c // nx != r // nx)
            d = 100.0 * (2 ** 0.5 if diag else 1.0)
            F = p.K * p.dt * (g.cnt[c] * p.area_scale) ** p.m / d ** 2
            res = h2.flat[c] - a.flat[c] + F * (h2.flat[c] - h2.flat[r]) ** 2
            assert abs(res) <= 1e-10 * max(1.0, abs(a.flat[c]))
