"""Pins Alg 6 of the oracle for a general slope exponent n-hat (the
Newton-Raphson iteration): the root of the quadratic for n-hat = 2 at every
cell, one Newton update written out, the 1-D channel steady state, and the
reading for cells without a downhill slope.  Each check recomputes the
receivers' new elevations by recursion over the receiver graph, independent of
the oracle's level order."""
import math

import numpy as np
import pytest

import oracle
from brute import is_perimeter
from paper_1803_02977_gb300 import synth


def _dist(nx, c, r, dx):
    diag = (c % nx != r % nx) and (c // nx != r // nx)
    return dx * math.sqrt(2.0) if diag else dx


def _sweep(h, rec, cnt, p, n_exp, update):
    """New elevations of one step with the per-cell solve `update(h0, hr, F)`,
    each receiver's value computed first (recursion on rec, not the queue)."""
    ny, nx = h.shape
    Uf = getattr(p, "_keep", None)
    new = {}

    def value(c):
        if c in new:
            return new[c]
        if is_perimeter(nx, ny, c):
            v = float(h.flat[c])
        else:
            u = p.U if Uf is None else float(Uf[c])
            h0 = float(h.flat[c]) + u * p.dt
            r = int(rec[c])
            if r == c:
                v = h0
            else:
                hr = value(r)
                F = p.K * p.dt * (float(cnt[c]) * p.area_scale) ** p.m / _dist(nx, c, r, p.dx) ** n_exp
                v = update(h0, hr, F)
        new[c] = v
        return v

    out = np.empty(nx * ny)
    for c in range(nx * ny):
        out[c] = value(c)
    return out.reshape(ny, nx)


@pytest.mark.parametrize("nx,ny,seed,K", [(12, 10, 21, 0.1), (9, 14, 22, 1e-3), (16, 16, 23, 1.0)])
def test_n2_equals_quadratic_root(nx, ny, seed, K):
    # n-hat = 2: F x^2 + x - b = 0 with x = h - h_r, b = h0 - h_r; the positive
    # root in the cancellation-free form x = 2b / (1 + sqrt(1 + 4 F b))
    h = synth.noise_surface(nx, ny, seed)
    p = oracle.params(K=K)
    got, g = oracle.step_newton(h, p, 2.0, 1e-14, 100)

    def root(h0, hr, F):
        b = h0 - hr
        if not b > 0:
            return h0
        return hr + 2.0 * b / (1.0 + math.sqrt(1.0 + 4.0 * F * b))

    want = _sweep(h, g.rec, g.cnt, p, 2.0, root)
    assert np.abs(got - want).max() <= 1e-12 * max(np.abs(want).max(), 1.0)
    # the erosion is not negligible at these parameters
    a = h.copy()
    oracle.uplift(a, p)
    assert np.abs(got - a).max() > 1e-3


@pytest.mark.parametrize("n_exp", [1.5, 2.0, 3.0])
def test_one_iteration_is_one_newton_update(n_exp):
    nx, ny = 11, 9
    h = synth.noise_surface(nx, ny, 24)
    p = oracle.params(K=0.05)
    got, g = oracle.step_newton(h, p, n_exp, 1e-14, 1)

    def one_update(h0, hr, F):
        b = h0 - hr
        if not b > 0:
            return h0
        return h0 - (F * b ** n_exp) / (1.0 + F * n_exp * b ** (n_exp - 1.0))

    want = _sweep(h, g.rec, g.cnt, p, n_exp, one_update)
    assert np.abs(got - want).max() <= 1e-12 * max(np.abs(want).max(), 1.0)


def _channel(nx):
    rec = np.arange(3 * nx, dtype=np.int32)
    for x in range(1, nx - 1):
        rec[nx + x] = nx + x - 1
    return rec


@pytest.mark.parametrize("n_exp", [1.5, 3.0])
def test_channel_steady_state_general_n(n_exp):
    # fixed point of h' (1 + ...) : F (h - h_r)^n = dt U  <=>  (slope)^n = U / (K A^m)
    nx, dx, K, m, U, dt = 30, 100.0, 1e-5, 0.5, 1e-3, 1000.0
    p = oracle.params(dx=dx, K=K, m=m, U=U, dt=dt)
    h = np.zeros((3, nx))
    for x in range(1, nx - 1):
        A = (nx - 1 - x) * p.area_scale
        h[1, x] = h[1, x - 1] + dx * (U / (K * A ** m)) ** (1.0 / n_exp)
    hn, g = oracle.step_newton(h, p, n_exp, 1e-14, 100, frozen_rec=_channel(nx))
    assert np.array_equal(g.cnt[nx + 1:2 * nx - 1], np.arange(nx - 2, 0, -1))
    assert np.abs(hn - h).max() <= 1e-11 * np.abs(h).max()


def test_residual_of_implicit_equation_n15():
    nx, ny = 14, 12
    h = synth.noise_surface(nx, ny, 25)
    p = oracle.params(K=0.02)
    hn, g = oracle.step_newton(h, p, 1.5, 1e-14, 100)
    a = h.copy()
    oracle.uplift(a, p)
    n_checked = 0
    for l in range(1, g.nlevels):
        for c in g.queue[g.levels[l]:g.levels[l + 1]]:
            r = g.rec[c]
            F = p.K * p.dt * (g.cnt[c] * p.area_scale) ** p.m / _dist(nx, c, r, p.dx) ** 1.5
            res = hn.flat[c] - a.flat[c] + F * (hn.flat[c] - hn.flat[r]) ** 1.5
            assert abs(res) <= 1e-11 * max(1.0, abs(a.flat[c]))
            assert hn.flat[c] > hn.flat[r]
            n_checked += 1
    assert n_checked > 50


def test_no_downhill_slope_keeps_uplifted_elevation():
    # a per-cell uplift that lifts the receiver above the cell's own uplifted
    # elevation: that cell keeps h0 for n-hat != 1
    nx = 8
    rec = _channel(nx)
    h = np.zeros((3, nx))
    for x in range(1, nx - 1):
        h[1, x] = 0.01 * x
    Uf = np.full(3 * nx, 1e-3)
    Uf[nx + 3] = 1.0     # the receiver of cell (4, 1) rises by 1000 m
    p = oracle.params(K=1e-4, Ufield=Uf)
    hn, g = oracle.step_newton(h, p, 2.0, 1e-14, 100, frozen_rec=rec)
    c = nx + 4
    assert hn.flat[c] == h.flat[c] + 1e-3 * p.dt
    assert hn.flat[nx + 3] < h.flat[nx + 3] + 1.0 * p.dt  # the receiver itself erodes
