"""Pins the oracle's tangent-linear and adjoint steps: central finite
differences of the forward oracle, and the dot-product identity."""
import numpy as np

import oracle
from paper_1803_02977_gb300 import synth


def _setup(nx=12, ny=10, seed=31):
    h0 = synth.noise_surface(nx, ny, seed)
    h0[1:-1, 1:-1] += 2.0
    Uf = 1e-3 * (1.0 + 0.3 * synth.signed_field(nx, ny, seed + 1))
    return h0, Uf


def test_tangent_matches_central_fd_of_frozen_step():
    nx, ny = 12, 10
    h0, Uf = _setup(nx, ny)
    K = 2e-5
    p = oracle.params(K=K, Ufield=Uf)
    h1, g = oracle.step(h0, p)
    rng = np.random.default_rng(0)
    dh = rng.standard_normal((ny, nx))
    dU = 1e-3 * rng.standard_normal((ny, nx))
    dK = 1e-5 * rng.standard_normal()
    eps = 1e-6
    hp, _ = oracle.step(h0 + eps * dh, oracle.params(K=K + eps * dK, Ufield=Uf + eps * dU),
                        frozen_rec=g.rec)
    hm, _ = oracle.step(h0 - eps * dh, oracle.params(K=K - eps * dK, Ufield=Uf - eps * dU),
                        frozen_rec=g.rec)
    fd = (hp - hm) / (2 * eps)
    tl = oracle.tangent_step(h1, g, p, dh, dU, dK)
    assert np.abs(tl - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


def test_adjoint_dot_product_identity():
    nx, ny = 14, 11
    h0, Uf = _setup(nx, ny, 41)
    p = oracle.params(K=3e-5, Ufield=Uf)
    h1, g = oracle.step(h0, p)
    rng = np.random.default_rng(1)
    dh = rng.standard_normal((ny, nx))
    dU = rng.standard_normal((ny, nx))
    dK = rng.standard_normal()
    w = rng.standard_normal((ny, nx))
    tl = oracle.tangent_step(h1, g, p, dh, dU, dK)
    lam_prev, gU, gK = oracle.adjoint_step(h1, g, p, w, np.zeros(nx * ny), 0.0)
    lhs = float(np.sum(tl * w))
    rhs = float(np.sum(dh * lam_prev) + np.sum(dU.ravel() * gU) + dK * gK)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_loss_gradient_matches_central_fd():
    nx, ny, T = 12, 12, 6
    h0, Uf = _setup(nx, ny, 51)
    K = 2e-5
    p = oracle.params(K=K, Ufield=Uf)
    h_obs = oracle.run(h0, oracle.params(K=1.2 * K, Ufield=Uf * 1.05), T)
    loss, gU, gK = oracle.loss_and_grad(h0, p, T, h_obs)
    eps = 1e-6

    def loss_at(Kv, Ufv):
        return float(np.sum((oracle.run(h0, oracle.params(K=Kv, Ufield=Ufv), T) - h_obs) ** 2))

    def same_graphs(Kv, Ufv):
        h = h0.copy()
        ha = h0.copy()
        for _ in range(T):
            ga = oracle.StepGraph(ha)
            gb = oracle.StepGraph(h)
            if not np.array_equal(ga.rec, gb.rec):
                return False
            h, _ = oracle.step(h, oracle.params(K=Kv, Ufield=Ufv))
            ha, _ = oracle.step(ha, p)
        return True

    fdK = (loss_at(K * (1 + eps), Uf) - loss_at(K * (1 - eps), Uf)) / (2 * eps * K)
    assert same_graphs(K * (1 + eps), Uf) and same_graphs(K * (1 - eps), Uf)
    assert abs(fdK - gK) <= 1e-5 * abs(gK)
    rng = np.random.default_rng(2)
    cells = rng.choice([c for c in range(nx * ny) if 0 < c % nx < nx - 1
                        and 0 < c // nx < ny - 1], 8, replace=False)
    for c in cells:
        e = np.zeros(nx * ny)
        e[c] = eps * 1e-3
        Up, Um = Uf + e.reshape(ny, nx), Uf - e.reshape(ny, nx)
        fd = (loss_at(K, Up) - loss_at(K, Um)) / (2 * eps * 1e-3)
        assert same_graphs(K, Up) and same_graphs(K, Um)
        assert abs(fd - gU.flat[c]) <= 1e-5 * max(abs(gU.flat[c]), 1e-3 * np.abs(gU).max())
