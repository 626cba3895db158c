"""The hand-written adjoint (lem_adjoint through torch.autograd) against the
FP64 oracle adjoint and central finite differences (eps = 1e-6)."""
import numpy as np
import pytest

import oracle
from paper_1803_02977_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(nx=48, ny=40, seed=31, T=8, K=2e-5):
    h0 = synth.noise_surface(nx, ny, seed)
    h0[1:-1, 1:-1] += 2.0
    Uf = 1e-3 * (1.0 + 0.3 * synth.signed_field(nx, ny, seed + 1))
    # observations from a run at perturbed parameters
    Uobs = Uf * (1.0 + 0.1 * synth.signed_field(nx, ny, seed + 2))
    h_obs = oracle.run(h0, oracle.params(K=1.2 * K, Ufield=Uobs), T)
    return h0, Uf, h_obs, K, T


def _gpu_grad(h0, Uf, h_obs, K, T, ckpt):
    from paper_1803_02977_gb300 import autodiff
    dev = torch.device("cuda:0")
    h0t = torch.tensor(h0, device=dev, requires_grad=True)
    Ut = torch.tensor(Uf, device=dev, requires_grad=True)
    Kt = torch.tensor(K, dtype=torch.float64, device=dev, requires_grad=True)
    hT = autodiff.run(h0t, Ut, Kt, T, ckpt_every=ckpt)
    loss = torch.sum((hT - torch.tensor(h_obs, device=dev)) ** 2)
    loss.backward()
    return (loss.item(), Ut.grad.cpu().numpy(), Kt.grad.item(), h0t.grad.cpu().numpy())


@pytest.mark.parametrize("ckpt", [1, 3, 8])
def test_adjoint_matches_oracle_adjoint(ckpt):
    h0, Uf, h_obs, K, T = _problem()
    loss_o, gU_o, gK_o = oracle.loss_and_grad(h0, oracle.params(K=K, Ufield=Uf), T, h_obs)
    loss, gU, gK, gh0 = _gpu_grad(h0, Uf, h_obs, K, T, ckpt)
    assert abs(loss - loss_o) <= 1e-10 * abs(loss_o)
    assert np.abs(gU - gU_o).max() <= 1e-9 * np.abs(gU_o).max()
    assert abs(gK - gK_o) <= 1e-9 * abs(gK_o)
    # perimeter carries no uplift
    assert np.all(gU[0, :] == 0) and np.all(gU[:, 0] == 0)


def test_adjoint_independent_of_checkpoint_spacing():
    h0, Uf, h_obs, K, T = _problem(seed=41, T=7)
    ref = _gpu_grad(h0, Uf, h_obs, K, T, 1)
    for ckpt in (2, 7):
        got = _gpu_grad(h0, Uf, h_obs, K, T, ckpt)
        assert np.array_equal(got[1], ref[1]) and got[2] == ref[2]


def test_adjoint_matches_central_finite_differences():
    from paper_1803_02977_gb300 import autodiff
    nx, ny = 40, 36
    h0, Uf, h_obs, K, T = _problem(nx, ny, seed=51, T=6)
    dev = torch.device("cuda:0")
    h_obs_t = torch.tensor(h_obs, device=dev)

    def loss_at(Kv, Ufv):
        hT = autodiff.run(torch.tensor(h0, device=dev), torch.tensor(Ufv, device=dev),
                          torch.tensor(Kv, dtype=torch.float64), T)
        return float(torch.sum((hT - h_obs_t) ** 2))

    def same_graphs(Kv, Ufv):
        # every step's receivers equal those of the unperturbed run (oracle)
        ha, hb = h0.copy(), h0.copy()
        for _ in range(T):
            if not np.array_equal(oracle.receivers(ha), oracle.receivers(hb)):
                return False
            ha, _ = oracle.step(ha, oracle.params(K=K, Ufield=Uf))
            hb, _ = oracle.step(hb, oracle.params(K=Kv, Ufield=Ufv))
        return True

    _, gU, gK, _ = _gpu_grad(h0, Uf, h_obs, K, T, 3)
    eps = 1e-6
    fdK = (loss_at(K * (1 + eps), Uf) - loss_at(K * (1 - eps), Uf)) / (2 * eps * K)
    assert same_graphs(K * (1 + eps), Uf) and same_graphs(K * (1 - eps), Uf)
    assert abs(fdK - gK) <= 1e-5 * abs(gK)
    rng = np.random.default_rng(3)
    interior = [c for c in range(nx * ny) if 0 < c % nx < nx - 1 and 0 < c // nx < ny - 1]
    dirs = [np.eye(1, nx * ny, c).reshape(ny, nx) for c in rng.choice(interior, 20, replace=False)]
    dirs += [rng.standard_normal((ny, nx)) for _ in range(3)]
    checked = 0
    for v in dirs:
        step = eps * 1e-3
        Up, Um = Uf + step * v, Uf - step * v
        if not (same_graphs(K, Up) and same_graphs(K, Um)):
            continue  # a receiver flipped: the loss is not differentiable there
        fd = (loss_at(K, Up) - loss_at(K, Um)) / (2 * step)
        ad = float(np.sum(gU * v))
        assert abs(fd - ad) <= 1e-5 * max(abs(ad), 1e-6 * np.abs(gU).max()), (fd, ad)
        checked += 1
    assert checked >= 20


def _funnel(nx, ny, seed, cx=48, cy=44, r=15.0):
    # one basin of ~700 cells around a single pit: deeper than an adjoint
    # warp tile holds, so every backward step reruns on device-wide levels
    h = 100.0 + synth.uniform01(seed, nx * ny).reshape(ny, nx)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = np.hypot(x - cx, y - cy)
    inside = d <= r
    h[inside] = 50.0 + d[inside] + 0.001 * h[inside]
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


def _cone(nx, ny, seed):
    # one tree draining the whole grid through a single outlet
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    cy = ny // 2
    h = 100.0 * np.hypot(x, y - cy) + 0.01 * synth.uniform01(seed, nx * ny).reshape(ny, nx)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 1e6
    h[cy, 0] = 0.0
    return h


@pytest.mark.parametrize("name,make", [("funnel_160x120", lambda: _funnel(160, 120, 13)),
                                       ("cone_90x70", lambda: _cone(90, 70, 11))])
def test_adjoint_device_wide_fallback_matches_oracle(name, make):
    """Trees that outgrow a warp's tile send the backward step to its
    device-wide form (lem_step_stats counts it): dL/dU, dL/dK and dL/dh0 must
    still match the oracle adjoint."""
    from paper_1803_02977_gb300 import lem
    dev = torch.device("cuda:0")
    h0 = make()
    ny, nx = h0.shape
    T, K = 4, 2e-5
    Uf = 1e-3 * (1.0 + 0.3 * synth.signed_field(nx, ny, 61))
    h_obs = oracle.run(h0, oracle.params(K=1.2 * K, Ufield=Uf * 1.05), T)
    loss_o, gU_o, gK_o = oracle.loss_and_grad(h0, oracle.params(K=K, Ufield=Uf), T, h_obs)
    # the run's final state, for lambda_T = dL/dh_T
    hT = oracle.run(h0, oracle.params(K=K, Ufield=Uf), T)
    h0t = torch.tensor(h0, device=dev)
    mdl = lem.Model(h0t.clone(), dx=100.0, K=K, m=0.5, U=0.0, dt=1000.0)
    Ut = torch.tensor(Uf, device=dev)
    mdl.set_uplift_field(Ut)
    lamT = torch.tensor(2.0 * (hT - h_obs), device=dev)
    dU = torch.empty_like(h0t)
    lam0 = torch.empty_like(h0t)
    dK = lem.lem_adjoint(mdl.ctx, h0t, lamT, T, 2, dU, lam0)
    priv, wide = lem.lem_step_stats(mdl.ctx)
    mdl.close()
    # lem_adjoint runs 2T forward steps (first pass and recomputation); every
    # further device-wide step counted is a backward step's fallback
    fallbacks = priv + wide - 2 * T
    assert fallbacks >= 1, (priv, wide)
    gU = dU.cpu().numpy()
    assert np.abs(gU - gU_o).max() <= 1e-9 * np.abs(gU_o).max()
    assert abs(dK - gK_o) <= 1e-9 * abs(gK_o)


def test_adjoint_gradient_1024_workload_50_steps():
    """The adjoint workload (1024^2 FP64, 50 steps, checkpoints every 10):
    dL/dU at every cell and dL/dK against the oracle adjoint."""
    w = synth.workload("grid1024_adjoint")
    h0 = w.initial()
    xi = synth.signed_field(w.nx, w.ny, 6)
    U = np.full_like(h0, w.U)
    p_obs = oracle.params(dx=w.dx, K=1.2 * w.K, m=w.m, dt=w.dt, U=0.0, Ufield=U * (1 + 0.1 * xi))
    h_obs = oracle.run(h0, p_obs, w.steps)
    p = oracle.params(dx=w.dx, K=w.K, m=w.m, dt=w.dt, U=0.0, Ufield=U)
    loss_o, gU_o, gK_o = oracle.loss_and_grad(h0, p, w.steps, h_obs)
    from paper_1803_02977_gb300 import autodiff
    dev = torch.device("cuda:0")
    Ut = torch.tensor(U, device=dev, requires_grad=True)
    Kt = torch.tensor(w.K, dtype=torch.float64, device=dev, requires_grad=True)
    hT = autodiff.run(torch.tensor(h0, device=dev), Ut, Kt, w.steps, ckpt_every=10, dx=w.dx,
                      m=w.m, dt=w.dt)
    loss = torch.sum((hT - torch.tensor(h_obs, device=dev)) ** 2)
    loss.backward()
    gU = Ut.grad.cpu().numpy()
    print(f"\nadjoint 1024^2, 50 steps: loss {loss.item():.6e} (oracle {loss_o:.6e}), dL/dK "
          f"{Kt.grad.item():.6e} (oracle {gK_o:.6e}), max |dL/dU - oracle| "
          f"{np.abs(gU - gU_o).max():.3e} of max {np.abs(gU_o).max():.3e}")
    assert abs(loss.item() - loss_o) <= 1e-10 * abs(loss_o)
    assert np.abs(gU - gU_o).max() <= 1e-9 * np.abs(gU_o).max()
    assert abs(Kt.grad.item() - gK_o) <= 1e-9 * abs(gK_o)
