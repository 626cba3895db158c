"""Parity of Alg 6 for a general slope exponent n-hat (lem_set_slope_exponent:
the Newton-Raphson erosion sweep) against the oracle's Newton iteration on
identical inputs: FP64 elevations within 1e-12 relative per step, FP32 within
the FP32 bound; the stages before it stay bit-exact.  Also the argument
checks, the return to the n-hat = 1 closed form, the adjoint's refusal and a
full-size 2048 x 2048 step checked at every cell."""
import numpy as np
import pytest

import oracle
from paper_1803_02977_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL64 = 1e-12
ULP32 = 2.0 ** -24


def _lem():
    from paper_1803_02977_gb300 import lem
    return lem


def _dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda:0")


def _tilted(nx, ny, seed, slope=0.05):
    x = np.arange(nx, dtype=np.float64)[None, :]
    h = slope * 100.0 * x + 0.01 * synth.uniform01(seed, nx * ny).reshape(ny, nx)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


def _rel(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1.0))


CASES = [
    # name, surface, n-hat, K (large K: F of order one, several Newton updates)
    ("3x3_n2", lambda: synth.noise_surface(3, 3, 1), 2.0, 1e-5),
    ("5x4_n1.5", lambda: synth.noise_surface(5, 4, 2), 1.5, 0.05),
    ("67x45_n2", lambda: synth.noise_surface(67, 45, 3), 2.0, 0.1),
    ("333x517_n1.5", lambda: synth.noise_surface(333, 517, 5), 1.5, 1e-3),
    ("tilted_300x200_n3", lambda: _tilted(300, 200, 6), 3.0, 1e-2),
    ("tilted_1500x64_n1.2", lambda: _tilted(1500, 64, 7, slope=0.2), 1.2, 1e-4),
    ("256x256_n2", lambda: synth.noise_surface(256, 256, 1), 2.0, 1e-5),
]


@pytest.mark.parametrize("name,make,n_exp,K", CASES, ids=[c[0] for c in CASES])
def test_step_matches_oracle_newton_per_step(name, make, n_exp, K):
    lem = _lem()
    h0 = make()
    par = dict(dx=100.0, K=K, m=0.5, U=1e-3, dt=1000.0)
    p = oracle.params(**par)
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h, **par)
    mdl.set_slope_exponent(n_exp, 1e-12, 100)
    cur = h0
    moved = 0.0
    for _ in range(3):
        mdl.step(1)
        mdl.sync()
        want, _ = oracle.step_newton(cur, p, n_exp, 1e-12, 100)
        got = h.cpu().numpy()
        assert _rel(got, want) <= REL64, name
        up = cur.copy()
        oracle.uplift(up, p)
        moved = max(moved, float(np.abs(want - up).max()))
        cur = got
    mdl.close()
    if h0.size > 9:
        assert moved > 0.0  # erosion took place


def test_stage_calls_newton_bit_exact_graph_and_erosion():
    lem = _lem()
    nx, ny = 211, 157
    h0 = synth.noise_surface(nx, ny, 11)
    par = dict(dx=100.0, K=0.02, m=0.45, U=1e-3, dt=1000.0)
    p = oracle.params(**par)
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h, **par)
    mdl.set_slope_exponent(3.0, 1e-13, 200)
    rec = mdl.receivers()
    q, lev, depth = mdl.levels()
    cnt = mdl.accumulate()
    mdl.erode()
    mdl.sync()
    g = oracle.StepGraph(h0)
    assert np.array_equal(rec.cpu().numpy(), g.rec)
    assert np.array_equal(q.cpu().numpy(), g.queue)
    assert np.array_equal(lev.cpu().numpy(), g.levels)
    assert np.array_equal(cnt.cpu().numpy(), g.cnt)
    want = h0.copy()
    oracle.uplift(want, p)
    oracle.erode_newton(want, g.rec, g.queue, g.levels, g.cnt, p, 3.0, 1e-13, 200)
    assert _rel(h.cpu().numpy(), want) <= REL64
    mdl.close()


def test_one_update_fixed_count():
    # max_iter = 1: a single Newton update from h0 (Alg 6's fixed-count form)
    lem = _lem()
    h0 = synth.noise_surface(120, 90, 12)
    par = dict(dx=100.0, K=0.05, m=0.5, U=1e-3, dt=1000.0)
    p = oracle.params(**par)
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h, **par)
    mdl.set_slope_exponent(2.5, 1e-12, 1)
    mdl.step(1)
    mdl.sync()
    want, _ = oracle.step_newton(h0, p, 2.5, 1e-12, 1)
    full, _ = oracle.step_newton(h0, p, 2.5, 1e-12, 100)
    assert _rel(h.cpu().numpy(), want) <= REL64
    assert np.abs(want - full).max() > 1e-9  # one update is not yet the root
    mdl.close()


def test_fp32_newton_within_fp32_bound():
    lem = _lem()
    nx, ny = 300, 200
    w = synth.workload("grid2048_f32")
    h0 = synth.noise_surface(nx, ny, 13).astype(np.float32)
    par = dict(dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
    p = oracle.params(**par)
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h, **par)
    mdl.set_slope_exponent(2.0, 1e-9, 100)
    mdl.step(1)
    mdl.sync()
    g = oracle.StepGraph(h0)
    want = h0.astype(np.float64)
    oracle.uplift(want, p)
    oracle.erode_newton(want, g.rec, g.queue, g.levels, g.cnt, p, 2.0, 1e-9, 100)
    got = h.cpu().numpy().astype(np.float64)
    assert np.abs(got - want).max() <= 4 * ULP32 * max(np.abs(want).max(), 1.0)
    mdl.close()


def test_int64_counts_and_uplift_field_with_no_downhill_cells():
    # a per-cell uplift that lifts some receivers above their donors' uplifted
    # elevations: those donors keep h0 (the reading for n-hat != 1)
    lem = _lem()
    nx, ny = 97, 83
    h0 = synth.noise_surface(nx, ny, 14)
    Uf = 1e-3 * (1.0 + 400.0 * (synth.uniform01(15, nx * ny) > 0.9))
    par = dict(dx=100.0, K=0.01, m=0.5, U=1e-3, dt=1000.0)
    p = oracle.params(Ufield=Uf, **par)
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h, count_bits=64, **par)
    mdl.set_uplift_field(torch.tensor(Uf, device=_dev()))
    mdl.set_slope_exponent(1.5, 1e-12, 100)
    mdl.step(1)
    mdl.sync()
    want, g = oracle.step_newton(h0, p, 1.5, 1e-12, 100)
    assert _rel(h.cpu().numpy(), want) <= REL64
    # the guard was exercised: some eroding cell kept its uplifted elevation
    up = h0.copy()
    oracle.uplift(up, p)
    eroding = np.array([g.rec[c] != c for c in range(nx * ny)]).reshape(ny, nx)
    assert np.any(eroding & (want == up))
    mdl.close()


def test_frozen_channel_steady_state_general_n():
    lem = _lem()
    nx, dx, K, m, U, dt, n_exp = 40, 100.0, 1e-5, 0.5, 1e-3, 1000.0, 1.5
    area = dx * dx
    h0 = np.zeros((3, nx))
    for x in range(1, nx - 1):
        h0[1, x] = h0[1, x - 1] + dx * (U / (K * ((nx - 1 - x) * area) ** m)) ** (1.0 / n_exp)
    rec = np.arange(3 * nx, dtype=np.int32)
    for x in range(1, nx - 1):
        rec[nx + x] = nx + x - 1
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h, dx=dx, K=K, m=m, U=U, dt=dt)
    mdl.set_receivers(torch.tensor(rec, device=_dev()))
    mdl.set_slope_exponent(n_exp, 1e-13, 100)
    mdl.step(2)
    mdl.sync()
    assert np.abs(h.cpu().numpy() - h0).max() <= 1e-11 * np.abs(h0).max()
    mdl.close()


def test_arguments_reset_and_adjoint_refusal():
    lem = _lem()
    h0 = synth.noise_surface(64, 48, 16)
    par = dict(dx=100.0, K=1e-5, m=0.5, U=1e-3, dt=1000.0)
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h, **par)
    for bad in [(0.5, 1e-12, 10), (float("nan"), 1e-12, 10), (float("inf"), 1e-12, 10),
                (2.0, 0.0, 10), (2.0, -1.0, 10), (2.0, float("nan"), 10), (2.0, 1e-12, 0),
                (2.0, 1e-12, 1001)]:
        with pytest.raises(lem.LemError) as e:
            mdl.set_slope_exponent(*bad)
        assert e.value.status == lem.LEM_EINVAL
    mdl.set_slope_exponent(2.0, 1e-12, 50)
    lam = torch.ones_like(h)
    dU = torch.zeros_like(h)
    with pytest.raises(lem.LemError) as e:
        lem.lem_adjoint(mdl.ctx, h.clone(), lam, 2, 1, dU)
    assert e.value.status == lem.LEM_EINVAL
    # n = 1 restores the closed form (and the tiered step)
    mdl.set_slope_exponent(1.0)
    mdl.step(1)
    mdl.sync()
    want = oracle.run(h0, oracle.params(**par), 1)
    assert _rel(h.cpu().numpy(), want) <= REL64
    mdl.close()


def test_grid2048_f64_n2_every_cell():
    # the benchmark's general-exponent form: 2048^2 FP64, n-hat = 2
    lem = _lem()
    w = synth.workload("grid2048_f64")
    h0 = w.initial()
    par = dict(dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
    p = oracle.params(**par)
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h, **par)
    mdl.set_slope_exponent(2.0, 1e-12, 100)
    cur = h0
    for _ in range(2):
        mdl.step(1)
        mdl.sync()
        want, _ = oracle.step_newton(cur, p, 2.0, 1e-12, 100)
        got = h.cpu().numpy()
        assert _rel(got, want) <= REL64
        cur = got
    mdl.close()


def test_newton_runs_in_the_private_tiers_and_matches_device_wide():
    # the tiered step (mode 0) solves Newton in the warp tile forests; mode 1
    # runs every cell on the device-wide levels; both give the oracle's result
    lem = _lem()
    h0 = synth.noise_surface(256, 256, 17)
    par = dict(dx=100.0, K=0.05, m=0.5, U=1e-3, dt=1000.0)
    p = oracle.params(**par)
    want, _ = oracle.step_newton(h0, p, 1.5, 1e-12, 100)
    got = {}
    for mode in (0, 1):
        h = torch.tensor(h0, device=_dev())
        mdl = lem.Model(h, **par)
        lem.lem_set_step_mode(mdl.ctx, mode)
        mdl.set_slope_exponent(1.5, 1e-12, 100)
        mdl.step(1)
        mdl.sync()
        got[mode] = h.cpu().numpy()
        if mode == 0:
            warp, block, device = lem.lem_tier_stats(mdl.ctx)
            assert warp > 0 and warp + block + device == h0.size
        mdl.close()
    for mode in (0, 1):
        assert _rel(got[mode], want) <= REL64
