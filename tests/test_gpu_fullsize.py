"""Parity at the full sizes the benchmark times, in the launch configuration it
times (one tiered-step launch per step, the batch in one launch):

- 2048 x 2048 FP64 grid (noise plus a south tilt): every cell against the
  oracle after each of several single-step launches, and every cell handled
  by exactly one tier in each step;
- 10000 x 10000 FP32 grid with int64 counts (the paper's largest size): one
  step, every cell against the FP64 oracle run on the same FP32 input;
- 512 FP32 realizations of 128^2 .. 1024^2 cells in one batch launch, for
  every kernel shape the autotuner chooses from: sampled realizations against
  the oracle, and on every realization the properties that hold at any size
  (perimeter cells keep their elevation; no cell rises above its uplifted
  elevation; all elevations finite)."""
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


def _oracle_params(w):
    return oracle.params(dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)


def test_grid2048_f64_every_cell_per_step():
    lem = _lem()
    w = synth.workload("grid2048_f64")
    p = _oracle_params(w)
    h0 = w.initial()
    h = torch.tensor(h0, device="cuda:0")
    mdl = lem.Model(h, dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
    cur = h0
    nsteps = 4
    for _ in range(nsteps):
        mdl.step(1)
        mdl.sync()
        want = oracle.run(cur, p, 1)
        got = h.cpu().numpy()
        err = np.abs(got - want).max()
        assert err <= REL64 * max(np.abs(want).max(), 1.0), err
        cur = got
    tiers = lem.lem_tier_stats(mdl.ctx)
    assert sum(tiers) == nsteps * h0.size  # each cell handled once per step
    mdl.close()


def test_grid10000_f32_one_step_every_cell():
    lem = _lem()
    w = synth.workload("grid10000_f32")
    h0 = w.initial().astype(np.float32)
    h = torch.tensor(h0, device="cuda:0")
    mdl = lem.Model(h, dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt, count_bits=64)
    mdl.step(1)
    mdl.sync()
    got = h.cpu().numpy().astype(np.float64)
    tiers = lem.lem_tier_stats(mdl.ctx)
    mdl.close()
    del h
    assert sum(tiers) == h0.size
    want = oracle.run(h0.astype(np.float64), _oracle_params(w), 1)
    # one step in FP32 arithmetic from the same FP32 input: a few roundings
    tol = 4 * ULP32 * np.maximum(np.abs(want), 1.0)
    bad = np.abs(got - want) > tol
    assert not bad.any(), f"{int(bad.sum())} cells beyond 4 ulp"


def test_batch512_f32_every_shape_sampled_against_oracle():
    lem = _lem()
    bw = synth.batch_workload(count=512)
    surfaces = [bw.initial(r).astype(np.float32) for r in range(bw.count)]
    B = lem.Batch(surfaces, dx=bw.dx, K=bw.K, m=bw.m, U=bw.U, dt=bw.dt)
    R = B.R
    sides = np.array(bw.sides)
    rng = np.random.default_rng(17)
    sample = sorted({int(np.argmax(sides)), int(np.argmin(sides)),
                     *rng.choice(R, size=6, replace=False).tolist()})
    want = {}
    for r in sample:
        p = oracle.params(dx=bw.dx, K=bw.K[r], m=bw.m[r], U=bw.U, dt=bw.dt)
        want[r] = oracle.run(surfaces[r].astype(np.float64), p, 1)
    saved = B.h.clone()
    udt = bw.U * bw.dt
    for bd, pi in lem.BATCH_CONFIGS:
        B.h.copy_(saved)
        B.set_config(bd, pi)
        B.step(1)
        B.sync()
        for r in sample:
            got = B.surface(r).cpu().numpy().astype(np.float64)
            tol = 4 * ULP32 * np.maximum(np.abs(want[r]), 1.0)
            assert np.all(np.abs(got - want[r]) <= tol), f"shape {bd}x{pi}, realization {r}"
        for r in range(R):
            got = B.surface(r).cpu().numpy()
            src = surfaces[r]
            assert np.isfinite(got).all(), f"shape {bd}x{pi}, realization {r}"
            edge = np.ones(src.shape, bool)
            edge[1:-1, 1:-1] = False
            assert np.array_equal(got[edge], src[edge]), f"shape {bd}x{pi}, realization {r}"
            up = src[1:-1, 1:-1].astype(np.float64) + udt
            assert np.all(got[1:-1, 1:-1] <= up * (1 + 4 * ULP32) + 4 * ULP32), \
                f"shape {bd}x{pi}, realization {r}"
    B.close()
