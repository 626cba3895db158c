"""The device tier's pointer-jumping form (deep receiver trees): counts from
ranking Euler tours, erosion by composing each cell's affine update along its
receivers.  Checked step by step against the oracle's level-by-level sweep
(FP64: 1e-12 of the elevations; FP32: the one-step FP32 bound), on surfaces
whose flow paths are hundreds to thousands of cells long."""
import numpy as np
import pytest

import oracle
from paper_1803_02977_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL64 = 1e-12


def _cone(nx, ny, seed):
    # one tree draining the whole grid through a single outlet
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    cy = ny // 2
    h = 100.0 * np.hypot(x, y - cy) + 0.01 * synth.uniform01(seed, nx * ny).reshape(ny, nx)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 1e6
    h[cy, 0] = 0.0
    return h


def _tilted(nx, ny, seed, slope=0.2):
    x = np.arange(nx, dtype=np.float64)[None, :]
    h = slope * 100.0 * x + 0.01 * synth.uniform01(seed, nx * ny).reshape(ny, nx)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


def _filled_noise(nx, ny, seed, npt=np.float64):
    # depression filling leaves every cell draining to the perimeter along
    # paths that cross whole basins (filled in the elevation type itself)
    return oracle.fill(synth.noise_surface(nx, ny, seed).astype(npt))


CASES = [
    ("cone_300x300", lambda npt: _cone(300, 300, 11).astype(npt)),
    ("tilted_1500x64", lambda npt: _tilted(1500, 64, 7).astype(npt)),
    ("filled_noise_400x300", lambda npt: _filled_noise(400, 300, 12, npt)),
    ("filled_noise_1024", lambda npt: _filled_noise(1024, 1024, 13, npt)),
    # the 2048^2 workload's surface after depression filling (~3100 levels)
    ("filled_grid2048", lambda npt: oracle.fill(synth.workload("grid2048_f64").initial().astype(npt))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_jumping_tier_matches_oracle_per_step(name, make, dtype):
    from paper_1803_02977_gb300 import lem
    dev = torch.device("cuda:0")
    npt = np.float64 if dtype == "f64" else np.float32
    h0 = make(npt)
    par = dict(dx=100.0, K=2e-5, m=0.5, U=1e-3, dt=1000.0)
    p = oracle.params(**par)
    h = torch.tensor(h0.astype(npt), device=dev)
    mdl = lem.Model(h, **par)
    cur = h0.astype(npt).astype(np.float64)
    for step in range(3):
        mdl.step(1)
        mdl.sync()
        want, g = oracle.step(cur, p)
        got = h.cpu().numpy().astype(np.float64)
        if dtype == "f64":
            assert np.abs(got - want).max() <= REL64 * max(np.abs(want).max(), 1.0), step
        else:
            tol = 4 * 2.0 ** -24 * np.maximum(np.abs(want), 1.0)
            assert np.all(np.abs(got - want) <= tol), step
        cur = got
    js, rounds = lem.lem_jump_stats(mdl.ctx)
    tiers = lem.lem_tier_stats(mdl.ctx)
    mdl.close()
    assert js >= 1, f"the pointer-jumping tier did not run ({g.nlevels} levels)"
    assert sum(tiers) == 3 * h0.size
    assert rounds >= 1


def test_deep_steps_are_deterministic():
    """Which tier takes a tree does not depend on timing (overflowed tiles
    are owned by block by tile index), so repeated runs agree bit for bit."""
    from paper_1803_02977_gb300 import lem
    dev = torch.device("cuda:0")
    h0 = _filled_noise(400, 300, 22)
    par = dict(dx=100.0, K=2e-5, m=0.5, U=1e-3, dt=1000.0)
    outs = []
    for _ in range(3):
        h = torch.tensor(h0, device=dev)
        m = lem.Model(h, **par)
        for _ in range(3):
            m.step(1)
        m.sync()
        outs.append((h.cpu(), lem.lem_tier_stats(m.ctx), lem.lem_jump_stats(m.ctx)))
        m.close()
    for o in outs[1:]:
        assert torch.equal(o[0], outs[0][0])
        assert o[1] == outs[0][1] and o[2] == outs[0][2]
    assert outs[0][2][0] >= 1


def test_jumping_tier_in_a_multi_step_launch_equals_single_launches():
    from paper_1803_02977_gb300 import lem
    dev = torch.device("cuda:0")
    h0 = _filled_noise(300, 200, 21)  # FP64
    par = dict(dx=100.0, K=2e-5, m=0.5, U=1e-3, dt=1000.0)
    ha = torch.tensor(h0, device=dev)
    hb = torch.tensor(h0, device=dev)
    ma, mb = lem.Model(ha, **par), lem.Model(hb, **par)
    ma.step(4)
    for _ in range(4):
        mb.step(1)
    ma.sync()
    mb.sync()
    assert lem.lem_jump_stats(ma.ctx)[0] >= 1
    assert torch.equal(ha, hb)
    ma.close()
    mb.close()
