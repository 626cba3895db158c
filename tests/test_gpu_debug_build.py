"""The LEM_DEBUG build (liblem_debug.so): the same kernels with index checks
on every guarded access (an index out of range is recorded as LEM_EBOUNDS
and the access skipped, never a trap).  Small cases through every tier and
stage run clean there and give the regular build's results bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1803_02977_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cone(nx, ny, seed):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    cy = ny // 2
    h = 100.0 * np.hypot(x, y - cy) + 0.01 * synth.uniform01(seed, nx * ny).reshape(ny, nx)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 1e6
    h[cy, 0] = 0.0
    return h


def _funnel(nx, ny, seed, cx=48, cy=44, r=15.0):
    h = 100.0 + synth.uniform01(seed, nx * ny).reshape(ny, nx)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = np.hypot(x - cx, y - cy)
    inside = d <= r
    h[inside] = 50.0 + d[inside] + 0.001 * h[inside]
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


CASES = [
    ("noise_f64", lambda: synth.noise_surface(300, 211, 1), 0),
    ("noise_f32", lambda: synth.noise_surface(256, 190, 2).astype(np.float32), 0),
    ("pitch_f32", lambda: synth.noise_surface(333, 157, 3).astype(np.float32), 0),
    ("funnel_block_tier", lambda: _funnel(256, 256, 13), 0),
    ("cone_jump_tier", lambda: _cone(200, 160, 11), 0),
    ("filled_jump_tier_f32", lambda: oracle.fill(synth.noise_surface(300, 200, 5).astype(np.float32)), 0),
    ("noise_device_wide_mode", lambda: synth.noise_surface(300, 211, 6), 1),
]


def _run(make, mode):
    from paper_1803_02977_gb300 import lem
    h = torch.tensor(make(), device="cuda:0")
    m = lem.Model(h)
    lem.lem_set_step_mode(m.ctx, mode)
    m.step(3)
    m.receivers()
    q, lev, depth = m.levels()
    cnt = m.accumulate()
    m.erode()
    m.sync()  # raises LemError (LEM_EBOUNDS) if a check failed
    out = [h.cpu(), q.cpu(), lev.cpu(), cnt.cpu(), torch.tensor(lem.lem_tier_stats(m.ctx))]
    m.close()
    return out


@pytest.mark.parametrize("name,make,mode", CASES, ids=[c[0] for c in CASES])
def test_debug_build_runs_clean_and_matches(name, make, mode):
    from paper_1803_02977_gb300 import lem
    want = _run(make, mode)
    with lem.use_debug_library():
        got = _run(make, mode)
    for a, b in zip(got, want):
        assert torch.equal(a, b)
