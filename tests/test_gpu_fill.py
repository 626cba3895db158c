"""Depression filling on the GPU (lem_fill: Priority-Flood with epsilon
increments as a relaxation over 32 x 32 tiles) against the oracle's
priority-queue flood, bit for bit, in FP64 and FP32; then the time step with
filling turned on against the oracle's fill followed by its step."""
import numpy as np
import pytest

import oracle
from paper_1803_02977_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL64 = 1e-12


def _lem():
    from paper_1803_02977_gb300 import lem
    return lem


def _dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda:0")


def _int_grid(nx, ny, seed, levels=4):
    u = synth.uniform01(seed, nx * ny).reshape(ny, nx)
    h = np.floor(u * levels)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


def _bowl(nx, ny, seed):
    # one depression spanning many tiles: a rim at 50 m around a basin whose
    # floor lies at about 10 m, with its outlet on the west side at 20 m
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = np.hypot(x - nx / 2, y - ny / 2) / (0.45 * min(nx, ny))
    h = np.where(d < 1.0, 10.0 + 5.0 * d, 50.0) + synth.uniform01(seed, nx * ny).reshape(ny, nx)
    band = (np.abs(y - ny / 2) < 2) & (x < nx / 2)
    h[band & (d >= 1.0)] = 20.0
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


def _serpentine(n):
    # one walled corridor winding back and forth across the grid, open to the
    # west edge at its start: its flood path crosses the same tiles again and
    # again, so the flood needs many rounds
    h = np.full((n, n), 100.0)
    rows = list(range(2, n - 2, 4))
    for i, y in enumerate(rows):
        h[y, 2:n - 2] = 1.0
        if i + 1 < len(rows):
            x = n - 3 if i % 2 == 0 else 2
            h[y:rows[i + 1] + 1, x] = 1.0
    h[2, 1] = 1.0  # the opening
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


CASES = [
    ("3x3", lambda: synth.noise_surface(3, 3, 1)),
    ("5x4", lambda: synth.noise_surface(5, 4, 2)),
    ("noise_40x33", lambda: synth.noise_surface(40, 33, 3)),
    ("noise_97x61", lambda: synth.noise_surface(97, 61, 4)),
    ("int_flats_100x80", lambda: _int_grid(100, 80, 5)),
    ("plateau_70x70", lambda: np.pad(np.full((68, 68), 7.0), 1)),
    ("all_flat_64x64", lambda: np.zeros((64, 64))),
    ("tilt_300x200", lambda: synth.noise_surface(300, 200, 6, south_tilt=1e-1)),
    ("bowl_500x400", lambda: _bowl(500, 400, 7)),
    ("serpentine_200", lambda: _serpentine(200)),
    ("noise_1031x777", lambda: synth.noise_surface(1031, 777, 8)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_fill_bit_exact(name, make, dtype):
    lem = _lem()
    h0 = make().astype(dtype)
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h)
    mdl.fill()
    mdl.sync()
    want = oracle.fill(h0)
    got = h.cpu().numpy()
    assert got.dtype == want.dtype
    assert np.array_equal(got, want), f"{name}: {np.count_nonzero(got != want)} cells differ"
    rounds, visits, passes, _ = lem.lem_fill_stats(mdl.ctx)
    assert rounds >= 1 and passes >= visits >= 0
    # filling a filled surface changes nothing
    mdl.fill()
    mdl.sync()
    assert np.array_equal(h.cpu().numpy(), want)
    mdl.close()


def test_no_interior_sink_after_fill():
    lem = _lem()
    h0 = synth.noise_surface(300, 257, 9)
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h)
    mdl.fill()
    rec = mdl.receivers().cpu().numpy()
    q, lev, depth = mdl.levels()
    ny, nx = h0.shape
    interior = np.zeros((ny, nx), bool)
    interior[1:-1, 1:-1] = True
    assert np.all((rec != np.arange(nx * ny)) == interior.ravel())
    # level 0 is exactly the perimeter
    assert int(lev[1]) == 2 * nx + 2 * ny - 4
    mdl.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_step_with_fill_matches_oracle(mode):
    lem = _lem()
    w = synth.workload("grid256_f64")
    p = oracle.params(dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
    h0 = w.initial()
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h, dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
    lem.lem_set_step_mode(mdl.ctx, mode)
    mdl.set_fill(True)
    for _ in range(3):
        before = h.cpu().numpy()
        mdl.step(1)
        mdl.sync()
        want, g = oracle.step(oracle.fill(before), p)
        assert g.nlevels >= 2 and g.levels[1] == 2 * 256 + 2 * 256 - 4  # sinks: the perimeter
        got = h.cpu().numpy()
        assert np.abs(got - want).max() <= REL64 * max(np.abs(want).max(), 1.0)
    # turning it off returns to the plain step
    mdl.set_fill(False)
    before = h.cpu().numpy()
    mdl.step(1)
    mdl.sync()
    want, _ = oracle.step(before, p)
    assert np.abs(h.cpu().numpy() - want).max() <= REL64 * max(np.abs(want).max(), 1.0)
    mdl.close()


def test_fill_with_newton_step():
    lem = _lem()
    h0 = synth.noise_surface(180, 140, 10)
    par = dict(dx=100.0, K=0.02, m=0.5, U=1e-3, dt=1000.0)
    p = oracle.params(**par)
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h, **par)
    mdl.set_fill(True)
    mdl.set_slope_exponent(2.0, 1e-12, 100)
    mdl.step(1)
    mdl.sync()
    want, _ = oracle.step_newton(oracle.fill(h0), p, 2.0, 1e-12, 100)
    assert np.abs(h.cpu().numpy() - want).max() <= REL64 * max(np.abs(want).max(), 1.0)
    mdl.close()


def test_grid2048_f64_fill_bit_exact():
    # the benchmark's workload: 2048^2 noise with a south tilt
    lem = _lem()
    w = synth.workload("grid2048_f64")
    h0 = w.initial()
    h = torch.tensor(h0, device=_dev())
    mdl = lem.Model(h, dx=w.dx, K=w.K, m=w.m, U=w.U, dt=w.dt)
    mdl.fill()
    mdl.sync()
    assert np.array_equal(h.cpu().numpy(), oracle.fill(h0))
    mdl.close()


def test_fill_argument_checks():
    lem = _lem()
    h = torch.tensor(synth.noise_surface(16, 16, 11), device=_dev())
    mdl = lem.Model(h)
    assert lem.lib().lem_set_fill(mdl.ctx, 2) == lem.LEM_EINVAL
    assert lem.lib().lem_fill(None) == lem.LEM_EINVAL
    assert lem.lem_fill_stats(mdl.ctx) == (0, 0, 0, 0)  # no flood yet
    mdl.close()
