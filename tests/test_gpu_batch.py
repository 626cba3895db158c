"""The batched form: every realization advanced in one launch must equal the
same grid advanced alone by the FP32 single-grid path (identical arithmetic),
for every kernel shape, and stay within the FP32 bound of the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1803_02977_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _funnel(nx, ny, seed, cx, cy, r):
    # one basin of ~pi*r^2 cells around a single pit in a noise field: too
    # many for a warp's queue, so its tile is finished by the block-wide forest
    h = 100.0 + synth.uniform01(seed, nx * ny).reshape(ny, nx)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d = np.hypot(x - cx, y - cy)
    inside = d <= r
    h[inside] = 50.0 + d[inside] + 0.001 * h[inside]
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


def _realizations(R=11, seed=4):
    u = synth.uniform01(seed, 4 * R).reshape(R, 4)
    shapes = [(int(3 + u[r, 0] * 300), int(3 + u[r, 1] * 260)) for r in range(R)]
    shapes[0] = (3, 3)          # degenerate: one interior cell
    shapes[1] = (513, 7)        # ragged, very wide
    Ks = [float(10 ** (-6 + 2 * u[r, 2])) for r in range(R)]
    ms = [float(0.4 + 0.2 * u[r, 3]) for r in range(R)]
    surfaces = [synth.noise_surface(nx, ny, 1000 + r) for r, (nx, ny) in enumerate(shapes)]
    surfaces[2] = _funnel(97, 83, 1002, cx=40, cy=41, r=16.0)
    return surfaces, Ks, ms


def _singles(surfaces, Ks, ms, steps):
    from paper_1803_02977_gb300 import lem
    out = []
    for i, (s, K, m) in enumerate(zip(surfaces, Ks, ms)):
        h = torch.tensor(s.astype(np.float32), device="cuda:0")
        mdl = lem.Model(h, dx=100.0, K=K, m=m, U=1e-3, dt=1000.0)
        mdl.step(steps)
        mdl.sync()
        if i == 2:  # the funnel exercises the fallback tier in both paths
            assert lem.lem_tier_stats(mdl.ctx)[1] > 0
        out.append(h.cpu().numpy())
        mdl.close()
    return out


def _ramp(nx, ny, seed):
    # a plane falling toward the west edge plus small noise: trees as long as
    # the grid is wide, hundreds of levels, all in the block-wide forest
    x = np.arange(nx, dtype=np.float64)[None, :]
    h = 5.0 * x + 0.01 * synth.uniform01(seed, nx * ny).reshape(ny, nx)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


@pytest.mark.parametrize("shape", [(256, 4), (1024, 8)])
def test_batch_deep_forests_against_oracle(shape):
    """Trees hundreds of levels deep (the block-wide forest: level offsets in
    shared memory, counts pushed to the receivers) per step against the
    oracle, with shallow realizations beside them."""
    from paper_1803_02977_gb300 import lem
    surfaces = [_ramp(700, 40, 21), _funnel(97, 83, 1002, cx=40, cy=41, r=16.0),
                synth.noise_surface(129, 65, 5), _ramp(310, 300, 22)]
    Ks, ms = [2e-5, 1e-5, 3e-5, 1e-6], [0.5, 0.45, 0.55, 0.6]
    b = lem.Batch(surfaces, dx=100.0, K=Ks, m=ms, U=1e-3, dt=1000.0)
    b.set_config(*shape)
    for _ in range(2):
        before = [b.surface(r).cpu().numpy().astype(np.float64) for r in range(b.R)]
        b.step(1)
        b.sync()
        for r in range(b.R):
            want, g = oracle.step(before[r], oracle.params(K=Ks[r], m=ms[r]))
            if r in (0, 3):
                assert g.levels.size - 1 > 250  # deep: far beyond a warp's 127 levels
            got = b.surface(r).cpu().numpy().astype(np.float64)
            tol = 4 * 2.0 ** -24 * np.maximum(np.abs(want), 1.0)
            assert np.all(np.abs(got - want) <= tol), f"realization {r}"
    b.close()


@pytest.mark.parametrize("shape", [(256, 4), (256, 8), (512, 4), (512, 8), (1024, 4), (1024, 8)])
def test_batch_equals_single_grid_path(shape):
    from paper_1803_02977_gb300 import lem
    surfaces, Ks, ms = _realizations()
    steps = 3
    b = lem.Batch(surfaces, dx=100.0, K=Ks, m=ms, U=1e-3, dt=1000.0)
    b.set_config(*shape)
    b.step(steps)
    b.sync()
    want = _singles(surfaces, Ks, ms, steps)
    for r in range(b.R):
        assert np.array_equal(b.surface(r).cpu().numpy(), want[r]), f"realization {r}"
    b.close()


def test_batch_per_step_against_oracle():
    from paper_1803_02977_gb300 import lem
    surfaces, Ks, ms = _realizations(R=5, seed=9)
    b = lem.Batch(surfaces, dx=100.0, K=Ks, m=ms, U=1e-3, dt=1000.0)
    for _ in range(3):
        before = [b.surface(r).cpu().numpy().astype(np.float64) for r in range(b.R)]
        b.step(1)
        b.sync()
        for r in range(b.R):
            want, _ = oracle.step(before[r], oracle.params(K=Ks[r], m=ms[r]))
            got = b.surface(r).cpu().numpy().astype(np.float64)
            tol = 4 * 2.0 ** -24 * np.maximum(np.abs(want), 1.0)
            assert np.all(np.abs(got - want) <= tol), f"realization {r}"
    b.close()


def test_autotuner_picks_a_shape_and_keeps_results(tmp_path, monkeypatch):
    from paper_1803_02977_gb300 import autotune, lem
    monkeypatch.setenv("LEM_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    surfaces, Ks, ms = _realizations(R=7, seed=5)
    b = lem.Batch(surfaces, dx=100.0, K=Ks, m=ms, U=1e-3, dt=1000.0)
    h0 = b.h.clone()
    shape, timings = autotune.tune_batch(b, steps=1)
    assert tuple(shape) in lem.BATCH_CONFIGS and len(timings) == len(lem.BATCH_CONFIGS)
    assert torch.equal(b.h, h0)  # tuning restores the elevations
    shape2, _ = autotune.tune_batch(b, steps=1)  # served from the cache
    assert tuple(shape2) == tuple(shape)
    b.close()


def test_step_tilings_agree_and_tuner_lists_them(tmp_path, monkeypatch):
    """Every tiling of the single-grid step (rows per strip of the codes
    pass, whole or half warp tiles) gives the same elevations on a grid whose
    trees fit the warp and block tiers; the tuner times every one."""
    from paper_1803_02977_gb300 import autotune, lem
    monkeypatch.setenv("LEM_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    dev = torch.device("cuda:0")
    for npt in (np.float32, np.float64):
        h0 = synth.noise_surface(517, 389, 9, south_tilt=1e-4).astype(npt)
        ref = None
        rows = (8, 16, 32) if npt == np.float32 else (8, 16)
        for k in rows:
            for hf in (0, 1):
                h = torch.tensor(h0, device=dev)
                m = lem.Model(h)
                lem.lem_set_tiling(m.ctx, k, hf)
                assert lem.lem_get_tiling(m.ctx) == (k, hf)
                m.step(3)
                m.sync()
                assert lem.lem_jump_stats(m.ctx)[0] == 0
                m.close()
                if ref is None:
                    ref = h.cpu()
                assert torch.equal(h.cpu(), ref), (npt, k, hf)
        h = torch.tensor(h0, device=dev)
        m = lem.Model(h)
        if npt == np.float64:
            with pytest.raises(lem.LemError):
                lem.lem_set_tiling(m.ctx, 32, 0)  # FP64 strips hold at most 16 rows
        (k, hf), table = autotune.tune_step(m, steps=1)
        assert sorted(table) == sorted(f"{r}x{f}" for r in rows for f in (0, 1))
        assert table[f"{k}x{hf}"] == min(table.values())
        assert lem.lem_get_tiling(m.ctx) == (k, hf)
        assert torch.equal(h, torch.tensor(h0, device=dev))  # tuning left h as it was
        m.close()
