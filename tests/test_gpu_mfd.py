"""Flow accumulation with multiple flow directions on the GPU
(lem_accumulate_mfd: Eq. 2 with a slope^p split, Kahn's levels) against the
oracle: bit for bit for p = 1, within 1e-12 relative for other exponents
(FP64 powers differ in the last place between libraries); the level count
exactly; FP32 elevations; a source field; the benchmark's full grid."""
import numpy as np
import pytest

import oracle
from paper_1803_02977_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lem():
    from paper_1803_02977_gb300 import lem
    return lem


def _dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda:0")


def _int_grid(nx, ny, seed, levels=6):
    u = synth.uniform01(seed, nx * ny).reshape(ny, nx)
    h = np.floor(u * levels)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


def _cone3():
    h = np.zeros((3, 3))
    h[1, 1] = 1.0
    return h


def _tilted(nx, ny, seed):
    x = np.arange(nx, dtype=np.float64)[None, :]
    h = 5.0 * x + 0.01 * synth.uniform01(seed, nx * ny).reshape(ny, nx)
    h[0, :] = h[-1, :] = h[:, 0] = h[:, -1] = 0.0
    return h


CASES = [
    ("cone_3x3", _cone3),
    ("noise_5x4", lambda: synth.noise_surface(5, 4, 2)),
    ("noise_64x64", lambda: synth.noise_surface(64, 64, 3)),
    ("int_flats_120x90", lambda: _int_grid(120, 90, 4)),
    ("tilted_300x200", lambda: _tilted(300, 200, 5)),
    ("noise_1031x777", lambda: synth.noise_surface(1031, 777, 6)),
]


def _run(h_np, p=1.0, w=None, dtype=torch.float64):
    lem = _lem()
    h = torch.tensor(h_np, dtype=dtype, device=_dev())
    mdl = lem.Model(h)
    wt = None if w is None else torch.tensor(w, device=_dev())
    A, L = mdl.accumulate_mfd(p, wt)
    out = A.cpu().numpy()
    mdl.close()
    return out, L


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_p1_bit_exact(name, make):
    h = make()
    A, L = _run(h, 1.0)
    want, _, Lw = oracle.accumulate_mfd(h, 1.0)
    assert np.array_equal(A, want), f"{name}: {np.count_nonzero(A != want)} cells differ"
    assert L == Lw


@pytest.mark.parametrize("p", [1.1, 2.0, 8.0])
def test_other_exponents_within_tolerance(p):
    h = synth.noise_surface(300, 257, 7)
    A, L = _run(h, p)
    want, _, Lw = oracle.accumulate_mfd(h, p)
    assert np.abs(A - want).max() <= 1e-12 * np.abs(want).max()
    assert L == Lw


def test_source_field_and_fp32_elevations():
    nx, ny = 211, 160
    h = synth.noise_surface(nx, ny, 8).astype(np.float32)
    w = (100.0 * 100.0) * (0.5 + synth.uniform01(9, nx * ny)).reshape(ny, nx)
    A, L = _run(h, 1.0, w, dtype=torch.float32)
    want, _, Lw = oracle.accumulate_mfd(h.astype(np.float64), 1.0, w)
    assert np.array_equal(A, want)
    assert L == Lw


def test_repeatable_and_argument_checks():
    lem = _lem()
    h = torch.tensor(synth.noise_surface(97, 61, 10), device=_dev())
    mdl = lem.Model(h)
    A1, _ = mdl.accumulate_mfd(1.1)
    A2, _ = mdl.accumulate_mfd(1.1)
    assert torch.equal(A1, A2)
    A = torch.empty_like(h)
    for p in (0.0, -1.0, float("nan"), float("inf")):
        assert lem.lib().lem_accumulate_mfd(mdl.ctx, p, None, lem._ptr(A), None) == lem.LEM_EINVAL
    assert lem.lib().lem_accumulate_mfd(mdl.ctx, 1.0, None, None, None) == lem.LEM_EINVAL
    mdl.close()


def test_grid2048_f64_bit_exact():
    w = synth.workload("grid2048_f64")
    h = w.initial()
    A, L = _run(h, 1.0)
    want, _, Lw = oracle.accumulate_mfd(h, 1.0)
    assert np.array_equal(A, want)
    assert L == Lw
