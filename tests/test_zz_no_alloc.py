"""The allocation-free step entry point (lem_step_noalloc).

It exists for callers that cannot allocate device memory (a framework whose
caching allocator owns the GPU, or loops where cudaMalloc's blocking and
implicit synchronisation are not allowed); its working memory is a fixed
array inside the library.  Checked through the C ABI against the ordinary
context-based entry point (lem_create + lem_step) on two calls in a row,
which also exercises the reuse of the shared array between calls.

This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1803_02977_gb300 import synth

torch = pytest.importorskip("torch")

REL64 = 1e-12


@pytest.mark.gpu
def test_noalloc_matches_context_step_on_two_calls():
    from paper_1803_02977_gb300 import lem
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    dev = torch.device("cuda:0")
    nx, ny = 257, 199  # ragged: not a multiple of any block or warp size
    par = dict(dx=100.0, K=2e-5, m=0.45, U=1e-3, dt=1000.0)
    h0 = synth.noise_surface(nx, ny, 77, south_tilt=1e-4)

    ref = torch.tensor(h0, device=dev)
    mdl = lem.Model(ref, **par)
    got = torch.tensor(h0, device=dev)
    for call in range(2):
        mdl.step(3)
        mdl.sync()
        rc = lem.lem_step_noalloc(got, par["dx"], par["K"], par["m"], par["U"], par["dt"], 3)
        assert rc == lem.LEM_OK, f"call {call}: status {rc}"
        want = ref.cpu().numpy()
        err = np.abs(got.cpu().numpy() - want).max()
        assert err <= REL64 * max(np.abs(want).max(), 1.0), f"call {call}: max |dh| {err}"
    mdl.close()


@pytest.mark.gpu
def test_noalloc_reuses_its_array_across_sizes_and_parameters():
    """A smaller grid after a larger one and back, with other parameters on
    every call: stale codes, queues and counts beyond the smaller grid and
    the erosion tables of the previous call must not leak into the next."""
    from paper_1803_02977_gb300 import lem
    dev = torch.device("cuda:0")
    calls = [((257, 199), dict(dx=100.0, K=2e-5, m=0.45, U=1e-3, dt=1000.0), 78),
             ((100, 60), dict(dx=50.0, K=4e-5, m=0.5, U=2e-3, dt=500.0), 79),
             ((257, 199), dict(dx=120.0, K=1e-5, m=0.55, U=1e-3, dt=800.0), 80)]
    for (nx, ny), par, seed in calls:
        h0 = synth.noise_surface(nx, ny, seed, south_tilt=1e-4)
        ref = torch.tensor(h0, device=dev)
        mdl = lem.Model(ref, **par)
        mdl.step(2)
        mdl.sync()
        mdl.close()
        got = torch.tensor(h0, device=dev)
        rc = lem.lem_step_noalloc(got, par["dx"], par["K"], par["m"], par["U"], par["dt"], 2)
        assert rc == lem.LEM_OK, f"{nx}x{ny}: status {rc}"
        want = ref.cpu().numpy()
        err = np.abs(got.cpu().numpy() - want).max()
        assert err <= REL64 * max(np.abs(want).max(), 1.0), f"{nx}x{ny}: max |dh| {err}"


@pytest.mark.gpu
def test_noalloc_rejects_oversized_grid_before_device_work():
    from paper_1803_02977_gb300 import lem
    dev = torch.device("cuda:0")
    side = int(lem.LEM_NOALLOC_MAX_CELLS ** 0.5) + 1
    h = torch.zeros((side, side), dtype=torch.float64, device=dev)
    rc = lem.lem_step_noalloc(h, 100.0, 1e-5, 0.5, 1e-3, 1000.0, 1)
    assert rc == lem.LEM_EINVAL
    assert torch.count_nonzero(h).item() == 0
