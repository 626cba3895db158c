"""Checkpoint / resume (lem_get_state, lem_set_state): the steps after a
resume equal, bit for bit, those the saved context would have taken --
including a deep surface whose device tier carries its pointer-jumping hint
across steps -- with the state in host or in device memory."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1803_02977_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _resume_equals_continue(h0, steps_before, steps_after, device_buf=False):
    from paper_1803_02977_gb300 import lem
    dev = torch.device("cuda:0")
    par = dict(dx=100.0, K=2e-5, m=0.5, U=1e-3, dt=1000.0)
    h = torch.tensor(h0, device=dev)
    mdl = lem.Model(h, **par)
    mdl.step(steps_before)
    if device_buf:
        n = lem.lem_state_size(mdl.ctx)
        buf = torch.empty(n, dtype=torch.uint8, device=dev)
        rc = lem.lib().lem_get_state(mdl.ctx, ctypes.c_void_p(buf.data_ptr()), n)
        assert rc == lem.LEM_OK
    else:
        buf = lem.lem_get_state(mdl.ctx)
    mdl.step(steps_after)
    mdl.sync()
    cont = h.clone()
    jumps = lem.lem_jump_stats(mdl.ctx)[0]
    h.zero_()  # the resume must restore every elevation
    if device_buf:
        rc = lem.lib().lem_set_state(mdl.ctx, ctypes.c_void_p(buf.data_ptr()), buf.numel())
        assert rc == lem.LEM_OK
    else:
        lem.lem_set_state(mdl.ctx, buf)
    mdl.step(steps_after)
    mdl.sync()
    assert torch.equal(h, cont)
    priv, wide = lem.lem_step_stats(mdl.ctx)
    assert priv + wide == steps_before + steps_after
    mdl.close()
    return jumps


def test_resume_equals_continue_noise():
    _resume_equals_continue(synth.noise_surface(300, 200, 3), 3, 3)


def test_resume_equals_continue_device_buffer_f32():
    _resume_equals_continue(synth.noise_surface(257, 130, 4).astype(np.float32), 2, 2,
                            device_buf=True)


def test_resume_equals_continue_deep_surface():
    h0 = oracle.fill(synth.noise_surface(400, 300, 12))
    assert _resume_equals_continue(h0, 2, 3) >= 1  # the deep tier ran after the resume too


def test_state_rejects_other_grid_and_short_buffer():
    from paper_1803_02977_gb300 import lem
    dev = torch.device("cuda:0")
    a = lem.Model(torch.tensor(synth.noise_surface(40, 30, 1), device=dev))
    b = lem.Model(torch.tensor(synth.noise_surface(30, 40, 1), device=dev))
    sa = lem.lem_get_state(a.ctx)
    with pytest.raises(lem.LemError) as e:
        lem.lem_set_state(b.ctx, sa)  # same size, other grid
    assert e.value.status == lem.LEM_EINVAL
    with pytest.raises(lem.LemError) as e:
        lem.lem_set_state(a.ctx, sa[:-1])
    assert e.value.status == lem.LEM_EINVAL
    a.close()
    b.close()
