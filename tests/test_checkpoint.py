"""Checkpoint and resume through the C ABI (bf_save / bf_load): a scene
saved mid-run and restored into a fresh scene of the same mesh continues
exactly as the original does (same state, same active set, same obstacle
targets; only the order of floating-point atomics may differ), and buffers
that are not checkpoints of the scene are refused."""
import numpy as np
import pytest

from paper_2512_12151_b300 import binding as B
from paper_2512_12151_b300 import scenes, serving

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.mark.parametrize("precision", [0, 1])
def test_resume_continues_the_run(torch_cuda, precision):
    s = scenes.two_cubes(0, precision=precision)
    a = B.Sim(s)
    a.step(6)
    keys0, _, _ = B.bf_get_active_set(a.h)
    assert len(keys0) > 0  # the checkpoint carries a non-empty active set
    blob = B.bf_save(a.h)
    a.step(3)
    xa, va = a.state()
    ka, la, ga = B.bf_get_active_set(a.h)
    b = B.Sim(s)
    B.bf_load(b.h, blob)
    assert B.bf_save(b.h)[:len(blob)] == blob  # restored exactly
    b.step(3)
    xb, vb = b.state()
    kb, lb, gb = B.bf_get_active_set(b.h)
    a.close()
    b.close()
    tol = (1e-9 if precision == 0 else 1e-5) * s.bbox_diag()
    assert np.abs(xa - xb).max() <= tol
    assert np.abs(va - vb).max() <= tol / s.params.dt
    assert sorted(map(tuple, ka)) == sorted(map(tuple, kb))


def test_resume_restores_obstacle_targets(torch_cuda):
    s = scenes.spiky_balls(0, precision=1, cell=0.012)  # coarse cells keep it small
    a = B.Sim(s)
    B.bf_set_obstacle_targets(a.h, scenes.plate_targets_schedule(s, 0))
    a.step(2)
    blob = B.bf_save(a.h)
    a.step(2)
    xa, _ = a.state()
    b = B.Sim(s)
    B.bf_load(b.h, blob)  # targets come back with the checkpoint
    b.step(2)
    xb, _ = b.state()
    a.close()
    b.close()
    assert np.abs(xa - xb).max() <= 1e-5 * s.bbox_diag()


def test_refused_buffers(torch_cuda):
    s = scenes.two_cubes(0)
    a = B.Sim(s)
    a.step(2)
    blob = B.bf_save(a.h)
    other = B.Sim(scenes.eight_cubes(0, cells=4))
    with pytest.raises(RuntimeError):
        B.bf_load(other.h, blob)  # another mesh: vertex count differs
    with pytest.raises(RuntimeError):
        B.bf_load(a.h, blob[:-8])  # cut short
    bad = bytearray(blob)
    bad[0] ^= 1
    with pytest.raises(RuntimeError):
        B.bf_load(a.h, bytes(bad))  # not a checkpoint
    x0, _ = a.state()
    B.bf_load(a.h, blob)  # the refusals left the scene usable
    assert np.array_equal(a.state()[0], x0)
    a.close()
    other.close()


def test_evict_and_readmit_in_a_batch(torch_cuda):
    s = scenes.batch_scene(7)
    h, keep = serving.create(s)
    B.bf_step(h, 6)
    x_straight, _ = B.bf_get_state(h, s.nv)
    B.bf_scene_destroy(h)
    h, keep = serving.create(s)
    b = B.bf_batch_create(2, 1 << 34)
    try:
        t = B.bf_batch_admit(b, h, 3)
        assert B.bf_batch_wait(b, t, 600000)
        assert B.bf_batch_result(b, t, 3)["status"] == 0
        B.bf_batch_release(b, t)
        blob = serving.evict(h)
        assert B.bf_batch_info(b)["resident_bytes"] == 0
        h, keep = serving.restore(s, blob)
        t = B.bf_batch_admit(b, h, 3)
        assert B.bf_batch_wait(b, t, 600000)
        assert B.bf_batch_result(b, t, 3)["status"] == 0
        B.bf_batch_release(b, t)
    finally:
        B.bf_batch_destroy(b)
    x_resumed, _ = B.bf_get_state(h, s.nv)
    B.bf_scene_destroy(h)
    assert np.abs(x_straight - x_resumed).max() <= 1e-5 * s.bbox_diag()
