"""CUDA library vs the FP64 oracle with the CCD-reuse option (one CCD along
the MaxStepSize segment serves the active-set update): one step from an
oracle contact state of the two-cube scene (FP64: the same outer
iterations and active set, positions within 1e-6 x the bounding-box
diagonal; mixed: 1e-4), a 20-step FP64 trajectory from rest (the same outer
iterations every step, positions within 1e-6 x the diagonal), and an
impact on the ground (one step, FP64)."""
import numpy as np
import pytest

import oracle as O
from paper_2512_12151_b300 import binding as B
from paper_2512_12151_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def keyset(keys):
    return {tuple(int(v) for v in k) for k in keys}


@pytest.fixture(scope="module")
def reuse_state():
    s = scenes.two_cubes(0)
    s.params.ccd_reuse = 1
    o = O.Oracle(s)
    st, _ = o.step(5)
    assert st == 0
    x, v = o.get_state()
    keys, lam, gam = o.active_get()
    assert len(keys) > 20
    return s, x, v, keys, lam, gam


@pytest.mark.parametrize("precision", [0, 1])
def test_one_step_with_ccd_reuse(torch_cuda, reuse_state, precision):
    s, x, v, keys, lam, gam = reuse_state
    p = scenes.Params(**{**s.params.__dict__, "precision": precision})
    sim = B.Sim(s, p)
    B.bf_set_state(sim.h, x, v)
    B.bf_set_active_set(sim.h, keys, lam, gam)
    o = O.Oracle(s, p)
    o.set_state(x, v)
    o.active_set(keys, lam, gam)
    _, so = o.step(1)
    st, sg = sim.step(1)
    assert st == 0
    xo, _ = o.get_state()
    xg, _ = sim.state()
    assert np.abs(xg - xo).max() <= (1e-6 if precision == 0 else 1e-4) * s.bbox_diag()
    if precision == 0:
        assert sg[0]["outer_iters"] == so[0]["outer_iters"]
        assert keyset(o.active_get()[0]) == keyset(B.bf_get_active_set(sim.h)[0])
    sim.close()


def test_trajectory_with_ccd_reuse(torch_cuda):
    s = scenes.two_cubes(1)
    s.params.ccd_reuse = 1
    o = O.Oracle(s)
    sim = B.Sim(s)
    for _ in range(20):
        st_o, so = o.step(1)
        st_g, sg = sim.step(1)
        assert st_o == 0 and st_g == 0
        assert sg[0]["outer_iters"] == so[0]["outer_iters"]
    xo, _ = o.get_state()
    xg, _ = sim.state()
    assert np.abs(xg - xo).max() <= 1e-6 * s.bbox_diag()
    sim.close()


def test_impact_with_ccd_reuse(torch_cuda):
    s = scenes.single_cube(seed=0, cells=2, z=0.012, with_ground=True, v0=(0.0, 0.0, -2.0))
    s.params.ccd_reuse = 1
    o = O.Oracle(s)
    sim = B.Sim(s)
    _, so = o.step(1)
    st, sg = sim.step(1)
    assert st == 0 and sg[0]["outer_iters"] == so[0]["outer_iters"] and so[0]["n_contacts"] > 0
    xo, _ = o.get_state()
    xg, _ = sim.state()
    assert np.abs(xg - xo).max() <= 1e-6 * s.bbox_diag()
    assert keyset(o.active_get()[0]) == keyset(B.bf_get_active_set(sim.h)[0])
    sim.close()
