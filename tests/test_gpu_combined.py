"""Features together, CUDA library vs the FP64 oracle: the corotated and
Neo-Hookean materials with the semi-implicit friction of appendix A (a
block resting on an incline, mu_f = 0.6 > tan theta), one step in FP64
(positions within 1e-6 x the bounding-box diagonal, the same contact count
and outer iterations) and mixed precision (1e-4); and a residual-terminated
step with friction and NH (the same outer iterations, residual log within
1e-5 relative, positions within 1e-6); and the CCD-reuse option with
friction and NH (one FP64 step)."""
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


def resting(model):
    s = scenes.slope_cube(0.6, n_steps=30)
    s.params.model = model
    o = O.Oracle(s)
    st, _ = o.step(20)
    assert st == 0
    x, v = o.get_state()
    keys, lam, gam = o.active_get()
    return s, x, v, keys, lam, gam, o.mu


def make_pair(state, **kw):
    s, x, v, keys, lam, gam, mu = state
    p = scenes.Params(**{**s.params.__dict__, **kw})
    sim = B.Sim(s, p)
    B.bf_set_state(sim.h, x, v)
    B.bf_set_active_set(sim.h, keys, lam, gam)
    B.bf_set_mu(sim.h, mu, p.delta)
    o = O.Oracle(s, p)
    o.set_state(x, v)
    o.active_set(keys, lam, gam)
    o.set_mu_delta(mu, p.delta)
    return sim, o


@pytest.mark.parametrize("model", [1, 2])
@pytest.mark.parametrize("precision", [0, 1])
def test_material_with_friction_one_step(torch_cuda, model, precision):
    state = resting(model)
    s = state[0]
    sim, o = make_pair(state, precision=precision)
    _, so = o.step(1)
    st, sg = sim.step(1)
    assert st == 0
    xo, _ = o.get_state()
    xg, _ = sim.state()
    assert sg[0]["n_contacts"] == so[0]["n_contacts"]
    assert np.abs(xg - xo).max() <= (1e-6 if precision == 0 else 1e-4) * s.bbox_diag()
    if precision == 0:
        assert sg[0]["outer_iters"] == so[0]["outer_iters"]
    sim.close()


def test_residual_mode_with_friction_and_nh(torch_cuda):
    state = resting(2)
    s = state[0]
    sim, o = make_pair(state, res_tol=1e-5)
    st_o, so = o.step(1)
    st_g, sg = sim.step(1)
    assert st_o == 0 and st_g == 0
    log_o, log_g = o.residual_log(), B.bf_get_residual_log(sim.h)
    assert sg[0]["outer_iters"] == so[0]["outer_iters"] and len(log_g) == len(log_o)
    assert np.abs(log_g - log_o).max() <= 1e-5 * log_o.max()
    xo, _ = o.get_state()
    xg, _ = sim.state()
    assert np.abs(xg - xo).max() <= 1e-6 * s.bbox_diag()
    sim.close()


def test_ccd_reuse_with_friction_and_nh(torch_cuda):
    """the CCD-reuse option with NH and friction: one FP64 step from the
    resting state equals the oracle's (outer iterations, contact count,
    positions within 1e-6 x the diagonal)"""
    state = resting(2)
    s = state[0]
    sim, o = make_pair(state, ccd_reuse=1)
    _, so = o.step(1)
    st, sg = sim.step(1)
    assert st == 0
    assert sg[0]["outer_iters"] == so[0]["outer_iters"] and sg[0]["n_contacts"] == so[0]["n_contacts"]
    xo, _ = o.get_state()
    xg, _ = sim.state()
    assert np.abs(xg - xo).max() <= 1e-6 * s.bbox_diag()
    sim.close()
