"""CUDA library vs the FP64 oracle for the gradient-norm residual of
section 6 ((1/h) |H^-1 grad L|_inf) and the residual-terminated time step:
the residual at a contact state of two colliding balls (PCG to 1e-10, to
1e-7 relative), in closed form for free fall, and one residual-terminated
step (FP64: the same outer iterations, residual log within 1e-5 relative,
positions within 1e-6 x the bounding-box diagonal; mixed precision: the
log ends below the tolerance and positions agree within 1e-4)."""
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


def dev(torch, a):
    return torch.tensor(np.ascontiguousarray(a, np.float64), device="cuda")


@pytest.fixture(scope="module")
def balls_state():
    s = scenes.colliding_balls(0)
    o = O.Oracle(s)
    st, _ = o.step(5)
    assert st == 0
    x, v = o.get_state()
    keys, lam, gam = o.active_get()
    return s, x, v, keys, lam, gam


def make_pair(state, **kw):
    s, x, v, keys, lam, gam = state
    p = scenes.Params(**{**s.params.__dict__, **kw})
    sim = B.Sim(s, p)
    B.bf_set_state(sim.h, x, v)
    B.bf_set_active_set(sim.h, keys, lam, gam)
    o = O.Oracle(s, p)
    o.set_state(x, v)
    o.active_set(keys, lam, gam)
    return sim, o


def test_residual_parity(torch_cuda, balls_state):
    torch = torch_cuda
    x = balls_state[1]
    sim, o = make_pair(balls_state, cg_tol=1e-10)
    xt = o.xtilde()
    o.mu_init(x, xt)
    B.bf_mu_init(sim.h, dev(torch, xt), dev(torch, x))
    r_o = o.newton_residual(xt, x)
    r_g = B.bf_newton_residual(sim.h, dev(torch, xt), dev(torch, x))
    assert r_g == pytest.approx(r_o, rel=1e-7)
    sim.close()


def test_free_fall_residual_on_the_gpu(torch_cuda):
    torch = torch_cuda
    s = scenes.single_cube(seed=0, cells=2, z=0.5, with_ground=False)
    s.params.cg_tol = 1e-12
    s.v0[:] = np.array([0.3, -0.2, 0.5])
    sim = B.Sim(s)
    x = dev(torch, s.x0)
    xt = torch.zeros_like(x)
    B.bf_xtilde(sim.h, xt)
    B.bf_mu_init(sim.h, xt, x)
    h, g = s.params.dt, np.array(s.params.gravity)
    assert B.bf_newton_residual(sim.h, xt, x) == pytest.approx(np.abs(s.v0[0] + h * g).max(), rel=1e-9)
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_residual_terminated_step(torch_cuda, balls_state, precision):
    s = balls_state[0]
    tol = 1e-5
    sim, o = make_pair(balls_state, res_tol=tol, precision=precision)
    st_o, so = o.step(1)
    st_g, sg = sim.step(1)
    assert st_o == 0 and st_g == 0
    log_o, log_g = o.residual_log(), B.bf_get_residual_log(sim.h)
    assert log_g[-1] < tol and np.all(log_g[:-1] >= tol)
    xo, _ = o.get_state()
    xg, _ = sim.state()
    if precision == 0:
        assert sg[0]["outer_iters"] == so[0]["outer_iters"]
        assert np.abs(log_g - log_o).max() <= 1e-5 * log_o.max()
        assert np.abs(xg - xo).max() <= 1e-6 * s.bbox_diag()
    else:
        assert np.abs(xg - xo).max() <= 1e-4 * s.bbox_diag()
    sim.close()
