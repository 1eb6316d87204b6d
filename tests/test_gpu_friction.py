"""CUDA library vs the FP64 oracle with the semi-implicit friction of
appendix A, teacher-forced from an oracle state of a block resting on an
incline: the friction pairs (vertices, weights, normals, coefficients),
the Newton system with friction (gradient, energy, Hessian products), one
time step, and the closed-form sliding acceleration and sticking run on
the GPU alone.  Tolerances as in the frictionless parity tests: 1e-9
relative for FP64 stage results, positions after a step within 1e-6 x
the bounding-box diagonal (1e-4 in mixed precision)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2512_12151_b300 import binding as B
from paper_2512_12151_b300 import scenes

pytestmark = pytest.mark.gpu
TH = math.atan(0.5)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def dev(torch, a):
    return torch.tensor(np.ascontiguousarray(a, np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def resting_state():
    """the oracle's block on the incline (mu_f = 0.6 > tan theta) after 20 steps"""
    s = scenes.slope_cube(0.6, n_steps=30)
    o = O.Oracle(s)
    st, _ = o.step(20)
    assert st == 0
    x, v = o.get_state()
    keys, lam, gam = o.active_get()
    return s, x, v, keys, lam, gam, o.mu


def make_pair(state, precision=0):
    s, x, v, keys, lam, gam, mu = state
    p = scenes.Params(**{**s.params.__dict__, "precision": precision})
    sim = B.Sim(s, p)
    B.bf_set_state(sim.h, x, v)
    B.bf_set_active_set(sim.h, keys, lam, gam)
    B.bf_set_mu(sim.h, mu, p.delta)
    o = O.Oracle(s, p)
    o.set_state(x, v)
    o.active_set(keys, lam, gam)
    o.set_mu_delta(mu, p.delta)
    return sim, o


def by_vertices(v4, *arrays):
    order = np.lexsort(v4.T[::-1])
    return (v4[order],) + tuple(a[order] for a in arrays)


def test_friction_pairs_match(torch_cuda, resting_state):
    sim, o = make_pair(resting_state)
    ng, no = B.bf_friction_setup(sim.h), o.friction_setup()
    assert ng == no > 4
    vg, wg, ng3, kg = by_vertices(*B.bf_friction_get(sim.h))
    vo, wo, no3, ko = by_vertices(*o.friction_get())
    assert (vg == vo).all()
    assert np.abs(wg - wo).max() <= 1e-12 and np.abs(ng3 - no3).max() <= 1e-12
    assert np.abs(kg - ko).max() <= 1e-9 * np.abs(ko).max()
    sim.close()


@pytest.mark.parametrize("slip", [0.3, 30.0])  # in units of h eps_v: inside and beyond the smoothing
def test_newton_system_with_friction(torch_cuda, resting_state, slip):
    torch = torch_cuda
    s = resting_state[0]
    sim, o = make_pair(resting_state)
    B.bf_friction_setup(sim.h)
    o.friction_setup()
    x, _ = o.get_state()
    rng = np.random.default_rng(3)
    free = (s.dirichlet == 0)[:, None]
    eh = s.params.dt * s.params.eps_v
    xh = x + slip * eh * rng.standard_normal(x.shape) * free
    xt = o.xtilde()
    o.linearize(x)
    B.bf_linearize(sim.h, dev(torch, x))
    _, g_o = o.assemble(xt, x, xh)
    g_g = torch.zeros((s.nv, 3), dtype=torch.float64, device="cuda")
    B.bf_assemble(sim.h, dev(torch, xt), dev(torch, x), dev(torch, xh), g_g)
    g_g = host(g_g)
    assert np.abs(g_g - g_o).max() <= 1e-9 * np.abs(g_o).max()
    L_o = o.energy_L(xt, x, xh, o.slacks())
    L_g = B.bf_energy(sim.h, dev(torch, xt), dev(torch, x), dev(torch, xh))
    assert L_g == pytest.approx(L_o, rel=1e-10)
    vec = rng.standard_normal(x.shape)
    y_o = o.hess_apply(vec)
    y_g = torch.zeros((s.nv, 3), dtype=torch.float64, device="cuda")
    B.bf_hess_apply(sim.h, dev(torch, vec), y_g)
    y_g = host(y_g)
    sel = s.dirichlet == 0  # prescribed rows differ only in their (irrelevant) diagonal scale
    assert np.abs(y_g[sel] - y_o[sel]).max() <= 1e-9 * np.abs(y_o[sel]).max()
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_one_step_with_friction(torch_cuda, resting_state, precision):
    s = resting_state[0]
    sim, o = make_pair(resting_state, precision)
    st_o = o.step(1)[1][0]
    _, st_g = sim.step(1)
    xo, _ = o.get_state()
    xg, _ = sim.state()
    assert st_g[0]["n_contacts"] == st_o["n_contacts"]
    tol = (1e-6 if precision == 0 else 1e-4) * s.bbox_diag()
    assert np.abs(xg - xo).max() <= tol
    sim.close()


def test_sliding_and_sticking_on_the_gpu(torch_cuda):
    """the closed forms of the oracle's pins, on the library alone (mixed
    precision): sliding at g (sin theta - mu_f cos theta) within 5 % at
    h = 2.5 ms, sticking (creep below eps_v) when mu_f > tan theta"""
    mu, h = 0.2, 0.0025
    s = scenes.slope_cube(mu, n_steps=240, precision=1)
    s.params.dt = h
    sim = B.Sim(s)
    free = s.dirichlet == 0
    vx = []
    for _ in range(240):
        sim.step(1)
        vx.append(sim.state()[1][free, 0].mean())
    a = (vx[239] - vx[79]) / (160 * h)
    assert a == pytest.approx(-9.8 * (math.sin(TH) - mu * math.cos(TH)), rel=0.05)
    sim.close()
    s = scenes.slope_cube(0.6, n_steps=30, precision=1)
    sim = B.Sim(s)
    sim.step(30)
    assert np.abs(sim.state()[1][s.dirichlet == 0, 0]).max() <= s.params.eps_v
    sim.close()
