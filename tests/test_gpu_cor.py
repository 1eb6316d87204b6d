"""CUDA library vs the FP64 oracle with the corotated material (COR):
teacher-forced from an oracle contact state of the two-cube scene, mu_init,
the gradient, Hessian products and energy of the Newton system (FP64 to
1e-9 relative), and one time step (positions within 1e-6 x the
bounding-box diagonal in FP64, 1e-4 in mixed precision; same active set in
FP64)."""
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


def host(t):
    return t.detach().cpu().numpy()


def keyset(keys):
    return {tuple(int(v) for v in k) for k in keys}


@pytest.fixture(scope="module")
def cor_state():
    s = scenes.two_cubes(0)
    s.params.model = 1
    o = O.Oracle(s)
    st, _ = o.step(5)
    assert st == 0
    x, v = o.get_state()
    keys, lam, gam = o.active_get()
    assert len(keys) > 50
    return s, x, v, keys, lam, gam


def make_pair(state, precision=0):
    s, x, v, keys, lam, gam = state
    p = scenes.Params(**{**s.params.__dict__, "precision": precision})
    sim = B.Sim(s, p)
    B.bf_set_state(sim.h, x, v)
    B.bf_set_active_set(sim.h, keys, lam, gam)
    o = O.Oracle(s, p)
    o.set_state(x, v)
    o.active_set(keys, lam, gam)
    return sim, o


def test_newton_system_with_cor(torch_cuda, cor_state):
    torch = torch_cuda
    s, x = cor_state[0], cor_state[1]
    sim, o = make_pair(cor_state)
    xt = o.xtilde()
    mu_o = o.mu_init(x, xt)
    mu_g = B.bf_mu_init(sim.h, dev(torch, xt), dev(torch, x))
    assert mu_g == pytest.approx(mu_o, rel=1e-10)
    o.linearize(x)
    B.bf_linearize(sim.h, dev(torch, x))
    rng = np.random.default_rng(2)
    free = (s.dirichlet == 0)[:, None]
    for amp in (2e-4, 3e-3):  # small and large deformation increments
        xh = x + (0.5 * (xt - x) + amp * rng.standard_normal(x.shape)) * free
        _, G_o = o.assemble(xt, x, xh)
        G_g = torch.zeros((s.nv, 3), dtype=torch.float64, device="cuda")
        B.bf_assemble(sim.h, dev(torch, xt), dev(torch, x), dev(torch, xh), G_g)
        assert np.abs(host(G_g) - G_o).max() <= 1e-9 * np.abs(G_o).max()
        w = rng.standard_normal((s.nv, 3))
        y_o = o.hess_apply(w)
        y_g = torch.zeros_like(G_g)
        B.bf_hess_apply(sim.h, dev(torch, w), y_g)
        sel = s.dirichlet == 0
        assert np.abs(host(y_g)[sel] - y_o[sel]).max() <= 1e-9 * np.abs(y_o[sel]).max()
        L_o = o.energy_L(xt, x, xh, o.slacks())
        L_g = B.bf_energy(sim.h, dev(torch, xt), dev(torch, x), dev(torch, xh))
        assert L_g == pytest.approx(L_o, rel=1e-11, abs=1e-15)
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_one_step_with_cor(torch_cuda, cor_state, precision):
    s = cor_state[0]
    sim, o = make_pair(cor_state, precision)
    st_o = o.step(1)[1][0]
    _, st_g = sim.step(1)
    xo, _ = o.get_state()
    xg, _ = sim.state()
    tol = (1e-6 if precision == 0 else 1e-4) * s.bbox_diag()
    assert np.abs(xg - xo).max() <= tol
    if precision == 0:
        assert st_g[0]["outer_iters"] == st_o["outer_iters"]
        assert keyset(o.active_get()[0]) == keyset(B.bf_get_active_set(sim.h)[0])
    sim.close()
