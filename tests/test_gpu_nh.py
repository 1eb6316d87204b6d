"""CUDA library vs the FP64 oracle with the Neo-Hookean material (NH):
teacher-forced from an oracle contact state of the two-cube scene, mu_init,
the gradient, Hessian products and energy of the Newton system (FP64 to
1e-9 relative); the inversion bound of MaxStepSize on random, compressing
and inverting motions (to 1e-9); MaxStepSize as min(CCD, inversion bound);
+inf energy at an inverted state; one time step (positions within 1e-6 x
the bounding-box diagonal in FP64, 1e-4 in mixed precision); the implosion
scene whose steps the inversion bound cuts; and, at the eight-cube size, the
property that no element inverts over several steps."""
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


def jacobians(s, x):
    x = np.asarray(x).reshape(-1, 3)
    Ds = np.stack([x[s.tets[:, k]] - x[s.tets[:, 0]] for k in (1, 2, 3)], axis=2)
    Dm = np.stack([s.rest[s.tets[:, k]] - s.rest[s.tets[:, 0]] for k in (1, 2, 3)], axis=2)
    return np.linalg.det(Ds) / np.linalg.det(Dm)


@pytest.fixture(scope="module")
def nh_state():
    s = scenes.two_cubes(0)
    s.params.model = 2
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


def test_newton_system_with_nh(torch_cuda, nh_state):
    torch = torch_cuda
    s, x = nh_state[0], nh_state[1]
    sim, o = make_pair(nh_state)
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
        assert jacobians(s, xh).min() > 0
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


def test_inverted_state_has_infinite_energy(torch_cuda, nh_state):
    """the GPU energy reports a non-finite value where the oracle's is +inf"""
    torch = torch_cuda
    s, x = nh_state[0], nh_state[1]
    sim, o = make_pair(nh_state)
    xt = o.xtilde()
    o.mu_init(x, xt)
    B.bf_mu_init(sim.h, dev(torch, xt), dev(torch, x))
    o.linearize(x)
    B.bf_linearize(sim.h, dev(torch, x))
    xh = x.copy()
    v = int(s.tets[0, 0])
    other = s.tets[0, 1:]
    c = x[other].mean(axis=0)
    n = np.cross(x[other[1]] - x[other[0]], x[other[2]] - x[other[0]])
    n /= np.linalg.norm(n)
    xh[v] = c - 1.5 * np.dot(x[v] - c, n) * n + (x[v] - c - np.dot(x[v] - c, n) * n)  # v reflected through its face
    assert jacobians(s, xh)[0] < 0
    o.assemble(xt, x, x)
    sl = o.slacks()
    assert np.isfinite(o.energy_L(xt, x, x, sl)) and o.energy_L(xt, x, xh, sl) == np.inf
    with pytest.raises(Exception):
        B.bf_energy(sim.h, dev(torch, xt), dev(torch, x), dev(torch, xh))
    sim.close()


def test_inversion_bound_parity(torch_cuda, nh_state):
    torch = torch_cuda
    s, x = nh_state[0], nh_state[1]
    sim, o = make_pair(nh_state)
    rng = np.random.default_rng(8)
    free = (s.dirichlet == 0)[:, None]
    cases = []
    for amp in (1e-3, 1e-2, 3e-2):
        cases.append(x + amp * rng.standard_normal(x.shape) * free)
    for half in (s.tets[: s.nt // 2], s.tets[s.nt // 2:]):  # one cube reflected through its centre, scaled
        sel = np.zeros(s.nv, bool)
        sel[np.unique(half)] = True
        c = x[sel].mean(axis=0)
        x1 = x.copy()
        x1[sel] = c - 0.8 * (x[sel] - c)
        cases.append(x1)
    bounded = 0
    for x1 in cases:
        a_o = o.inversion_step(x, x1)
        a_g = B.bf_inversion_step(sim.h, dev(torch, x), dev(torch, x1))
        assert a_g == pytest.approx(a_o, abs=1e-9)
        bounded += a_o < 1.0
        # MaxStepSize combines the CCD and inversion bounds on both sides
        m_o = o.max_step_size(x, x1)
        m_g = B.bf_max_step_size(sim.h, dev(torch, x), dev(torch, x1))
        assert m_g == pytest.approx(m_o, abs=1e-9) and m_o <= a_o
    assert bounded >= 3
    # an already inverted start allows no step
    xi = x.copy()
    xi[s.tets[0, 0]] = 2 * x[s.tets[0, 1:]].mean(axis=0) - x[s.tets[0, 0]]
    assert jacobians(s, xi)[0] < 0
    assert B.bf_inversion_step(sim.h, dev(torch, xi), dev(torch, x)) == 0.0 == o.inversion_step(xi, x)
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_one_step_with_nh(torch_cuda, nh_state, precision):
    s = nh_state[0]
    sim, o = make_pair(nh_state, precision)
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


def implosion():
    s = scenes.single_cube(seed=0, cells=3, z=0.5, with_ground=False, gravity=(0, 0, 0))
    s.mats[:, 0] = 1e3
    s.params.model = 2
    c = s.x0.mean(axis=0)
    s.v0[:] = -300.0 * (s.x0 - c)
    return s


def test_implosion_matches_the_oracle(torch_cuda):
    """steps cut by the inversion bound: the same outer iterations and
    positions as the oracle, and no inverted element"""
    s = implosion()
    o = O.Oracle(s)
    sim = B.Sim(s)
    for k in range(3):
        st_o, so = o.step(1)
        st_g, sg = sim.step(1)
        assert st_o == 0 and st_g == 0
        xo, _ = o.get_state()
        xg, _ = sim.state()
        assert np.abs(xg - xo).max() <= 1e-6 * s.bbox_diag()
        assert sg[0]["outer_iters"] == so[0]["outer_iters"]
        assert sg[0]["min_alpha"] == pytest.approx(so[0]["min_alpha"], rel=1e-6, abs=1e-12)
        assert jacobians(s, xg).min() > 0
    sim.close()


def test_eight_cubes_nh_never_inverts(torch_cuda):
    """the eight-cube scene (8 x 16^3 cells) with NH in mixed precision:
    every step succeeds and leaves every element with J > 0"""
    s = scenes.eight_cubes(0, precision=1)
    s.params.model = 2
    sim = B.Sim(s)
    for _ in range(6):
        st, stats = sim.step(1)
        assert st == 0
        x, _ = sim.state()
        assert jacobians(s, x).min() > 0
    sim.close()
