"""The spiky-ball compression scene at full size (5 balls, about 2.3M tets,
432k vertices; mixed precision, as the large bench line runs it) against
the oracle on sampled outputs: the FP64 gradient and the FP32 Hessian
action at 300 random free vertices, each computed one by one from the
oracle's element function (incident tets), the lumped mass and the
inertia term; the CCD hit set and TOIs of a full-size motion (bit-exact);
and two time steps of the moving plate that complete, with and without the
CCD-reuse option."""
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


@pytest.fixture(scope="module")
def spiky():
    return scenes.spiky_balls(0, precision=1)


def dev(torch, a):
    return torch.tensor(np.ascontiguousarray(a, np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def incident(s, verts):
    """{v: [(tet, local index)]} for the sampled vertices"""
    want = set(int(v) for v in verts)
    out = {v: [] for v in want}
    hit = np.isin(s.tets, list(want))
    for e, k in zip(*np.nonzero(hit)):
        out[int(s.tets[e, k])].append((int(e), int(k)))
    return out


def test_large_assembly_sampled(torch_cuda, spiky):
    torch = torch_cuda
    s = spiky
    assert len(s.tets) > 2_000_000
    o = O.Oracle(s, scenes.Params(**{**s.params.__dict__, "precision": 0}))
    mass = o.mass()
    sim = B.Sim(s)
    x = s.x0
    free = s.dirichlet == 0
    rng = np.random.default_rng(3)
    xt_g = torch.zeros((s.nv, 3), dtype=torch.float64, device="cuda")
    B.bf_xtilde(sim.h, xt_g)
    xt = host(xt_g)
    h, g = s.params.dt, np.array(s.params.gravity)
    assert np.abs(xt[free] - (x[free] + h * s.v0[free] + h * h * g)).max() <= 1e-15
    xh = x + 3e-4 * rng.standard_normal(x.shape) * free[:, None]
    B.bf_set_mu(sim.h, 1.0, s.params.delta)
    B.bf_linearize(sim.h, dev(torch, x))  # no pair is active at the start
    G_g = torch.zeros_like(xt_g)
    B.bf_assemble(sim.h, xt_g, dev(torch, x), dev(torch, xh), G_g)
    G_g = host(G_g)
    w = rng.standard_normal((s.nv, 3))
    y_g = torch.zeros_like(xt_g)
    B.bf_hess_apply(sim.h, dev(torch, w), y_g)
    y_g = host(y_g)
    sample = rng.choice(np.nonzero(free)[0], 300, replace=False)
    inc = incident(s, sample)
    mats = s.mats[s.tet_mat]
    gmax, ymax, gerr, yerr = 0.0, 0.0, 0.0, 0.0
    for v in sample:
        G = mass[v] * (xh[v] - xt[v])
        y = mass[v] * w[v]
        for e, k in inc[int(v)]:
            t = s.tets[e]
            Dm = (s.rest[t[1:]] - s.rest[t[0]]).T
            mu_e, lam_e = O.lame(mats[e, 0], mats[e, 1])
            _, ge, He = O.elem_grad_hess(xh[t].reshape(-1), np.linalg.inv(Dm).reshape(-1), np.linalg.det(Dm) / 6,
                                         mu_e, lam_e, project=True)
            G = G + h * h * ge[3 * k:3 * k + 3]
            for j in range(4):
                if free[t[j]]:
                    y = y + h * h * He[3 * k:3 * k + 3, 3 * j:3 * j + 3] @ w[t[j]]
        gmax, ymax = max(gmax, np.abs(G).max()), max(ymax, np.abs(y).max())
        gerr, yerr = max(gerr, np.abs(G_g[v] - G).max()), max(yerr, np.abs(y_g[v] - y).max())
    assert gerr <= 1e-9 * gmax
    assert yerr <= 1e-5 * ymax
    sim.close()


def test_large_ccd_full_size(torch_cuda, spiky):
    """a full-size motion (the plate to its next target, the balls falling
    1 cm with noise): hit sets equal and TOIs bit-exact"""
    torch = torch_cuda
    s = spiky
    o = O.Oracle(s, scenes.Params(**{**s.params.__dict__, "precision": 0}))
    sim = B.Sim(s)
    rng = np.random.default_rng(4)
    x = s.x0
    free = s.dirichlet == 0
    x1 = x.copy()
    x1[~free] = scenes.plate_targets_schedule(s, 0)
    x1[free] = x[free] + np.array([0.0, 0.0, -0.01]) + 1e-3 * rng.standard_normal((int(free.sum()), 3))
    k_o, t_o = o.ccd_hits(x, x1)
    k_g, t_g = B.bf_ccd_hits(sim.h, dev(torch, x), dev(torch, x1))
    assert len(k_o) > 1000
    A = {tuple(k): t for k, t in zip(k_o.tolist(), t_o)}
    Bm = {tuple(k): t for k, t in zip(k_g.tolist(), t_g)}
    assert A.keys() == Bm.keys()
    assert all(Bm[k] == A[k] for k in A)
    sim.close()


@pytest.mark.parametrize("reuse", [0, 1])
def test_large_steps_complete(torch_cuda, spiky, reuse):
    """two steps of the moving plate, with and without the CCD-reuse option"""
    s = spiky
    sim = B.Sim(s, scenes.Params(**{**s.params.__dict__, "ccd_reuse": reuse}))
    for i in range(2):
        B.bf_set_obstacle_targets(sim.h, scenes.plate_targets_schedule(s, i))
        st, stats = sim.step(1)
        assert st == 0
        x, v = sim.state()
        assert np.isfinite(x).all() and np.isfinite(v).all()
    sim.close()


def test_large_subproblem_teacher_forced(torch_cuda):
    """One outer iteration of the compression, teacher-forced from the same
    state on both sides, on the spiky-ball scene meshed at twice the cell
    size (287,448 tets, 1/8 of the full scene's; the same generator): the
    plate's targets 6 cm lower, into the top ball's spikes; UpdateActiveSet
    along x^t -> xhat^[0] gives the same pairs; the AL subproblem (Alg. 2,
    mixed precision on the GPU, FP64 in the oracle) lands within 1e-4 x the
    bounding-box diagonal with the same multiplier signs and decay factors;
    MaxStepSize from the oracle's xhat^[1] is bit-identical."""
    torch = torch_cuda
    s = scenes.spiky_balls(0, cell=0.0078, precision=1)
    assert 250_000 < s.nt < 330_000
    o = O.Oracle(s, scenes.Params(**{**s.params.__dict__, "precision": 0}))
    sim = B.Sim(s)
    x = s.x0
    xh = x.copy()
    xh[s.meta["plate_vertices"], 2] -= 0.06
    xt = o.xtilde()
    mu = o.mu_init(xh, xt)
    B.bf_set_mu(sim.h, mu, s.params.delta)
    o.update_active_set(x, xh)
    B.bf_update_active_set(sim.h, dev(torch, x), dev(torch, xh))
    ko, lo, go = o.active_get()
    kg, lg, gg = B.bf_get_active_set(sim.h)
    Ao = {tuple(k): (l, g) for k, l, g in zip(ko.tolist(), lo, go)}
    Ag = {tuple(k): (l, g) for k, l, g in zip(kg.tolist(), lg, gg)}
    assert len(Ao) > 20 and Ao == Ag  # same pairs (lambda = 0, gamma = 1 for new pairs)
    xh_o, nn_o, cg_o, lsf_o = o.solve_subproblem(xt, x, xh)
    xh_g = dev(torch, xh)
    nn_g, cg_g = B.bf_solve_subproblem(sim.h, dev(torch, xt), dev(torch, x), xh_g)
    err = np.abs(host(xh_g) - xh_o).max() / s.bbox_diag()
    print(f"subproblem: Newton {nn_g} (oracle {nn_o}), CG {cg_g} ({cg_o}), max error / diagonal {err:.2e}")
    assert err <= 1e-4
    ko, lo, go = o.active_get()
    kg, lg, gg = B.bf_get_active_set(sim.h)
    Ao = {tuple(k): (l, g) for k, l, g in zip(ko.tolist(), lo, go)}
    Ag = {tuple(k): (l, g) for k, l, g in zip(kg.tolist(), lg, gg)}
    assert Ao.keys() == Ag.keys() and all(Ao[k][1] == Ag[k][1] for k in Ao)
    lmax = max(1e-12, max(abs(v[0]) for v in Ao.values()))
    assert all(abs(Ao[k][0] - Ag[k][0]) <= 1e-3 * lmax for k in Ao)
    assert B.bf_max_step_size(sim.h, dev(torch, x), dev(torch, xh_o)) == o.max_step_size(x, xh_o)
    sim.close()


def test_large_pcg_symmetric_matches_full_rows(torch_cuda, spiky):
    """At full size the default PCG is the symmetric variant (upper blocks
    streamed once, transposed products by vector reductions); on the
    assembled Newton system of the compression it reaches the tolerance on
    the library's own operator and agrees with the variant that streams
    both triangles (bf_set_pcg_mode 97) and with the per-phase launches."""
    torch = torch_cuda
    s = spiky
    sim = B.Sim(s)
    x = s.x0
    xd = dev(torch, x)
    xt = torch.zeros_like(xd)
    B.bf_xtilde(sim.h, xt)
    B.bf_mu_init(sim.h, xt, xd)
    B.bf_linearize(sim.h, xd)
    G = torch.zeros_like(xd)
    B.bf_assemble(sim.h, xt, xd, xd, G)
    b = -G
    sols, its = [], []
    for mode in (1, 97, 0):
        B.bf_set_pcg_mode(sim.h, mode)
        p = torch.zeros_like(xd)
        it, _ = B.bf_pcg(sim.h, b, p, 1e-6, 100000)
        if mode == 1:
            assert B.bf_get_pcg_config(sim.h)["resident"] == 3  # the symmetric variant
        Hp = torch.zeros_like(xd)
        B.bf_hess_apply(sim.h, p, Hp)
        res = float(torch.linalg.norm(Hp - b) / torch.linalg.norm(b))
        assert res <= 1e-4, (mode, res)
        sols.append(host(p).reshape(-1))
        its.append(it)
    assert abs(its[0] - its[1]) <= max(2, its[1] // 20), its
    for k in (0, 1):
        assert np.linalg.norm(sols[k] - sols[2]) <= 1e-4 * np.linalg.norm(sols[2])
    sim.close()
