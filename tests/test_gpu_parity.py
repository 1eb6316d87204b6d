"""CUDA library vs the FP64 oracle, teacher-forced: both sides start from the
same oracle-produced state (positions, velocities, active set, mu, delta)
and each stage of Alg. 1-3 is compared.

Tolerances: FP64 floating-point results agree to 1e-9 relative (different
summation orders and an analytic instead of a Jacobi eigensystem); TOIs are
bit-exact (both sides evaluate the distances and the additive CCD in the
same FP64 operation order, without FMA contraction); pair sets are equal;
positions after a step agree within 1e-6 x the bounding-box diagonal
(1e-4 in mixed precision)."""
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
def contact_state():
    """two-cube scene (FP64) advanced by the oracle into first contact"""
    s = scenes.two_cubes(0)
    o = O.Oracle(s)
    o.step(5)
    x, v = o.get_state()
    keys, lam, gam = o.active_get()
    assert len(keys) > 50
    return s, x, v, keys, lam, gam


def make_pair(s, x, v, keys, lam, gam, precision=0):
    p = scenes.Params(**{**s.params.__dict__, "precision": precision})
    sim = B.Sim(s, p)
    B.bf_set_state(sim.h, x, v)
    B.bf_set_active_set(sim.h, keys, lam, gam)
    o = O.Oracle(s, p)
    o.set_state(x, v)
    o.active_set(keys, lam, gam)
    return sim, o


def test_xtilde_mu_linearize_assemble(torch_cuda, contact_state):
    torch = torch_cuda
    s, x, v, keys, lam, gam = contact_state
    sim, o = make_pair(s, x, v, keys, lam, gam)
    xt_o = o.xtilde()
    xt_g = torch.zeros((s.nv, 3), dtype=torch.float64, device="cuda")
    B.bf_xtilde(sim.h, xt_g)
    assert np.abs(host(xt_g) - xt_o).max() <= 1e-15
    mu_o = o.mu_init(x, xt_o)
    mu_g = B.bf_mu_init(sim.h, dev(torch, xt_o), dev(torch, x))
    assert mu_g == pytest.approx(mu_o, rel=1e-10)
    # linearisation at x
    d_o, g_o = o.linearize(x)
    d_g = torch.zeros(len(keys), dtype=torch.float64, device="cuda")
    g_g = torch.zeros((len(keys), 12), dtype=torch.float64, device="cuda")
    B.bf_linearize(sim.h, dev(torch, x), d_g, g_g)
    assert np.abs(host(d_g) - d_o).max() <= 1e-12 * max(1.0, np.abs(d_o).max())
    assert np.abs(host(g_g) - g_o).max() <= 1e-9
    # gradient and Hessian action at a perturbed xhat
    rng = np.random.default_rng(1)
    xh = x + (0.5 * (xt_o - x) + 2e-4 * rng.standard_normal(x.shape)) * (s.dirichlet == 0)[:, None]
    E_o, G_o = o.assemble(xt_o, x, xh)
    G_g = torch.zeros((s.nv, 3), dtype=torch.float64, device="cuda")
    E_g = B.bf_assemble(sim.h, dev(torch, xt_o), dev(torch, x), dev(torch, xh), G_g)
    assert np.abs(host(G_g) - G_o).max() <= 1e-9 * np.abs(G_o).max()
    for k in range(3):
        w = rng.standard_normal((s.nv, 3))
        y_o = o.hess_apply(w)
        y_g = torch.zeros_like(G_g)
        B.bf_hess_apply(sim.h, dev(torch, w), y_g)
        free = s.dirichlet == 0
        assert np.abs(host(y_g)[free] - y_o[free]).max() <= 1e-9 * np.abs(y_o[free]).max()
    # AL energy with the slacks of this assembly
    L_o = o.energy_L(xt_o, x, xh, o.slacks())
    L_g = B.bf_energy(sim.h, dev(torch, xt_o), dev(torch, x), dev(torch, xh))
    assert L_g == pytest.approx(L_o, rel=1e-11, abs=1e-15)
    sim.close()


def test_pcg_solution(torch_cuda, contact_state):
    torch = torch_cuda
    s, x, v, keys, lam, gam = contact_state
    sim, o = make_pair(s, x, v, keys, lam, gam)
    xt = o.xtilde()
    o.mu_init(x, xt)
    B.bf_mu_init(sim.h, dev(torch, xt), dev(torch, x))
    o.linearize(x)
    B.bf_linearize(sim.h, dev(torch, x))
    E_o, G_o = o.assemble(xt, x, x)
    G_g = torch.zeros((s.nv, 3), dtype=torch.float64, device="cuda")
    B.bf_assemble(sim.h, dev(torch, xt), dev(torch, x), dev(torch, x), G_g)
    b = -G_o
    H = o.hess_dense()
    ref = np.linalg.solve(H, b.reshape(-1))
    for tol in (1e-6, 1e-10):
        xg = torch.zeros_like(G_g)
        it, _ = B.bf_pcg(sim.h, dev(torch, b), xg, tol, 100000)
        p_o, it_o = o.pcg(b, tol=tol, maxit=100000)
        pg = host(xg).reshape(-1)
        assert np.linalg.norm(H @ pg - b.reshape(-1)) <= tol * np.linalg.norm(b) * 1.01
        assert abs(it - it_o) <= max(2, it_o // 20)
        assert np.linalg.norm(pg - ref) <= tol * np.linalg.cond(H) * np.linalg.norm(ref)
    sim.close()


def test_accd_bit_exact(torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(7)
    for ptype in (0, 1):
        n = 4000
        x0 = rng.standard_normal((n, 12)) * 0.1
        x1 = x0 + rng.standard_normal((n, 12)) * 0.12
        toi = torch.zeros(n, dtype=torch.float64, device="cuda")
        B.bf_accd(ptype, dev(torch, x0), dev(torch, x1), 0.1, toi)
        tg = host(toi)
        to = np.array([O.accd(ptype, x0[i], x1[i]) for i in range(n)])
        assert (np.isinf(tg) == np.isinf(to)).all()
        fin = np.isfinite(to)
        assert fin.sum() > 50
        assert (tg[fin] == to[fin]).all(), np.abs(tg[fin] - to[fin]).max()


def contact_motion(s, x, seed=0, scale=3e-3):
    rng = np.random.default_rng(seed)
    free = (s.dirichlet == 0)[:, None]
    return x + free * (scale * rng.standard_normal(x.shape) + np.array([0, 0, -2.0 * scale]))


@pytest.mark.parametrize("seed", [0, 1])
def test_ccd_hits_and_alpha(torch_cuda, contact_state, seed):
    torch = torch_cuda
    s, x, v, keys, lam, gam = contact_state
    sim, o = make_pair(s, x, v, keys, lam, gam)
    x1 = contact_motion(s, x, seed)
    k_o, t_o = o.ccd_hits(x, x1)
    k_g, t_g = B.bf_ccd_hits(sim.h, dev(torch, x), dev(torch, x1))
    assert len(k_o) > 20
    A = {tuple(k): t for k, t in zip(k_o.tolist(), t_o)}
    Bm = {tuple(k): t for k, t in zip(k_g.tolist(), t_g)}
    assert A.keys() == Bm.keys()
    assert all(Bm[k] == A[k] for k in A)  # bit-exact TOIs
    a_o = o.max_step_size(x, x1)
    a_g = B.bf_max_step_size(sim.h, dev(torch, x), dev(torch, x1))
    assert a_g == a_o
    sim.close()


def test_update_active_set(torch_cuda, contact_state):
    torch = torch_cuda
    s, x, v, keys, lam, gam = contact_state
    # drop some pairs and decay others so that adding and pruning both happen
    sel = np.arange(len(keys)) % 3 != 0
    gam2 = gam.copy()
    gam2[::5] = 0.005
    sim, o = make_pair(s, x, v, keys[sel], lam[sel], gam2[sel])
    x1 = contact_motion(s, x, 3)
    n_o = o.update_active_set(x, x1)
    n_g = B.bf_update_active_set(sim.h, dev(torch, x), dev(torch, x1))
    ko, lo, go = o.active_get()
    kg, lg, gg = B.bf_get_active_set(sim.h)
    assert n_o == n_g == len(ko) == len(kg)
    assert keyset(ko) == keyset(kg)
    Lo = {tuple(k): (l, g) for k, l, g in zip(ko.tolist(), lo, go)}
    Lg = {tuple(k): (l, g) for k, l, g in zip(kg.tolist(), lg, gg)}
    assert all(Lo[k] == Lg[k] for k in Lo)
    sim.close()


def test_solve_subproblem(torch_cuda, contact_state):
    torch = torch_cuda
    s, x, v, keys, lam, gam = contact_state
    sim, o = make_pair(s, x, v, keys, lam, gam)
    xt = o.xtilde()
    mu = o.mu_init(x, xt)
    B.bf_set_mu(sim.h, mu, s.params.delta)
    xh_o, nn_o, cg_o, lsf_o = o.solve_subproblem(xt, x, x)
    xh_g = dev(torch, x)
    nn_g, cg_g = B.bf_solve_subproblem(sim.h, dev(torch, xt), dev(torch, x), xh_g)
    diag = s.bbox_diag()
    assert nn_g == nn_o
    assert np.abs(host(xh_g) - xh_o).max() <= 1e-9 * diag
    ko, lo, go = o.active_get()
    kg, lg, gg = B.bf_get_active_set(sim.h)
    assert (ko == kg).all()
    assert np.abs(lg - lo).max() <= 1e-7 * max(1e-12, np.abs(lo).max())
    assert (gg == go).all()
    sim.close()


@pytest.mark.parametrize("start", [0, 4, 6])
def test_one_step_from_oracle_state(torch_cuda, start):
    s = scenes.two_cubes(0)
    o = O.Oracle(s)
    if start:
        o.step(start)
    x, v = o.get_state()
    keys, lam, gam = o.active_get()
    sim = B.Sim(s)
    B.bf_set_state(sim.h, x, v)
    B.bf_set_active_set(sim.h, keys, lam, gam)
    st_o = o.step(1)[1][0]
    _, st_g = sim.step(1)
    xo, vo = o.get_state()
    xg, vg = sim.state()
    diag = s.bbox_diag()
    assert np.abs(xg - xo).max() <= 1e-6 * diag
    assert st_g[0]["outer_iters"] == st_o["outer_iters"]
    ko, _, _ = o.active_get()
    kg, _, _ = B.bf_get_active_set(sim.h)
    assert keyset(ko) == keyset(kg)
    sim.close()


def test_trajectory_fp64(torch_cuda):
    s = scenes.two_cubes(0)
    o = O.Oracle(s)
    sim = B.Sim(s)
    diag = s.bbox_diag()
    errs = []
    for step in range(s.n_steps):
        o.step(1)
        sim.step(1)
        xo, _ = o.get_state()
        xg, _ = sim.state()
        errs.append(np.abs(xg - xo).max() / diag)
    print("per-step max error / bbox diagonal:", ["%.2e" % e for e in errs])
    assert max(errs) <= 1e-6
    sim.close()


def test_trajectory_mixed(torch_cuda):
    s = scenes.two_cubes(0, precision=1)
    p64 = scenes.Params(**{**s.params.__dict__, "precision": 0})
    o = O.Oracle(s, p64)
    sim = B.Sim(s)
    diag = s.bbox_diag()
    errs = []
    for step in range(s.n_steps):
        o.step(1)
        sim.step(1)
        xo, _ = o.get_state()
        xg, _ = sim.state()
        errs.append(np.abs(xg - xo).max() / diag)
    print("mixed per-step max error / bbox diagonal:", ["%.2e" % e for e in errs])
    assert max(errs) <= 1e-4
    sim.close()


def test_step_host_matches_device_path(torch_cuda):
    """bf_step_host (state through host buffers) computes the same steps as
    bf_step; the atomics of the assembly and SpMV make the summation order,
    hence the last bits, vary between runs, so the bar is the FP64 parity
    tolerance."""
    s = scenes.two_cubes(1)
    a = B.Sim(s)
    b = B.Sim(s)
    a.step(6)
    x, v = s.x0.copy(), s.v0.copy()
    xo, vo = np.zeros_like(x), np.zeros_like(v)
    for i in range(6):
        B.bf_step_host(b.h, x, v, xo, vo)
        x, v = xo.copy(), vo.copy()
    xa, va = a.state()
    assert np.abs(xa - xo).max() <= 1e-6 * s.bbox_diag()
    a.close()
    b.close()


def test_free_fall_and_no_obstacles(torch_cuda):
    s = scenes.single_cube(seed=3, cells=3, v0=(0.2, 0.1, -0.3))
    sim = B.Sim(s)
    _, st = sim.step(1)
    assert st[0]["outer_iters"] == 2 and st[0]["n_contacts"] == 0
    x, v = sim.state()
    h, g = s.params.dt, np.array(s.params.gravity)
    assert np.abs(x - (s.x0 + h * s.v0 + h * h * g)).max() <= 1e-9
    sim.close()


def test_mixed_assembly_full_size_sampled(torch_cuda):
    """eight-cube scene at full size (196,608 tets, FP32 Hessian blocks):
    the FP64 gradient and the FP32 Hessian action agree with the oracle."""
    torch = torch_cuda
    s = scenes.eight_cubes(0)
    p64 = scenes.Params(**{**s.params.__dict__, "precision": 0})
    o = O.Oracle(s, p64)
    sim = B.Sim(s)
    x = s.x0
    xt = o.xtilde()
    rng = np.random.default_rng(2)
    xh = x + 3e-4 * rng.standard_normal(x.shape) * (s.dirichlet == 0)[:, None]
    mu = o.mu_init(xh, xt)
    mu_g = B.bf_mu_init(sim.h, dev(torch, xt), dev(torch, xh))
    assert mu_g == pytest.approx(mu, rel=1e-5)
    B.bf_set_mu(sim.h, mu, s.params.delta)
    E_o, G_o = o.assemble(xt, x, xh)
    G_g = torch.zeros((s.nv, 3), dtype=torch.float64, device="cuda")
    B.bf_assemble(sim.h, dev(torch, xt), dev(torch, x), dev(torch, xh), G_g)
    assert np.abs(host(G_g) - G_o).max() <= 1e-9 * np.abs(G_o).max()
    w = rng.standard_normal((s.nv, 3))
    y_o = o.hess_apply(w)
    y_g = torch.zeros_like(G_g)
    B.bf_hess_apply(sim.h, dev(torch, w), y_g)
    free = s.dirichlet == 0
    assert np.abs(host(y_g)[free] - y_o[free]).max() <= 1e-5 * np.abs(y_o[free]).max()
    sim.close()


def test_ccd_full_size(torch_cuda):
    """eight-cube scene: a falling motion of one time step; hit sets and
    TOIs equal the oracle's."""
    torch = torch_cuda
    s = scenes.eight_cubes(0)
    o = O.Oracle(s)
    sim = B.Sim(s)
    x = s.x0
    rng = np.random.default_rng(5)
    free = (s.dirichlet == 0)[:, None]
    x1 = x + free * (np.array([0.0, 0.0, -0.07]) + 2e-3 * rng.standard_normal(x.shape))
    k_o, t_o = o.ccd_hits(x, x1)
    k_g, t_g = B.bf_ccd_hits(sim.h, dev(torch, x), dev(torch, x1))
    assert len(k_o) > 100
    A = {tuple(k): t for k, t in zip(k_o.tolist(), t_o)}
    Bm = {tuple(k): t for k, t in zip(k_g.tolist(), t_g)}
    assert A.keys() == Bm.keys()
    assert all(Bm[k] == A[k] for k in A)
    sim.close()


def test_empty_and_edge_cases(torch_cuda):
    torch = torch_cuda
    s = scenes.single_cube(seed=0, cells=1, with_ground=True, z=0.3)
    sim = B.Sim(s)
    # empty active set: update with no motion adds nothing
    x = dev(torch, s.x0)
    assert B.bf_update_active_set(sim.h, x, x) == 0
    assert B.bf_max_step_size(sim.h, x, x) == 1.0
    k, l, g = B.bf_get_active_set(sim.h)
    assert len(k) == 0
    # unknown key is rejected, bad sizes are rejected
    with pytest.raises(B.BfError):
        B.bf_set_active_set(sim.h, np.array([[0, 0, 1, 2, 3]]), np.zeros(1), np.ones(1))
    toi = torch.zeros(0, dtype=torch.float64, device="cuda")
    B.bf_accd(0, toi, toi, 0.1, toi)
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_pcg_persistent_matches_per_phase_launches(torch_cuda, contact_state, precision):
    """The persistent cooperative PCG (resident with the single-reduction
    recurrence under mode 1, resident with two reductions per iteration under
    mode 129, streamed, and the two global-memory variants: in mixed
    precision the symmetric one under mode 33 and the full-row one under 97)
    and the one-launch-per-phase PCG reach the same solution in about the
    same number of iterations (the same Krylov iterates in exact
    arithmetic); all solve the oracle's system to the tolerance (mixed
    precision: FP32 matrix, so the FP64 residual is looser)."""
    torch = torch_cuda
    s, x, v, keys, lam, gam = contact_state
    sim, o = make_pair(s, x, v, keys, lam, gam, precision)
    xt = o.xtilde()
    o.mu_init(x, xt)
    B.bf_mu_init(sim.h, dev(torch, xt), dev(torch, x))
    o.linearize(x)
    B.bf_linearize(sim.h, dev(torch, x))
    _, G_o = o.assemble(xt, x, x)
    G_g = torch.zeros((s.nv, 3), dtype=torch.float64, device="cuda")
    B.bf_assemble(sim.h, dev(torch, xt), dev(torch, x), dev(torch, x), G_g)
    b = -G_o
    H = o.hess_dense()
    sols, its = [], []
    # resident (one reduction per iteration), resident with two, streamed,
    # global (symmetric in mixed), full-row global, per-phase
    modes = (1, 129, 17, 33, 97, 0)
    for mode in modes:
        B.bf_set_pcg_mode(sim.h, mode)
        xg = torch.zeros_like(G_g)
        it, _ = B.bf_pcg(sim.h, dev(torch, b), xg, 1e-6, 100000)
        if mode in (33, 97):
            assert B.bf_get_pcg_config(sim.h)["resident"] == (3 if precision and mode == 33 else 2)
        if mode in (1, 129) and precision:  # FP64 blocks of this system do not fit in one CTA's shared memory
            assert B.bf_get_pcg_config(sim.h)["resident"] == (4 if mode == 1 else 1)
        sols.append(host(xg).reshape(-1))
        its.append(it)
    bar = 1e-6 * 1.01 if precision == 0 else 1e-4
    for p in sols:
        assert np.linalg.norm(H @ p - b.reshape(-1)) <= bar * np.linalg.norm(b)
    last = len(modes) - 1
    for k in range(last):
        assert abs(its[k] - its[last]) <= max(2, its[last] // 20)
        assert np.linalg.norm(sols[k] - sols[last]) <= 1e-4 * np.linalg.norm(sols[last])
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_pcg_modes_agree_on_a_multi_cta_system(torch_cuda, precision):
    """On a system split over several CTAs (a 20k-tet scene after a few
    steps, with contacts), the resident (two reductions per iteration, and
    the single-reduction recurrence), streamed and global-vector persistent
    variants (in mixed precision both the symmetric one and the one
    streaming both triangles) at one and two CTAs per SM and the per-phase
    launches reach the tolerance on the library's own operator and agree
    with each other, iteration counts within 5 %; the autotuner then times
    them and sets one whose solve meets the tolerance."""
    torch = torch_cuda
    from paper_2512_12151_b300 import serving
    s = scenes.batch_scene(11, 1.8e4, 2e4, precision=precision)
    h, keep = serving.create(s)
    try:
        B.bf_step(h, 6)
        x, _ = B.bf_get_state(h, s.nv)
        xd = dev(torch, x)
        xt = torch.zeros_like(xd)
        B.bf_xtilde(h, xt)
        B.bf_mu_init(h, xt, xd)
        B.bf_linearize(h, xd)
        G = torch.zeros_like(xd)
        B.bf_assemble(h, xt, xd, xd, G)
        b = -G
        sols, its, grids = [], [], []
        modes = (1, 2, 129, 130, 17, 18, 33, 34, 97, 98, 0)
        for mode in modes:
            B.bf_set_pcg_mode(h, mode)
            p = torch.zeros_like(xd)
            it, _ = B.bf_pcg(h, b, p, 1e-6, 100000)
            Hp = torch.zeros_like(xd)
            B.bf_hess_apply(h, p, Hp)
            res = float(torch.linalg.norm(Hp - b) / torch.linalg.norm(b))
            assert res <= (1.01e-6 if precision == 0 else 1e-4), (mode, res)
            sols.append(host(p).reshape(-1))
            its.append(it)
            grids.append(B.bf_get_pcg_config(h))
        # several CTAs; the single-reduction resident variant under 1 and 2,
        # the two-reduction one under 129 and 130, the symmetric variant
        # (mixed) or the full-row one (FP64) under 33, the full-row one under 97
        assert grids[0]["ctas"] > 1 and grids[6]["resident"] == (3 if precision else 2)
        if precision:  # FP64 blocks: the resident variants do not fit at this split
            assert [g["resident"] for g in grids[:4]] == [4, 4, 1, 1]
        assert grids[8]["resident"] == 2
        last = len(modes) - 1
        for k in range(last):
            assert abs(its[k] - its[last]) <= max(2, its[last] // 20), its
            assert np.linalg.norm(sols[k] - sols[last]) <= 1e-4 * np.linalg.norm(sols[last])
        best, timed = B.bf_autotune_pcg(h, 64)
        assert best in timed and set(timed) <= set(modes) and 1 in timed and 0 in timed
        # the choice is within 2 % of the fastest (a later candidate must win by more)
        assert all(t > 0 for t in timed.values()) and 0.98 * timed[best] <= min(timed.values())
        assert B.bf_get_pcg_config(h)["mode"] == (0 if best == 0 else 1)
        p = torch.zeros_like(xd)
        B.bf_pcg(h, b, p, 1e-6, 100000)
        Hp = torch.zeros_like(xd)
        B.bf_hess_apply(h, p, Hp)
        assert float(torch.linalg.norm(Hp - b) / torch.linalg.norm(b)) <= (1.01e-6 if precision == 0 else 1e-4)
    finally:
        B.bf_scene_destroy(h)


@pytest.fixture(scope="module")
def multi_cta_state():
    """a 16k-tet scene (two stacked cubes, 3,460 vertices: the persistent
    PCG splits it over several CTAs) advanced by the oracle into contact"""
    s = scenes.batch_scene(11, 1.8e4, 2e4, precision=0)
    o = O.Oracle(s)
    o.step(5)
    x, v = o.get_state()
    keys, lam, gam = o.active_get()
    assert len(keys) > 100
    return s, x, v, keys, lam, gam


@pytest.mark.parametrize("precision,mode", [(0, 1), (1, 1), (0, 129), (1, 129), (1, 257), (1, 385)])
def test_one_step_multi_cta_scene(torch_cuda, multi_cta_state, precision, mode):
    """One time step from an oracle contact state on a system the persistent
    PCG spreads over several CTAs, with the single-reduction recurrence (mode
    1) and with two reductions per iteration (mode 129), each also with no
    contact pair cached in shared memory (+256: every pair takes the path
    that reads it from global memory): positions within 1e-6 (FP64) or 1e-4
    (mixed) x the bounding-box diagonal, same active set in FP64."""
    s, x, v, keys, lam, gam = multi_cta_state
    sim, o = make_pair(s, x, v, keys, lam, gam, precision)
    B.bf_set_pcg_mode(sim.h, mode)
    o.step(1)
    _, st = sim.step(1)
    cfg = B.bf_get_pcg_config(sim.h)
    assert cfg["ctas"] > 1
    if precision:  # FP64 blocks: the resident variants do not fit at this split
        assert cfg["resident"] == (1 if mode & 128 else 4)
    xo, vo = o.get_state()
    xg, vg = sim.state()
    tol = (1e-6 if precision == 0 else 1e-4) * s.bbox_diag()
    assert np.abs(xg - xo).max() <= tol, np.abs(xg - xo).max()
    if precision == 0:
        ko, _, _ = o.active_get()
        kg, _, _ = B.bf_get_active_set(sim.h)
        assert keyset(ko) == keyset(kg)
    sim.close()


@pytest.mark.parametrize("mode", [1, 129])
def test_one_step_fp64_resident_scene(torch_cuda, mode):
    """FP64 on a scene whose FP64 blocks fit in shared memory (a 2k-tet
    stack over three CTAs): one time step from an oracle contact state with
    the single-reduction recurrence (mode 1, variant 4) and with two
    reductions per iteration (mode 129, variant 1) lands within 1e-6 x the
    bounding-box diagonal of the oracle's step, with the same active set."""
    s = scenes.batch_scene(5, 1e3, 2e3, precision=0)
    o = O.Oracle(s)
    for _ in range(40):
        o.step(1)
        if len(o.active_get()[0]) > 0:
            break
    x, v = o.get_state()
    keys, lam, gam = o.active_get()
    assert len(keys) > 0
    sim, o2 = make_pair(s, x, v, keys, lam, gam, 0)
    B.bf_set_pcg_mode(sim.h, mode)
    o2.step(1)
    st, _ = sim.step(1)
    assert st == 0
    cfg = B.bf_get_pcg_config(sim.h)
    assert cfg["ctas"] > 1 and cfg["resident"] == (4 if mode == 1 else 1)
    xo, _ = o2.get_state()
    xg, _ = sim.state()
    assert np.abs(xg - xo).max() <= 1e-6 * s.bbox_diag(), np.abs(xg - xo).max()
    assert keyset(o2.active_get()[0]) == keyset(B.bf_get_active_set(sim.h)[0])
    sim.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_pcg_uncached_contact_pairs(torch_cuda, precision):
    """With no contact pair cached in shared memory (bf_set_pcg_mode + 256),
    every persistent variant reads its pairs, and for the single-reduction
    form the recurrences at the pairs' vertices, from global memory; on a
    multi-CTA system in contact the solutions agree with the cached runs and
    with the per-phase launches, iteration counts within 5 %."""
    torch = torch_cuda
    from paper_2512_12151_b300 import serving
    s = scenes.batch_scene(11, 1.8e4, 2e4, precision=precision)
    h, keep = serving.create(s)
    try:
        B.bf_step(h, 6)
        x, _ = B.bf_get_state(h, s.nv)
        xd = dev(torch, x)
        xt = torch.zeros_like(xd)
        B.bf_xtilde(h, xt)
        B.bf_mu_init(h, xt, xd)
        B.bf_linearize(h, xd)
        assert len(B.bf_get_active_set(h)[0]) > 0
        G = torch.zeros_like(xd)
        B.bf_assemble(h, xt, xd, xd, G)
        b = -G
        modes = (1, 257, 385, 273, 289, 353, 0)  # resident 1-red., 2-red., streamed, global (sym), full-row, per-phase
        sols, its, res = [], [], []
        for mode in modes:
            B.bf_set_pcg_mode(h, mode)
            p = torch.zeros_like(xd)
            it, _ = B.bf_pcg(h, b, p, 1e-6, 100000)
            Hp = torch.zeros_like(xd)
            B.bf_hess_apply(h, p, Hp)
            res.append(float(torch.linalg.norm(Hp - b) / torch.linalg.norm(b)))
            sols.append(host(p).reshape(-1))
            its.append(it)
        assert max(res) <= (1.01e-6 if precision == 0 else 1e-4), res
        last = len(modes) - 1
        for k in range(last):
            assert abs(its[k] - its[last]) <= max(2, its[last] // 20), its
            assert np.linalg.norm(sols[k] - sols[last]) <= 1e-4 * np.linalg.norm(sols[last])
    finally:
        B.bf_scene_destroy(h)


def test_pcg_bounded_waits_report_and_recover(torch_cuda):
    """Failure detection without a GPU fault: with the grid barriers waiting
    on a word that no CTA increments (bf_test_pcg_barrier_fail), the first
    grid-wide reduction of a solve never completes, every CTA of each
    persistent variant (single-reduction resident, two-reduction resident,
    symmetric) gives up after its 2 s limit and the solve returns BF_E_CUDA;
    the next solve on the same scene and context succeeds."""
    import time
    torch = torch_cuda
    from paper_2512_12151_b300 import serving
    s = scenes.batch_scene(11, 1.8e4, 2e4, precision=1)
    h, keep = serving.create(s)
    try:
        B.bf_step(h, 2)
        x, _ = B.bf_get_state(h, s.nv)
        xd = dev(torch, x)
        xt = torch.zeros_like(xd)
        B.bf_xtilde(h, xt)
        B.bf_mu_init(h, xt, xd)
        B.bf_linearize(h, xd)
        G = torch.zeros_like(xd)
        B.bf_assemble(h, xt, xd, xd, G)
        for mode, variant in ((1, 4), (129, 1), (33, 3)):
            B.bf_set_pcg_mode(h, mode)
            p = torch.zeros_like(xd)
            B.bf_pcg(h, -G, p, 1e-6, 100000)  # set-up solve
            assert B.bf_get_pcg_config(h)["resident"] == variant
            B.bf_test_pcg_barrier_fail(h, 1)
            t0 = time.perf_counter()
            with pytest.raises(B.BfError) as e:
                B.bf_pcg(h, -G, torch.zeros_like(xd), 1e-6, 100000)
            assert e.value.status == -3  # BF_E_CUDA
            assert 1.5 < time.perf_counter() - t0 < 30.0  # every CTA waited out its 2 s limit, no longer
            B.bf_test_pcg_barrier_fail(h, 0)
            p = torch.zeros_like(xd)
            it, _ = B.bf_pcg(h, -G, p, 1e-6, 100000)
            Hp = torch.zeros_like(xd)
            B.bf_hess_apply(h, p, Hp)
            assert it > 0 and float(torch.linalg.norm(Hp + G) / torch.linalg.norm(G)) <= 1e-4
        assert B.bf_step(h, 1)[0] == 0  # the scene steps on
    finally:
        B.bf_scene_destroy(h)
