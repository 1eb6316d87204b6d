"""Pins of the oracle's corotated linear elasticity (COR, one of the
material models of Tab. 2): stress and Hessian by central differences of
the energy (also for inverted elements), rotation invariance, zero energy
and stress at rotations, the small-strain Hessian equal to the linear
elasticity tensor 2 mu sym + lam I (x) I in closed form, the element
gradient by differences, a PSD projected element Hessian, and free fall in
closed form with a COR body."""
import numpy as np
import pytest

import oracle as O
from paper_2512_12151_b300 import scenes

MU, LAM = 2.0, 3.0


def rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    return q if np.linalg.det(q) > 0 else -q


def vec(M):  # column-major, the oracle's 9-vector order
    return M.T.reshape(-1)


@pytest.mark.parametrize("inverted", [False, True])
def test_stress_and_hessian_by_differences(inverted):
    rng = np.random.default_rng(7 if inverted else 3)
    for _ in range(4):
        F = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
        if inverted:
            F[:, 2] *= -1.0  # det F < 0
        assert (np.linalg.det(F) < 0) == inverted
        P, H = O.cor_pk1(F, MU, LAM), O.cor_hess9(F, MU, LAM)
        eps = 1e-6
        for a in range(3):
            for b in range(3):
                E = np.zeros((3, 3))
                E[a, b] = eps
                fd = (O.cor_psi(F + E, MU, LAM) - O.cor_psi(F - E, MU, LAM)) / (2 * eps)
                assert fd == pytest.approx(P[a, b], abs=1e-8 * np.abs(P).max())
                dP = (O.cor_pk1(F + E, MU, LAM) - O.cor_pk1(F - E, MU, LAM)) / (2 * eps)
                assert np.abs(vec(dP) - H[:, a + 3 * b]).max() <= 1e-7 * np.abs(H).max()
        assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()


def test_rotation_invariance_and_rest_state():
    rng = np.random.default_rng(1)
    F = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
    for _ in range(3):
        Q = rotation(rng)
        assert O.cor_psi(Q @ F, MU, LAM) == pytest.approx(O.cor_psi(F, MU, LAM), rel=1e-12)
        assert np.abs(O.cor_pk1(Q @ F, MU, LAM) - Q @ O.cor_pk1(F, MU, LAM)).max() <= 1e-12
        assert abs(O.cor_psi(Q, MU, LAM)) <= 1e-24 and np.abs(O.cor_pk1(Q, MU, LAM)).max() <= 1e-12


def test_small_strain_hessian_is_the_linear_elasticity_tensor():
    """d2Psi/dF2 at F = I: 2 mu (symmetrisation) + lam vec(I) vec(I)^T"""
    H = O.cor_hess9(np.eye(3), MU, LAM)
    sym = np.zeros((9, 9))
    for a in range(3):
        for b in range(3):
            E = np.zeros((3, 3))
            E[a, b] = 1.0
            sym[:, a + 3 * b] = vec(0.5 * (E + E.T))
    ref = 2 * MU * sym + LAM * np.outer(vec(np.eye(3)), vec(np.eye(3)))
    assert np.abs(H - ref).max() <= 1e-12


def test_element_gradient_by_differences_and_psd_projection():
    rng = np.random.default_rng(5)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]]) * 0.1
    Dm = (X[1:] - X[0]).T
    B = np.linalg.inv(Dm)
    vol = np.linalg.det(Dm) / 6
    x = (X + 0.02 * rng.standard_normal(X.shape)).reshape(-1)
    psi, g, H = O.elem_grad_hess(x, B.reshape(-1), vol, MU, LAM, project=True, model=1)
    eps = 1e-7
    for k in range(12):
        d = np.zeros(12)
        d[k] = eps
        fd = (O.elem_grad_hess(x + d, B.reshape(-1), vol, MU, LAM, model=1)[0] -
              O.elem_grad_hess(x - d, B.reshape(-1), vol, MU, LAM, model=1)[0]) / (2 * eps)
        assert fd == pytest.approx(g[k], abs=1e-7 * np.abs(g).max())
    assert np.linalg.eigvalsh(H).min() >= -1e-10 * np.abs(H).max()


def test_free_fall_with_cor():
    """translation keeps F = I, so one step of free fall lands on
    x + h v + h^2 g as with SNH (exactly 2 outer iterations)"""
    s = scenes.single_cube(seed=0, cells=2, z=0.5, with_ground=False)
    s.params.model = 1
    o = O.Oracle(s)
    st, stats = o.step(1)
    assert st == 0 and stats[0]["outer_iters"] == 2
    x, v = o.get_state()
    h, g = s.params.dt, np.array(s.params.gravity)
    assert np.abs(x - (s.x0 + h * s.v0 + h * h * g)).max() <= 1e-9
