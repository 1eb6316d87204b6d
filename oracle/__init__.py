"""ctypes wrapper of the plain FP64 C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline leg.  The CUDA library never imports or calls it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile oracle.c (FP64, -ffp-contract=off, single-threaded)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-o", _LIB, _SRC, "-lm"])
    return _LIB


class OrParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("delta", C.c_double), ("gravity", C.c_double * 3),
                ("eps", C.c_double), ("cg_tol", C.c_double), ("gamma_decay", C.c_double),
                ("c_mu", C.c_double), ("s_ccd", C.c_double), ("mu_f", C.c_double),
                ("eps_v", C.c_double), ("res_tol", C.c_double), ("k_min", C.c_int32),
                ("max_outer", C.c_int32), ("max_newton", C.c_int32), ("max_ls", C.c_int32),
                ("max_cg", C.c_int32), ("precision", C.c_int32), ("model", C.c_int32),
                ("ccd_reuse", C.c_int32)]


class OrStats(C.Structure):
    _fields_ = [("outer_iters", C.c_int32), ("newton_iters", C.c_int32), ("cg_iters", C.c_int32),
                ("n_contacts", C.c_int32), ("status", C.c_int32), ("ls_fail", C.c_int32),
                ("cg_maxit", C.c_int32), ("stalls", C.c_int32), ("mean_alpha", C.c_double),
                ("min_alpha", C.c_double), ("mu", C.c_double), ("beta", C.c_double),
                ("delta", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int32)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.or_snh_psi.restype = C.c_double
        L.or_pt_dist2.restype = C.c_double
        L.or_ee_dist2.restype = C.c_double
        L.or_pair_dist_grad.restype = C.c_double
        L.or_friction_f0.restype = C.c_double
        L.or_friction_f0.argtypes = [C.c_double, C.c_double, _D, _D]
        L.or_friction_eval.restype = C.c_double
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.c_int32, _D, _D, _D, C.c_int32, _I, _I, C.c_int32, _D, C.c_int32, _I,
                                C.POINTER(C.c_uint8), C.POINTER(OrParams)]
        L.or_destroy.argtypes = [C.c_void_p]
        for name in ("or_get_mu", "or_mu_init", "or_assemble", "or_energy_L", "or_max_step_size", "or_inversion_step",
                     "or_newton_residual"):
            getattr(L, name).restype = C.c_double
        L.or_set_mu_delta.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.or_get_residual_log.argtypes = [C.c_void_p, C.c_int32, _D]
        L.or_pcg.argtypes = [C.c_void_p, _D, _D, C.c_double, C.c_int32]
        L.or_accd.argtypes = [C.c_int, _D, _D, C.c_double, C.c_double, C.c_int32, _D]
        L.or_lame.argtypes = [C.c_double, C.c_double, _D, _D]
        L.or_snh_psi.argtypes = [_D, C.c_double, C.c_double]
        L.or_snh_pk1.argtypes = [_D, C.c_double, C.c_double, _D]
        L.or_snh_hess9.argtypes = [_D, C.c_double, C.c_double, _D]
        L.or_elem_grad_hess.argtypes = [_D, _D, C.c_double, C.c_double, C.c_double, C.c_int, _D, _D, _D]
        L.or_elem_grad_hess_model.argtypes = [C.c_int, _D, _D, C.c_double, C.c_double, C.c_double, C.c_int, _D, _D,
                                              _D]
        L.or_cor_psi.restype = C.c_double
        L.or_cor_psi.argtypes = [_D, C.c_double, C.c_double]
        L.or_cor_pk1.argtypes = [_D, C.c_double, C.c_double, _D]
        L.or_cor_hess9.argtypes = [_D, C.c_double, C.c_double, _D]
        L.or_nh_psi.restype = C.c_double
        L.or_nh_psi.argtypes = [_D, C.c_double, C.c_double]
        L.or_nh_pk1.argtypes = [_D, C.c_double, C.c_double, _D]
        L.or_nh_hess9.argtypes = [_D, C.c_double, C.c_double, _D]
        L.or_cubic_first_root.restype = C.c_double
        L.or_cubic_first_root.argtypes = [_D]
        L.or_det_cubic.argtypes = [_D, _D, C.c_double, _D]
        L.or_pair_dist_grad.argtypes = [C.c_int, _D, _D]
    return _lib


def _p(a):
    """pointer to a contiguous numpy array (float64 / int32 / uint8)"""
    if a is None:
        return None
    if a.dtype == np.float64:
        return a.ctypes.data_as(_D)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_I)
    if a.dtype == np.uint8:
        return a.ctypes.data_as(C.POINTER(C.c_uint8))
    raise TypeError(a.dtype)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


# ---------------- element-level functions ----------------
def lame(E, nu):
    mu, lam = C.c_double(), C.c_double()
    lib().or_lame(E, nu, C.byref(mu), C.byref(lam))
    return mu.value, lam.value


def snh_psi(F, mu, lam):
    return lib().or_snh_psi(_p(_f64(F, 9)), mu, lam)


def snh_pk1(F, mu, lam):
    P = np.zeros(9)
    lib().or_snh_pk1(_p(_f64(F, 9)), C.c_double(mu), C.c_double(lam), _p(P))
    return P.reshape(3, 3)


def snh_hess9(F, mu, lam):
    H = np.zeros(81)
    lib().or_snh_hess9(_p(_f64(F, 9)), C.c_double(mu), C.c_double(lam), _p(H))
    return H.reshape(9, 9)


def cor_psi(F, mu, lam):
    return lib().or_cor_psi(_p(_f64(F, 9)), mu, lam)


def cor_pk1(F, mu, lam):
    P = np.zeros(9)
    lib().or_cor_pk1(_p(_f64(F, 9)), mu, lam, _p(P))
    return P.reshape(3, 3)


def cor_hess9(F, mu, lam):
    H = np.zeros(81)
    lib().or_cor_hess9(_p(_f64(F, 9)), mu, lam, _p(H))
    return H.reshape(9, 9)


def nh_psi(F, mu, lam):
    return lib().or_nh_psi(_p(_f64(F, 9)), mu, lam)


def nh_pk1(F, mu, lam):
    P = np.zeros(9)
    lib().or_nh_pk1(_p(_f64(F, 9)), mu, lam, _p(P))
    return P.reshape(3, 3)


def nh_hess9(F, mu, lam):
    H = np.zeros(81)
    lib().or_nh_hess9(_p(_f64(F, 9)), mu, lam, _p(H))
    return H.reshape(9, 9)


def cubic_first_root(c):
    """smallest root in (0, 1] of c0 + c1 t + c2 t^2 + c3 t^3 (c0 > 0), else 1"""
    return lib().or_cubic_first_root(_p(_f64(c, 4)))


def det_cubic(A, B, s):
    """coefficients (c0..c3) of det(A + t B) - s det(A)"""
    c = np.zeros(4)
    lib().or_det_cubic(_p(_f64(A, 9)), _p(_f64(B, 9)), s, _p(c))
    return c


def sym_eig(A):
    A = _f64(A)
    n = A.shape[0]
    w, Q = np.zeros(n), np.zeros((n, n))
    lib().or_sym_eig(C.c_int(n), _p(A), _p(w), _p(Q))
    return w, Q


def psd_project(A):
    A = _f64(A)
    n = A.shape[0]
    out = np.zeros((n, n))
    lib().or_psd_project(C.c_int(n), _p(A), _p(out))
    return out


def elem_F(x12, B):
    F = np.zeros(9)
    lib().or_elem_F(_p(_f64(x12, 12)), _p(_f64(B, 9)), _p(F))
    return F.reshape(3, 3)


def elem_grad_hess(x12, B, vol, mu, lam, project=True, model=0):
    psi = C.c_double()
    g, H = np.zeros(12), np.zeros(144)
    lib().or_elem_grad_hess_model(int(model), _p(_f64(x12, 12)), _p(_f64(B, 9)), vol, mu, lam, int(project),
                                  C.byref(psi), _p(g), _p(H))
    return psi.value, g, H.reshape(12, 12)


def pt_dist2(p, a, b, c):
    return lib().or_pt_dist2(*[_p(_f64(v, 3)) for v in (p, a, b, c)])


def ee_dist2(a0, a1, b0, b1):
    return lib().or_ee_dist2(*[_p(_f64(v, 3)) for v in (a0, a1, b0, b1)])


def pair_dist_grad(ptype, x12):
    g = np.zeros(12)
    d = lib().or_pair_dist_grad(ptype, _p(_f64(x12, 12)), _p(g))
    return d, g


def accd(ptype, x0, x1, s=0.1, tmax=1.0, max_iter=100000):
    t = C.c_double(np.inf)
    hit = lib().or_accd(ptype, _p(_f64(x0, 12)), _p(_f64(x1, 12)), s, tmax, max_iter, C.byref(t))
    return t.value if hit else np.inf


def friction_f0(y, eh):
    """(f0, f0', f0'') of the smoothed norm at y (appendix A)"""
    f1, f2 = C.c_double(), C.c_double()
    f0 = lib().or_friction_f0(float(y), float(eh), C.byref(f1), C.byref(f2))
    return f0, f1.value, f2.value


def params_struct(p) -> OrParams:
    s = OrParams()
    s.dt, s.delta = p.dt, p.delta
    s.gravity[:] = list(p.gravity)
    s.eps, s.cg_tol, s.gamma_decay, s.c_mu, s.s_ccd = p.eps, p.cg_tol, p.gamma_decay, p.c_mu, p.s_ccd
    s.mu_f, s.eps_v = p.mu_f, p.eps_v
    s.res_tol = getattr(p, "res_tol", 0.0)
    s.k_min, s.max_outer, s.max_newton, s.max_ls, s.max_cg = (p.k_min, p.max_outer, p.max_newton,
                                                             p.max_ls, p.max_cg)
    s.precision = p.precision
    s.model = p.model
    s.ccd_reuse = getattr(p, "ccd_reuse", 0)
    return s


class Oracle:
    """One scene in the oracle.  Mirrors the C functions of oracle.h."""

    def __init__(self, scene, params=None):
        self.scene = scene
        p = params if params is not None else scene.params
        self.params = p
        self._keep = [_f64(scene.rest), _f64(scene.x0), _f64(scene.v0),
                      np.ascontiguousarray(scene.tets, np.int32), np.ascontiguousarray(scene.tet_mat, np.int32),
                      _f64(scene.mats), np.ascontiguousarray(scene.tris, np.int32),
                      np.ascontiguousarray(scene.dirichlet, np.uint8)]
        r, x0, v0, t, tm, m, tr, d = self._keep
        self._prm = params_struct(p)
        self.h = lib().or_create(scene.nv, _p(r), _p(x0), _p(v0), scene.nt, _p(t), _p(tm), len(m), _p(m),
                                 len(tr), _p(tr), _p(d), C.byref(self._prm))
        self.nv = scene.nv

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_destroy(self.h)
            self.h = None

    # state
    def get_state(self):
        x, v = np.zeros((self.nv, 3)), np.zeros((self.nv, 3))
        lib().or_get_state(C.c_void_p(self.h), _p(x), _p(v))
        return x, v

    def set_state(self, x=None, v=None):
        lib().or_set_state(C.c_void_p(self.h), _p(None if x is None else _f64(x)),
                           _p(None if v is None else _f64(v)))

    def set_dirichlet_targets(self, targets):
        lib().or_set_dirichlet_targets(C.c_void_p(self.h), _p(_f64(targets)))

    def surface(self):
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        lib().or_surface_sizes(C.c_void_p(self.h), C.byref(a), C.byref(b), C.byref(c))
        sv, st, se = (np.zeros(a.value, np.int32), np.zeros((b.value, 3), np.int32),
                      np.zeros((c.value, 2), np.int32))
        lib().or_surface(C.c_void_p(self.h), _p(sv), _p(st), _p(se))
        return sv, st, se

    def mass(self):
        m = np.zeros(self.nv)
        lib().or_mass(C.c_void_p(self.h), _p(m))
        return m

    @property
    def mu(self):
        return lib().or_get_mu(C.c_void_p(self.h))

    def set_mu_delta(self, mu, delta):
        lib().or_set_mu_delta(C.c_void_p(self.h), C.c_double(mu), C.c_double(delta))

    # active set
    def active_get(self):
        n = lib().or_active_count(C.c_void_p(self.h))
        keys, lam, gam = np.zeros((n, 5), np.int32), np.zeros(n), np.zeros(n)
        if n:
            lib().or_active_get(C.c_void_p(self.h), _p(keys), _p(lam), _p(gam))
        return keys, lam, gam

    def active_verts(self):
        n = lib().or_active_count(C.c_void_p(self.h))
        v4 = np.zeros((n, 4), np.int32)
        if n:
            lib().or_active_verts(C.c_void_p(self.h), _p(v4))
        return v4

    def active_set(self, keys, lam, gam):
        keys = np.ascontiguousarray(keys, np.int32).reshape(-1, 5)
        n = lib().or_active_set(C.c_void_p(self.h), C.c_int32(len(keys)), _p(keys), _p(_f64(lam)),
                                _p(_f64(gam)))
        if n < 0:
            raise ValueError("unknown pair key")
        return n

    # pieces of Alg. 1-3
    def xtilde(self):
        o = np.zeros((self.nv, 3))
        lib().or_xtilde(C.c_void_p(self.h), _p(o))
        return o

    def mu_init(self, xhat, xtilde):
        return lib().or_mu_init(C.c_void_p(self.h), _p(_f64(xhat)), _p(_f64(xtilde)))

    def linearize(self, xlin):
        n = lib().or_active_count(C.c_void_p(self.h))
        d, g = np.zeros(n), np.zeros((n, 12))
        lib().or_linearize(C.c_void_p(self.h), _p(_f64(xlin)), _p(d), _p(g))
        return d, g

    def assemble(self, xtilde, xlin, xhat):
        g = np.zeros((self.nv, 3))
        E = lib().or_assemble(C.c_void_p(self.h), _p(_f64(xtilde)), _p(_f64(xlin)), _p(_f64(xhat)), _p(g))
        return E, g

    def slacks(self):
        n = lib().or_active_count(C.c_void_p(self.h))
        s = np.zeros(n)
        if n:
            lib().or_slacks(C.c_void_p(self.h), _p(s))
        return s

    def hess_apply(self, v):
        o = np.zeros((self.nv, 3))
        lib().or_hess_apply(C.c_void_p(self.h), _p(_f64(v)), _p(o))
        return o

    def hess_dense(self):
        n = 3 * self.nv
        o = np.zeros((n, n))
        lib().or_hess_dense(C.c_void_p(self.h), _p(o))
        return o

    def pcg(self, b, tol=None, maxit=None):
        x = np.zeros((self.nv, 3))
        it = lib().or_pcg(C.c_void_p(self.h), _p(_f64(b)), _p(x),
                          C.c_double(self.params.cg_tol if tol is None else tol),
                          C.c_int32(self.params.max_cg if maxit is None else maxit))
        return x, it

    def energy_L(self, xtilde, xlin, xhat, sfix):
        return lib().or_energy_L(C.c_void_p(self.h), _p(_f64(xtilde)), _p(_f64(xlin)), _p(_f64(xhat)),
                                 _p(_f64(sfix)))

    def solve_subproblem(self, xtilde, xlin, xhat):
        xh = _f64(xhat).copy()
        cg, lsf = C.c_int32(), C.c_int32()
        nn = lib().or_solve_subproblem(C.c_void_p(self.h), _p(_f64(xtilde)), _p(_f64(xlin)), _p(xh),
                                       C.byref(cg), C.byref(lsf))
        return xh, nn, cg.value, lsf.value

    def ccd_hits(self, x0, x1, brute=False, cap=1 << 22):
        x0, x1 = _f64(x0), _f64(x1)
        n = lib().or_ccd_hits(C.c_void_p(self.h), _p(x0), _p(x1), int(brute), 0, None, None)
        keys, toi = np.zeros((n, 5), np.int32), np.zeros(n)
        if n:
            lib().or_ccd_hits(C.c_void_p(self.h), _p(x0), _p(x1), int(brute), n, _p(keys), _p(toi))
        return keys, toi

    def update_active_set(self, x, xhat):
        return lib().or_update_active_set(C.c_void_p(self.h), _p(_f64(x)), _p(_f64(xhat)))

    def max_step_size(self, x0, x1):
        return lib().or_max_step_size(C.c_void_p(self.h), _p(_f64(x0)), _p(_f64(x1)))

    def newton_residual(self, xtilde, x):
        """(1/h) |H^-1 grad L|_inf at x with L linearised at x"""
        return lib().or_newton_residual(C.c_void_p(self.h), _p(_f64(xtilde)), _p(_f64(x)))

    def residual_log(self):
        """gradient-norm residuals of the last step's outer iterations"""
        n = lib().or_get_residual_log(C.c_void_p(self.h), 0, None)
        out = np.zeros(max(n, 1))
        lib().or_get_residual_log(C.c_void_p(self.h), n, _p(out))
        return out[:n]

    def inversion_step(self, x0, x1):
        """the inversion bound of MaxStepSize over x0 -> x1 (any model)"""
        return lib().or_inversion_step(C.c_void_p(self.h), _p(_f64(x0)), _p(_f64(x1)))

    def min_distance(self, x):
        d = C.c_double()
        lib().or_min_distance(C.c_void_p(self.h), _p(_f64(x)), C.byref(d))
        return d.value

    # ---- friction (appendix A) ----
    def friction_setup(self):
        return lib().or_friction_setup(C.c_void_p(self.h))

    def friction_get(self):
        """(vertex ids (nf, 4), weights (nf, 4), normals (nf, 3), coefficients (nf,))"""
        nf = lib().or_friction_count(C.c_void_p(self.h))
        v4, w4 = np.zeros((nf, 4), np.int32), np.zeros((nf, 4))
        n3, k = np.zeros((nf, 3)), np.zeros(nf)
        if nf:
            lib().or_friction_get(C.c_void_p(self.h), _p(v4), _p(w4), _p(n3), _p(k))
        return v4, w4, n3, k

    def friction_eval(self, xhat):
        """(energy, gradient (nv, 3), per-pair 3x3 tangent Hessians (nf, 3, 3))"""
        nf = lib().or_friction_count(C.c_void_p(self.h))
        g, A = np.zeros((self.nv, 3)), np.zeros((max(nf, 1), 3, 3))
        E = lib().or_friction_eval(C.c_void_p(self.h), _p(_f64(xhat, 3 * self.nv)), _p(g), _p(A))
        return E, g, A[:nf]

    def step_logged(self, max_iters=200):
        """one time step with its logs: (status, stats, alphas, xhats) where
        alphas[k] = alpha^[k+1] and xhats[k] = xhat^[k+1] of outer iteration k"""
        n = 3 * self.nv
        buf = np.zeros((max_iters, n))
        lib().or_set_xhat_log(C.c_void_p(self.h), _p(buf), C.c_int32(max_iters))
        try:
            status, st, alog = self.step(1, alpha_cap=max_iters)
            m = lib().or_xhat_log_count(C.c_void_p(self.h))
        finally:
            lib().or_set_xhat_log(C.c_void_p(self.h), None, C.c_int32(0))
        k = st[0]["outer_iters"]
        assert m == k <= max_iters
        return status, st, alog[:k], buf[:k].reshape(k, self.nv, 3)

    def step(self, n=1, alpha_cap=0):
        st = (OrStats * max(n, 1))()
        alog = np.zeros(max(alpha_cap, 1))
        status = lib().or_step(C.c_void_p(self.h), C.c_int32(n), st, _p(alog), C.c_int32(alpha_cap))
        out = [st[i].as_dict() for i in range(n)]
        if alpha_cap:
            return status, out, alog
        return status, out
