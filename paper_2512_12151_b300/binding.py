"""Thin ctypes binding of include/bf.h (argument marshalling only).

Every function named bf_* mirrors the C entry point of the same name.  The
shared library libbf.so must have been built (paper_2512_12151_b300.build);
importing the binding without it raises: there is no fallback path.
Device buffers are passed as torch CUDA tensors (their data_ptr()), host
buffers as numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbf.so")

BF_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "device allocation failed", -3: "CUDA error",
          -4: "PCG reached max_cg", -5: "Newton loop reached max_newton", -6: "line search failed",
          -7: "time step reached max_outer", -8: "non-finite value", -9: "work buffer capacity exceeded",
          -10: "pair key or ticket not found", -11: "HBM budget exceeded"}
BF_E_BUDGET = -11


class BfError(RuntimeError):
    def __init__(self, fn, status):
        super().__init__(f"{fn} failed with status {status} ({STATUS.get(status, '?')})")
        self.status = status


class bf_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("delta", C.c_double), ("gravity", C.c_double * 3),
                ("eps", C.c_double), ("cg_tol", C.c_double), ("gamma_decay", C.c_double),
                ("c_mu", C.c_double), ("s_ccd", C.c_double), ("mu_f", C.c_double),
                ("eps_v", C.c_double), ("res_tol", C.c_double), ("k_min", C.c_int32),
                ("max_outer", C.c_int32), ("max_newton", C.c_int32), ("max_ls", C.c_int32),
                ("max_cg", C.c_int32), ("precision", C.c_int32), ("model", C.c_int32),
                ("ccd_reuse", C.c_int32)]


class bf_step_stats(C.Structure):
    _fields_ = [("outer_iters", C.c_int32), ("newton_iters", C.c_int32), ("cg_iters", C.c_int32),
                ("n_contacts", C.c_int32), ("status", C.c_int32), ("ls_fail", C.c_int32),
                ("cg_maxit", C.c_int32), ("stalls", C.c_int32), ("mean_alpha", C.c_double),
                ("min_alpha", C.c_double), ("mu", C.c_double), ("beta", C.c_double),
                ("delta", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bf_mesh_desc(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tets", C.c_int32), ("n_mats", C.c_int32),
                ("n_obst_tris", C.c_int32), ("rest_pos", C.c_void_p), ("init_pos", C.c_void_p),
                ("init_vel", C.c_void_p), ("tets", C.c_void_p), ("tet_mat", C.c_void_p),
                ("mats", C.c_void_p), ("obst_tris", C.c_void_p), ("dirichlet", C.c_void_p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class bf_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


_lib = None
_P = C.c_void_p


def lib():
    """Load libbf.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                           "(run paper_2512_12151_b300.build.build())")
    L = C.CDLL(LIB_PATH)
    sig = {
        "bf_scene_create": [C.POINTER(bf_mesh_desc), C.POINTER(bf_params), C.POINTER(bf_allocator), _P,
                            C.POINTER(_P)],
        "bf_scene_destroy": [_P], "bf_set_stream": [_P, _P],
        "bf_step": [_P, C.c_int32, C.POINTER(bf_step_stats)],
        "bf_step_host": [_P, _P, _P, _P, _P, C.POINTER(bf_step_stats)],
        "bf_get_state": [_P, _P, _P], "bf_set_state": [_P, _P, _P],
        "bf_set_obstacle_targets": [_P, _P],
        "bf_get_active_set": [_P, C.c_int32, C.POINTER(C.c_int32), _P, _P, _P],
        "bf_set_active_set": [_P, C.c_int32, _P, _P, _P],
        "bf_get_mu": [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "bf_set_mu": [_P, C.c_double, C.c_double],
        "bf_scene_info": [_P, _P],
        "bf_xtilde": [_P, _P], "bf_mu_init": [_P, _P, _P, C.POINTER(C.c_double)],
        "bf_linearize": [_P, _P, _P, _P],
        "bf_assemble": [_P, _P, _P, _P, _P, C.POINTER(C.c_double)],
        "bf_hess_apply": [_P, _P, _P], "bf_get_bsr": [_P, _P, _P, _P],
        "bf_pcg": [_P, _P, _P, C.c_double, C.c_int32, C.POINTER(C.c_int32)],
        "bf_energy": [_P, _P, _P, _P, C.POINTER(C.c_double)],
        "bf_solve_subproblem": [_P, _P, _P, _P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
        "bf_ccd_hits": [_P, _P, _P, C.c_int32, C.POINTER(C.c_int32), _P, _P],
        "bf_update_active_set": [_P, _P, _P, C.POINTER(C.c_int32)],
        "bf_max_step_size": [_P, _P, _P, C.POINTER(C.c_double)],
        "bf_inversion_step": [_P, _P, _P, C.POINTER(C.c_double)],
        "bf_newton_residual": [_P, _P, _P, C.POINTER(C.c_double)],
        "bf_get_residual_log": [_P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double)],
        "bf_accd": [C.c_int32, C.c_int32, _P, _P, C.c_double, _P, _P],
        "bf_max_step_size_pairs_noalloc": [C.c_int32, C.c_int32, _P, _P, C.c_double, _P, _P],
        "bf_enable_timers": [_P, C.c_int32],
        "bf_get_launch_count": [_P, C.POINTER(C.c_int64)],
        "bf_set_pcg_mode": [_P, C.c_int32],
        "bf_test_pcg_barrier_fail": [_P, C.c_int32],
        "bf_autotune_pcg": [_P, C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                            C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
        "bf_get_pcg_config": [_P, _P],
        "bf_get_timers": [_P, C.c_int32, _P, _P, _P],
        "bf_scene_bytes": [_P, C.POINTER(C.c_int64)],
        "bf_save": [_P, _P, C.c_size_t, C.POINTER(C.c_size_t)],
        "bf_friction_setup": [_P, C.POINTER(C.c_int32)],
        "bf_friction_get": [_P, C.c_int32, C.POINTER(C.c_int32), _P, _P, _P, _P],
        "bf_load": [_P, _P, C.c_size_t],
        "bf_batch_create": [C.c_int32, C.c_int64, C.POINTER(_P)],
        "bf_batch_destroy": [_P],
        "bf_batch_admit": [_P, _P, C.c_int32, C.POINTER(C.c_int64)],
        "bf_batch_wait": [_P, C.c_int64, C.c_int32, C.POINTER(C.c_int32)],
        "bf_batch_result": [_P, C.c_int64, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                            C.POINTER(C.c_double), _P, _P],
        "bf_batch_release": [_P, C.c_int64],
        "bf_batch_info": [_P, _P],
        "bf_batch_set_autotune": [_P, C.c_int32],
        "bf_batch_set_blocking_sync": [_P, C.c_int32],
        "bf_set_sync_mode": [_P, C.c_int32],
        "bf_batch_tuned": [_P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.bf_status_str.argtypes = [C.c_int]
    L.bf_status_str.restype = C.c_char_p
    L.bf_batch_now.argtypes = [_P]
    L.bf_batch_now.restype = C.c_double
    _lib = L
    return L


def exported_symbols():
    return ["bf_status_str"] + [n for n in dir(lib()) if n.startswith("bf_")]


def _check(fn, st, ok=(BF_OK,)):
    if st not in ok:
        raise BfError(fn, st)
    return st


def _np_ptr(a):
    return None if a is None else a.ctypes.data


def _dptr(t):
    """device pointer of a torch CUDA tensor (or None / int pass-through)"""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return t.data_ptr()


def make_params(p) -> bf_params:
    s = bf_params()
    s.dt, s.delta = p.dt, p.delta
    s.gravity[:] = list(p.gravity)
    s.eps, s.cg_tol, s.gamma_decay, s.c_mu, s.s_ccd = p.eps, p.cg_tol, p.gamma_decay, p.c_mu, p.s_ccd
    s.mu_f, s.eps_v = p.mu_f, p.eps_v
    s.res_tol = getattr(p, "res_tol", 0.0)
    s.ccd_reuse = getattr(p, "ccd_reuse", 0)
    s.k_min, s.max_outer, s.max_newton, s.max_ls, s.max_cg = (p.k_min, p.max_outer, p.max_newton,
                                                             p.max_ls, p.max_cg)
    s.model = p.model
    s.precision = p.precision
    return s


def torch_allocator():
    """A bf_allocator backed by torch's CUDA caching allocator."""
    import torch

    def _alloc(n, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(n))
        except Exception:  # allocation failure -> NULL
            return None

    def _free(p, ctx):
        torch.cuda.caching_allocator_delete(p)
    a = bf_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    return a


# ---------------------------------------------------------------------------
# one function per entry point
# ---------------------------------------------------------------------------
def bf_scene_create(scene, params=None, allocator=None, stream=None):
    """scene: paper_2512_12151_b300.scenes.Scene; returns (handle, keepalive)."""
    keep = [np.ascontiguousarray(scene.rest, np.float64), np.ascontiguousarray(scene.x0, np.float64),
            np.ascontiguousarray(scene.v0, np.float64), np.ascontiguousarray(scene.tets, np.int32),
            np.ascontiguousarray(scene.tet_mat, np.int32), np.ascontiguousarray(scene.mats, np.float64),
            np.ascontiguousarray(scene.tris, np.int32), np.ascontiguousarray(scene.dirichlet, np.uint8)]
    m = bf_mesh_desc(scene.nv, scene.nt, len(scene.mats), len(scene.tris), *[_np_ptr(a) for a in keep])
    prm = make_params(params if params is not None else scene.params)
    h = _P()
    st = lib().bf_scene_create(C.byref(m), C.byref(prm), None if allocator is None else C.byref(allocator),
                               stream, C.byref(h))
    _check("bf_scene_create", st)
    return h.value, keep + [allocator]


def bf_scene_destroy(h):
    _check("bf_scene_destroy", lib().bf_scene_destroy(h))


def bf_set_stream(h, stream):
    _check("bf_set_stream", lib().bf_set_stream(h, stream))


def bf_step(h, n=1, ok=(BF_OK,)):
    st = (bf_step_stats * max(n, 1))()
    status = lib().bf_step(h, n, st)
    _check("bf_step", status, ok)
    return status, [st[i].as_dict() for i in range(n)]


def bf_step_host(h, x_in=None, v_in=None, x_out=None, v_out=None):
    st = bf_step_stats()
    status = lib().bf_step_host(h, _np_ptr(x_in), _np_ptr(v_in), _np_ptr(x_out), _np_ptr(v_out), C.byref(st))
    _check("bf_step_host", status)
    return st.as_dict()


def bf_get_state(h, nv):
    x, v = np.zeros((nv, 3)), np.zeros((nv, 3))
    _check("bf_get_state", lib().bf_get_state(h, _np_ptr(x), _np_ptr(v)))
    return x, v


def bf_set_state(h, x=None, v=None):
    x = None if x is None else np.ascontiguousarray(x, np.float64)
    v = None if v is None else np.ascontiguousarray(v, np.float64)
    _check("bf_set_state", lib().bf_set_state(h, _np_ptr(x), _np_ptr(v)))


def bf_set_obstacle_targets(h, targets):
    t = None if targets is None else np.ascontiguousarray(targets, np.float64)
    _check("bf_set_obstacle_targets", lib().bf_set_obstacle_targets(h, _np_ptr(t)))


def bf_get_active_set(h):
    n = C.c_int32()
    _check("bf_get_active_set", lib().bf_get_active_set(h, 0, C.byref(n), None, None, None))
    k, lam, gam = np.zeros((n.value, 5), np.int32), np.zeros(n.value), np.zeros(n.value)
    if n.value:
        _check("bf_get_active_set", lib().bf_get_active_set(h, n.value, C.byref(n), _np_ptr(k), _np_ptr(lam),
                                                            _np_ptr(gam)))
    return k, lam, gam


def bf_set_active_set(h, keys, lam, gam):
    keys = np.ascontiguousarray(keys, np.int32).reshape(-1, 5)
    lam = np.ascontiguousarray(lam, np.float64)
    gam = np.ascontiguousarray(gam, np.float64)
    _check("bf_set_active_set", lib().bf_set_active_set(h, len(keys), _np_ptr(keys), _np_ptr(lam), _np_ptr(gam)))


def bf_get_mu(h):
    mu, delta = C.c_double(), C.c_double()
    _check("bf_get_mu", lib().bf_get_mu(h, C.byref(mu), C.byref(delta)))
    return mu.value, delta.value


def bf_set_mu(h, mu, delta):
    _check("bf_set_mu", lib().bf_set_mu(h, mu, delta))


def bf_scene_info(h):
    info = np.zeros(5, np.int32)
    _check("bf_scene_info", lib().bf_scene_info(h, _np_ptr(info)))
    return dict(zip(("n_surface_verts", "n_surface_tris", "n_surface_edges", "nnzb", "n_prescribed"),
                    info.tolist()))


def bf_status_str(status):
    return lib().bf_status_str(status).decode()


def bf_xtilde(h, out):
    _check("bf_xtilde", lib().bf_xtilde(h, _dptr(out)))


def bf_mu_init(h, xtilde, xhat):
    mu = C.c_double()
    _check("bf_mu_init", lib().bf_mu_init(h, _dptr(xtilde), _dptr(xhat), C.byref(mu)))
    return mu.value


def bf_linearize(h, xlin, dist=None, grad=None):
    _check("bf_linearize", lib().bf_linearize(h, _dptr(xlin), _dptr(dist), _dptr(grad)))


def bf_assemble(h, xtilde, xlin, xhat, grad=None):
    e = C.c_double()
    _check("bf_assemble", lib().bf_assemble(h, _dptr(xtilde), _dptr(xlin), _dptr(xhat), _dptr(grad), C.byref(e)))
    return e.value


def bf_hess_apply(h, x, y):
    _check("bf_hess_apply", lib().bf_hess_apply(h, _dptr(x), _dptr(y)))


def bf_get_bsr(h, nv, nnzb):
    rp, col, val = np.zeros(nv + 1, np.int32), np.zeros(nnzb, np.int32), np.zeros((nnzb, 3, 3))
    _check("bf_get_bsr", lib().bf_get_bsr(h, _np_ptr(rp), _np_ptr(col), _np_ptr(val)))
    return rp, col, val


def bf_pcg(h, b, x, tol, maxit, ok=(BF_OK,)):
    it = C.c_int32()
    st = lib().bf_pcg(h, _dptr(b), _dptr(x), tol, maxit, C.byref(it))
    _check("bf_pcg", st, ok)
    return it.value, st


def bf_energy(h, xtilde, xlin, xhat):
    L = C.c_double()
    _check("bf_energy", lib().bf_energy(h, _dptr(xtilde), _dptr(xlin), _dptr(xhat), C.byref(L)))
    return L.value


def bf_solve_subproblem(h, xtilde, xlin, xhat):
    nn, cg = C.c_int32(), C.c_int32()
    _check("bf_solve_subproblem", lib().bf_solve_subproblem(h, _dptr(xtilde), _dptr(xlin), _dptr(xhat),
                                                            C.byref(nn), C.byref(cg)))
    return nn.value, cg.value


def bf_ccd_hits(h, x0, x1):
    n = C.c_int32()
    _check("bf_ccd_hits", lib().bf_ccd_hits(h, _dptr(x0), _dptr(x1), 0, C.byref(n), None, None))
    k, t = np.zeros((n.value, 5), np.int32), np.zeros(n.value)
    if n.value:
        _check("bf_ccd_hits", lib().bf_ccd_hits(h, _dptr(x0), _dptr(x1), n.value, C.byref(n), _np_ptr(k),
                                                _np_ptr(t)))
    return k, t


def bf_update_active_set(h, x, xhat):
    n = C.c_int32()
    _check("bf_update_active_set", lib().bf_update_active_set(h, _dptr(x), _dptr(xhat), C.byref(n)))
    return n.value


def bf_max_step_size(h, x0, x1):
    a = C.c_double()
    _check("bf_max_step_size", lib().bf_max_step_size(h, _dptr(x0), _dptr(x1), C.byref(a)))
    return a.value


def _check_pairs(n, x0, x1, out):
    """the kernels read 12 n doubles of x0 and x1 and write out: refuse
    tensors that are too small or of another type before the launch"""
    import torch
    assert out is not None and out.dtype == torch.float64 and out.is_cuda, "output must be a float64 CUDA tensor"
    if n > 0:
        for t in (x0, x1):
            assert t is not None and t.dtype == torch.float64 and t.is_cuda, "x0, x1 must be float64 CUDA tensors"
            assert t.is_contiguous() and t.numel() >= 12 * n, "x0, x1 need 12 contiguous doubles per pair"


def bf_accd(ptype, x0, x1, s, toi, stream=None):
    n = toi.numel()
    _check_pairs(n, x0, x1, toi)
    _check("bf_accd", lib().bf_accd(ptype, n, _dptr(x0), _dptr(x1), s, _dptr(toi), stream))


def bf_newton_residual(h, xtilde, x):
    """gradient-norm residual (1/h) |H^-1 grad L|_inf at x (device tensors)"""
    r = C.c_double()
    _check("bf_newton_residual", lib().bf_newton_residual(h, _dptr(xtilde), _dptr(x), C.byref(r)))
    return r.value


def bf_get_residual_log(h):
    """residuals of the last step's outer iterations (residual mode)"""
    n = C.c_int32()
    _check("bf_get_residual_log", lib().bf_get_residual_log(h, 0, C.byref(n), None))
    out = np.zeros(max(n.value, 1))
    _check("bf_get_residual_log", lib().bf_get_residual_log(h, n.value, C.byref(n),
                                                            out.ctypes.data_as(C.POINTER(C.c_double))))
    return out[: n.value]


def bf_inversion_step(h, x0, x1):
    """inversion bound of MaxStepSize along x0 -> x1 (device tensors)"""
    a = C.c_double()
    _check("bf_inversion_step", lib().bf_inversion_step(h, _dptr(x0), _dptr(x1), C.byref(a)))
    return a.value


def bf_max_step_size_pairs_noalloc(ptype, n, x0, x1, s, alpha, stream=None):
    """alpha[0] = min(1, min TOI) over the first n pairs of x0 -> x1, with no
    device allocation (see include/bf.h for the limits)."""
    _check_pairs(n, x0, x1, alpha)
    assert alpha.numel() >= 1
    _check("bf_max_step_size_pairs_noalloc",
           lib().bf_max_step_size_pairs_noalloc(ptype, n, _dptr(x0), _dptr(x1), s, _dptr(alpha), stream))


def bf_enable_timers(h, on=True):
    _check("bf_enable_timers", lib().bf_enable_timers(h, int(on)))


def bf_autotune_pcg(h, iters=64):
    """times each PCG execution configuration on the last assembled system
    and sets the fastest: (best mode, {mode: us per iteration})"""
    cap = 16
    modes = (C.c_int32 * cap)()
    us = (C.c_double * cap)()
    n, best = C.c_int32(), C.c_int32()
    _check("bf_autotune_pcg", lib().bf_autotune_pcg(h, iters, cap, modes, us, C.byref(n), C.byref(best)))
    return best.value, {int(modes[i]): float(us[i]) for i in range(min(n.value, cap))}


def bf_set_pcg_mode(h, mode):
    _check("bf_set_pcg_mode", lib().bf_set_pcg_mode(h, mode))


def bf_test_pcg_barrier_fail(h, on):
    _check("bf_test_pcg_barrier_fail", lib().bf_test_pcg_barrier_fail(h, on))


def bf_get_pcg_config(h):
    cfg = np.zeros(8, np.int32)
    _check("bf_get_pcg_config", lib().bf_get_pcg_config(h, _np_ptr(cfg)))
    return dict(zip(("mode", "ctas", "threads", "smem_bytes", "resident", "max_rows", "max_blocks", "max_window"),
                    cfg.tolist()))


def bf_get_launch_count(h):
    n = C.c_int64()
    _check("bf_get_launch_count", lib().bf_get_launch_count(h, C.byref(n)))
    return n.value


def bf_get_timers(h):
    cap = 32
    launches, ms = np.zeros(cap, np.int64), np.zeros(cap)
    names = (C.c_char_p * cap)()
    n = lib().bf_get_timers(h, cap, _np_ptr(launches), _np_ptr(ms), names)
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(n)}


def bf_friction_setup(h):
    n = C.c_int32()
    _check("bf_friction_setup", lib().bf_friction_setup(h, C.byref(n)))
    return n.value


def bf_friction_get(h):
    """(vertex ids (nf, 4), weights (nf, 4), normals (nf, 3), coefficients (nf,))"""
    n = C.c_int32()
    _check("bf_friction_get", lib().bf_friction_get(h, 0, C.byref(n), None, None, None, None))
    v4, w4 = np.zeros((n.value, 4), np.int32), np.zeros((n.value, 4))
    n3, k = np.zeros((n.value, 3)), np.zeros(n.value)
    if n.value:
        _check("bf_friction_get", lib().bf_friction_get(h, n.value, C.byref(n), _np_ptr(v4), _np_ptr(w4),
                                                        _np_ptr(n3), _np_ptr(k)))
    return v4, w4, n3, k


def bf_save(h):
    """checkpoint of the scene's evolving state as bytes"""
    n = C.c_size_t()
    _check("bf_save", lib().bf_save(h, None, 0, C.byref(n)))
    buf = (C.c_ubyte * n.value)()
    _check("bf_save", lib().bf_save(h, buf, n.value, C.byref(n)))
    return bytes(buf)


def bf_load(h, data):
    buf = (C.c_ubyte * len(data)).from_buffer_copy(data)
    _check("bf_load", lib().bf_load(h, buf, len(data)))


def bf_scene_bytes(h):
    n = C.c_int64()
    _check("bf_scene_bytes", lib().bf_scene_bytes(h, C.byref(n)))
    return n.value


def bf_batch_create(n_workers, hbm_budget_bytes):
    b = _P()
    _check("bf_batch_create", lib().bf_batch_create(n_workers, int(hbm_budget_bytes), C.byref(b)))
    return b


def bf_batch_destroy(b):
    _check("bf_batch_destroy", lib().bf_batch_destroy(b))


def bf_batch_admit(b, h, n_steps):
    """ticket, or None when the HBM budget refuses the scene"""
    t = C.c_int64()
    st = lib().bf_batch_admit(b, h, n_steps, C.byref(t))
    _check("bf_batch_admit", st, (BF_OK, BF_E_BUDGET))
    return None if st == BF_E_BUDGET else t.value


def bf_batch_wait(b, ticket, timeout_ms=-1):
    done = C.c_int32()
    _check("bf_batch_wait", lib().bf_batch_wait(b, ticket, timeout_ms, C.byref(done)))
    return bool(done.value)


def bf_batch_result(b, ticket, cap):
    n, status, t_admit = C.c_int32(), C.c_int32(), C.c_double()
    t_steps = np.zeros(max(cap, 1))
    stats = (bf_step_stats * max(cap, 1))()
    _check("bf_batch_result", lib().bf_batch_result(b, ticket, cap, C.byref(n), C.byref(status), C.byref(t_admit),
                                                    _np_ptr(t_steps), stats))
    k = min(n.value, cap)
    return {"steps_done": n.value, "status": status.value, "t_admit": t_admit.value,
            "t_steps": t_steps[:k].copy(), "stats": [stats[i].as_dict() for i in range(k)]}


def bf_batch_release(b, ticket):
    _check("bf_batch_release", lib().bf_batch_release(b, ticket))


def bf_batch_set_blocking_sync(b, on=True):
    _check("bf_batch_set_blocking_sync", lib().bf_batch_set_blocking_sync(b, 1 if on else 0))


def bf_set_sync_mode(h, blocking):
    _check("bf_set_sync_mode", lib().bf_set_sync_mode(h, 1 if blocking else 0))


def bf_batch_set_autotune(b, on=True):
    _check("bf_batch_set_autotune", lib().bf_batch_set_autotune(b, 1 if on else 0))


def bf_batch_tuned(b):
    """{size bucket: PCG mode} tuned by the batch so far"""
    cap = 64
    bk, md = (C.c_int32 * cap)(), (C.c_int32 * cap)()
    n = C.c_int32()
    _check("bf_batch_tuned", lib().bf_batch_tuned(b, cap, bk, md, C.byref(n)))
    return {int(bk[i]): int(md[i]) for i in range(min(n.value, cap))}


def bf_batch_info(b):
    info = np.zeros(6, np.int64)
    _check("bf_batch_info", lib().bf_batch_info(b, _np_ptr(info)))
    return dict(zip(("resident_bytes", "budget", "workers", "queued", "finished", "issued"), info.tolist()))


def bf_batch_now(b):
    return lib().bf_batch_now(b)


class Sim:
    """Convenience owner of one scene handle (destroys it on close)."""

    def __init__(self, scene, params=None, stream=None, use_torch_allocator=True):
        self.scene = scene
        self.params = params if params is not None else scene.params
        alloc = None
        if use_torch_allocator:
            alloc = torch_allocator()
        self.h, self._keep = bf_scene_create(scene, self.params, alloc, stream)
        self.nv = scene.nv

    def close(self):
        if getattr(self, "h", None):
            bf_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1, ok=(BF_OK,)):
        return bf_step(self.h, n, ok)

    def state(self):
        return bf_get_state(self.h, self.nv)

    def info(self):
        return bf_scene_info(self.h)
