"""Seeded synthetic scene generators.

This module produces INPUTS only: vertex positions, tetrahedra, obstacle
triangles, Dirichlet flags, materials and solver parameters.  It holds none
of the method's arithmetic (no mass lumping, no surface extraction, no
energies, no distances); both the CUDA library and the CPU oracle derive
everything else from these arrays on their own.

The scenes stand in for the paper's assets (its meshes are not available):
tetrahedralised cubes (Kuhn 6-tet split of a regular grid) dropped onto
static triangle obstacles, shaped like the workloads of the paper's
evaluation (section 6, Tab. 2): stable Neo-Hookean solids, E = 1e5 Pa,
nu = 0.4, rho = 1000 kg/m^3, h = 0.01 s, contact radius delta = 1e-3 m.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field

import numpy as np

# Kuhn (Freudenthal) split of a unit cell into 6 tets sharing the main
# diagonal 0 -> 7.  Corners are numbered by bits (x = 1, y = 2, z = 4).
# Every cell uses the same diagonal, so neighbouring cells conform.
_KUHN = []
for a, b in ((0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1)):
    ca = 1 << a
    cb = ca | (1 << b)
    _KUHN.append((0, ca, cb, 7))
_KUHN = np.array(_KUHN, dtype=np.int64)


@dataclass
class Params:
    """Solver parameters (defaults: section 6 and Alg. 1-3 of the paper).

    dt: time step h; delta: contact offset (section 4.2); eps, k_min:
    termination rule (Eq. termination, section 6 uses 1e-3 and 2);
    cg_tol: relative PCG tolerance; gamma_decay: Gamma of section 4.2;
    c_mu: C of section 5.2; s_ccd: ACCD conservative rescaling; mu_f,
    eps_v: friction coefficient and velocity threshold of the smoothed
    friction of appendix A (mu_f = 0: no friction).
    """
    dt: float = 0.01
    delta: float = 1e-3
    gravity: tuple = (0.0, 0.0, -9.8)
    eps: float = 1e-3
    k_min: int = 2
    cg_tol: float = 1e-6
    gamma_decay: float = 0.9
    c_mu: float = 0.1
    s_ccd: float = 0.1
    mu_f: float = 0.0
    eps_v: float = 1e-3
    res_tol: float = 0.0  # > 0: end a step's outer loop on the gradient-norm residual instead of beta
    max_outer: int = 1000
    max_newton: int = 50
    max_ls: int = 30
    max_cg: int = 10000
    precision: int = 0  # 0 = FP64, 1 = mixed (FP32 Hessian/SpMV/preconditioner)
    model: int = 0      # material: 0 = stable Neo-Hookean (SNH), 1 = corotated linear (COR), 2 = Neo-Hookean (NH)
    ccd_reuse: int = 0  # 1: UpdateActiveSet reuses the MaxStepSize CCD (x^[k] -> xhat^[k+1])


@dataclass
class Scene:
    name: str
    rest: np.ndarray          # (nv, 3) float64 rest positions
    x0: np.ndarray            # (nv, 3) float64 initial positions
    v0: np.ndarray            # (nv, 3) float64 initial velocities
    tets: np.ndarray          # (nt, 4) int32, positively oriented at rest
    tet_mat: np.ndarray       # (nt,) int32 material index
    mats: np.ndarray          # (nm, 3) float64: E [Pa], nu, rho [kg/m^3]
    tris: np.ndarray          # (nx, 3) int32 obstacle triangles (vertex ids)
    dirichlet: np.ndarray     # (nv,) uint8, 1 = prescribed (obstacle) vertex
    params: Params = field(default_factory=Params)
    n_steps: int = 20
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.x0.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tets.shape[0])

    def bbox_diag(self, elastic_only: bool = True) -> float:
        sel = self.dirichlet == 0 if elastic_only else slice(None)
        p = self.x0[sel]
        return float(np.linalg.norm(p.max(0) - p.min(0)))


def cube_mesh(cells: int, side: float):
    """Regular (cells+1)^3 grid on [0, side]^3 split into 6*cells^3 tets."""
    v, t = _cube_mesh_cached(int(cells), float(side))
    return v.copy(), t.copy()


@functools.lru_cache(maxsize=64)
def _cube_mesh_cached(cells: int, side: float):
    n = cells + 1
    g = np.arange(n, dtype=np.float64) * (side / cells)
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    verts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
    ii, jj, kk = np.meshgrid(np.arange(cells), np.arange(cells), np.arange(cells), indexing="ij")
    base = (kk.ravel() + n * jj.ravel() + n * n * ii.ravel())  # (x=kk, y=jj, z=ii)
    corner_off = np.array([(c & 1) + n * ((c >> 1) & 1) + n * n * ((c >> 2) & 1) for c in range(8)])
    tets = base[:, None, None] + corner_off[_KUHN][None, :, :]
    tets = tets.reshape(-1, 4)
    # orient positively on the regular grid
    d = verts[tets[:, 1:]] - verts[tets[:, :1]]
    neg = np.linalg.det(d) < 0
    tets[neg] = tets[neg][:, [0, 2, 1, 3]]
    return verts, tets.astype(np.int32)


def ground_quad(half: float, z: float = 0.0, center=(0.0, 0.0)):
    cx, cy = center
    v = np.array([[cx - half, cy - half, z], [cx + half, cy - half, z],
                  [cx + half, cy + half, z], [cx - half, cy + half, z]])
    t = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    return v, t


def open_box(half: float, height: float):
    """Floor (z=0) plus four walls, as 10 static triangles on 8 vertices."""
    v = np.array([[-half, -half, 0], [half, -half, 0], [half, half, 0], [-half, half, 0],
                  [-half, -half, height], [half, -half, height], [half, half, height],
                  [-half, half, height]], dtype=np.float64)
    t = [[0, 1, 2], [0, 2, 3]]
    for a in range(4):
        b = (a + 1) % 4
        t += [[a, b, b + 4], [a, b + 4, a + 4]]
    return v, np.array(t, dtype=np.int32)


class _Builder:
    def __init__(self):
        self.verts, self.tets, self.mat, self.tris, self.dir = [], [], [], [], []
        self.nv = 0

    def add_solid(self, verts, tets, mat):
        self.verts.append(verts)
        self.tets.append(tets + self.nv)
        self.mat.append(np.full(len(tets), mat, dtype=np.int32))
        self.dir.append(np.zeros(len(verts), dtype=np.uint8))
        self.nv += len(verts)

    def add_obstacle(self, verts, tris):
        self.verts.append(verts)
        self.tris.append(tris + self.nv)
        self.dir.append(np.ones(len(verts), dtype=np.uint8))
        self.nv += len(verts)

    def build(self, name, mats, params, n_steps, meta=None):
        x = np.concatenate(self.verts).astype(np.float64)
        tets = np.concatenate(self.tets).astype(np.int32) if self.tets else np.zeros((0, 4), np.int32)
        tm = np.concatenate(self.mat) if self.mat else np.zeros(0, np.int32)
        tris = np.concatenate(self.tris).astype(np.int32) if self.tris else np.zeros((0, 3), np.int32)
        return Scene(name=name, rest=x.copy(), x0=x.copy(), v0=np.zeros_like(x), tets=tets,
                     tet_mat=tm.astype(np.int32), mats=np.asarray(mats, np.float64).reshape(-1, 3),
                     tris=tris, dirichlet=np.concatenate(self.dir), params=params,
                     n_steps=n_steps, meta=meta or {})


def _jittered_cube(rng, cells, side, origin, yaw=0.0, jitter=1e-4):
    v, t = cube_mesh(cells, side)
    v = v + rng.uniform(-jitter, jitter, size=v.shape)
    if yaw != 0.0:
        c, s = math.cos(yaw), math.sin(yaw)
        ctr = np.array([side / 2, side / 2, 0.0])
        r = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
        v = (v - ctr) @ r.T + ctr
    return v + np.asarray(origin, dtype=np.float64), t


def two_cubes(seed: int = 0, cells: int = 4, side: float = 0.1, precision: int = 0) -> Scene:
    """Two jittered cubes (4^3 cells, 384 tets, 125 verts each), the upper one
    1 mm above the lower, falling onto a static 2 m x 2 m ground quad at z = 0;
    20 steps, FP64."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    z0 = 0.01
    for k in range(2):
        v, t = _jittered_cube(rng, cells, side, (-side / 2, -side / 2, z0 + k * (side + 1e-3)))
        b.add_solid(v, t, 0)
    gv, gt = ground_quad(1.0)
    b.add_obstacle(gv, gt)
    return b.build(f"two_cubes_{cells}^3_seed{seed}", [[1e5, 0.4, 1000.0]],
                   Params(precision=precision), 20, {"seed": seed, "cells": cells})


def slope_cube(mu_f: float, theta: float = math.atan(0.5), cells: int = 2, side: float = 0.1, E: float = 1e6,
               precision: int = 0, n_steps: int = 40, eps_v: float = 1e-3) -> Scene:
    """A cube (side 0.1 m, cells^3 cells) resting on an incline of angle theta
    (the paper's sliding-friction test: tan theta = 0.5, friction coefficients
    around 0.5).  The incline is the static quad z = 0 (4 m x 4 m) and gravity
    is tilted instead, g = 9.8 (-sin theta, 0, -cos theta): the cube slides
    along -x when mu_f < tan theta, at g (sin theta - mu_f cos theta).  Its
    bottom starts 1.2 delta above the plane, at rest; k_min = 6 (the paper's
    setting with friction); E = 1e6 Pa, nu = 0.3, rho = 1000.  The quad is
    offset so that its diagonal stays clear of the cube's path: pairs with
    the second triangle would enter the active set only once the step's CCD
    catches a vertex (Alg. 3), after a transient sinking."""
    b = _Builder()
    p = Params(precision=precision, mu_f=mu_f, eps_v=eps_v, k_min=6,
               gravity=(-9.8 * math.sin(theta), 0.0, -9.8 * math.cos(theta)))
    v, t = cube_mesh(cells, side)
    b.add_solid(v + np.array([-side / 2, -side / 2, 1.2 * p.delta]), t, 0)
    gv, gt = ground_quad(2.0, center=(0.0, 1.5))  # the quad's diagonal stays clear of the cube's path
    b.add_obstacle(gv, gt)
    return b.build(f"slope_cube_{cells}^3_mu{mu_f:g}", [[E, 0.3, 1000.0]], p, n_steps,
                   {"mu_f": mu_f, "theta": theta, "cells": cells})


def eight_cubes(seed: int = 0, cells: int = 16, side: float = 0.1, precision: int = 1) -> Scene:
    """Eight jittered cubes (16^3 cells: 24,576 tets / 4,913 verts each) in a
    2x2x2 layout with seeded yaw and offsets, dropped into a static open box
    (0.6 x 0.6 m floor, 0.6 m walls); 50 steps, mixed precision."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    spacing = 0.17
    for layer, zbase in enumerate((0.06, 0.20)):
        for iy in range(2):
            for ix in range(2):
                cx = (ix - 0.5) * spacing + rng.uniform(-0.01, 0.01)
                cy = (iy - 0.5) * spacing + rng.uniform(-0.01, 0.01)
                yaw = rng.uniform(0.0, 2 * math.pi)
                z = zbase + rng.uniform(0.0, 0.02)
                v, t = _jittered_cube(rng, cells, side, (cx - side / 2, cy - side / 2, z), yaw)
                b.add_solid(v, t, 0)
    bv, bt = open_box(0.3, 0.6)
    b.add_obstacle(bv, bt)
    return b.build(f"eight_cubes_{cells}^3_seed{seed}", [[1e5, 0.4, 1000.0]],
                   Params(precision=precision), 50, {"seed": seed, "cells": cells})


def batch_scene(seed: int, t_lo: float = 1e3, t_hi: float = 2e4, precision: int = 1, side: float = 0.1) -> Scene:
    """One scene of a batch of independent scenes of uneven size: target
    tet count T ~ log-uniform [t_lo, t_hi], a single cube or a stack of two
    (probability 1/2 each), n = max(2, round((T / (6 k))^(1/3))) cells per
    cube edge (k cubes), E ~ log-uniform [1e4, 1e6] Pa, nu ~ U(0.3, 0.45),
    rho = 1000 kg/m^3; cubes of side 0.1 m centred at a seeded xy position
    U(-0.3, 0.3)^2 with a seeded yaw U(0, 2 pi), the lower one 1 cm above a
    static 2 m x 2 m ground quad, the upper one 1 mm above it; h = 0.01 s,
    10 steps."""
    rng = np.random.default_rng(seed)
    target = math.exp(rng.uniform(math.log(t_lo), math.log(t_hi)))
    k = 1 + int(rng.random() < 0.5)
    cells = max(2, int(round((target / (6 * k)) ** (1.0 / 3.0))))
    E = math.exp(rng.uniform(math.log(1e4), math.log(1e6)))
    nu = rng.uniform(0.3, 0.45)
    cx, cy = rng.uniform(-0.3, 0.3, size=2)
    yaw = rng.uniform(0.0, 2 * math.pi)
    b = _Builder()
    for j in range(k):
        v, t = _jittered_cube(rng, cells, side, (cx - side / 2, cy - side / 2, 0.01 + j * (side + 1e-3)), yaw)
        b.add_solid(v, t, 0)
    gv, gt = ground_quad(1.0)
    b.add_obstacle(gv, gt)
    return b.build(f"batch_{seed}_{k}x{cells}^3", [[E, nu, 1000.0]], Params(precision=precision), 10,
                   {"seed": seed, "cells": cells, "cubes": k, "E": E, "nu": nu, "target_tets": target})


def batch_scene_size(seed: int, t_lo: float = 1e3, t_hi: float = 2e4) -> int:
    """tet count of batch_scene(seed, t_lo, t_hi) without building it (the
    same seeded draws)"""
    rng = np.random.default_rng(seed)
    target = math.exp(rng.uniform(math.log(t_lo), math.log(t_hi)))
    k = 1 + int(rng.random() < 0.5)
    cells = max(2, int(round((target / (6 * k)) ** (1.0 / 3.0))))
    return 6 * k * cells ** 3


def single_cube(seed: int = 0, cells: int = 2, side: float = 0.1, z: float = 0.5,
                v0=(0.0, 0.0, 0.0), with_ground: bool = False, gravity=(0.0, 0.0, -9.8),
                xy=(0.0, 0.0)) -> Scene:
    """One jittered cube, optionally above a ground quad (small test scene)."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    v, t = _jittered_cube(rng, cells, side, (xy[0] - side / 2, xy[1] - side / 2, z))
    b.add_solid(v, t, 0)
    if with_ground:
        gv, gt = ground_quad(1.0)
        b.add_obstacle(gv, gt)
    s = b.build(f"single_cube_{cells}^3_seed{seed}", [[1e5, 0.4, 1000.0]],
                Params(gravity=tuple(gravity)), 10, {"seed": seed})
    s.v0[:] = 0.0
    s.v0[s.dirichlet == 0] = np.asarray(v0, dtype=np.float64)
    return s


def colliding_cubes(seed: int = 0, cells: int = 2, side: float = 0.1, gap: float = 0.004,
                    speed: float = 1.0) -> Scene:
    """Two cubes approaching each other along x with no gravity and no
    obstacles (momentum-conservation test scene)."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    v, t = _jittered_cube(rng, cells, side, (-side - gap / 2, -side / 2, 0.0))
    b.add_solid(v, t, 0)
    v2, t2 = _jittered_cube(rng, cells, side, (gap / 2, -side / 2 + 0.02, 0.01))
    b.add_solid(v2, t2, 0)
    s = b.build(f"colliding_cubes_{cells}^3_seed{seed}", [[1e5, 0.4, 1000.0]],
                Params(gravity=(0.0, 0.0, 0.0)), 10, {"seed": seed})
    n1 = len(v)
    s.v0[:n1, 0] = speed
    return s


def ball_mesh(cells: int, radius: float):
    """A ball of `radius` centred at the origin: the Kuhn grid of a cube
    [-r, r]^3 with `cells` cells per side, each vertex p moved to
    p |p|_inf / |p|_2 (the cube's shells become spheres), so the surface is
    a curved polyhedron without flat faces."""
    v, t = cube_mesh(cells, 2.0 * radius)
    v = v - radius
    n2 = np.linalg.norm(v, axis=1)
    ninf = np.abs(v).max(axis=1)
    scale = np.where(n2 > 0, ninf / np.where(n2 > 0, n2, 1.0), 1.0)
    v = v * scale[:, None]
    d = v[t[:, 1:]] - v[t[:, :1]]
    assert np.linalg.det(d).min() > 0, "ball mesh has inverted tets"
    return v, t


def colliding_balls(seed: int = 0, cells: int = 6, radius: float = 0.05, gap: float = 0.004,
                    speed: float = 1.0, offset: float = 0.02, E: float = 1e5) -> Scene:
    """Two balls, no gravity and no obstacles: the left one moves along +x at
    `speed` toward the right one at rest, their centres `offset` apart in y
    (an oblique hit: they collide and separate).  Seeded jitter of 1e-4 x
    the radius on every vertex, rest shape included."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    v, t = ball_mesh(cells, radius)
    j = 1e-4 * radius
    v1 = v + rng.uniform(-j, j, size=v.shape) + np.array([-radius - gap / 2, 0.0, 0.0])
    v2 = v + rng.uniform(-j, j, size=v.shape) + np.array([radius + gap / 2, offset, 0.0])
    b.add_solid(v1, t, 0)
    b.add_solid(v2, t, 0)
    s = b.build(f"colliding_balls_{cells}_seed{seed}", [[E, 0.4, 1000.0]],
                Params(gravity=(0.0, 0.0, 0.0)), 10, {"seed": seed})
    s.v0[: len(v1), 0] = speed
    return s


def moving_plate(seed: int = 0, cells: int = 3, side: float = 0.1, speed: float = 0.5) -> Scene:
    """A cube resting near a ground quad, with a 2-triangle plate above it
    that moves down at `speed` (moving Dirichlet boundary, section 5.3)."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    v, t = _jittered_cube(rng, cells, side, (-side / 2, -side / 2, 0.002))
    b.add_solid(v, t, 0)
    gv, gt = ground_quad(0.3)
    b.add_obstacle(gv, gt)
    pv, pt = ground_quad(0.12, z=side + 0.012)
    pt = pt[:, [0, 2, 1]]
    b.add_obstacle(pv, pt)
    s = b.build(f"moving_plate_{cells}^3_seed{seed}", [[1e5, 0.4, 1000.0]], Params(), 10,
                {"seed": seed, "plate_speed": speed})
    s.meta["plate_vertices"] = np.arange(s.nv - 4, s.nv)
    return s


def plate_targets(scene: Scene, step: int) -> np.ndarray:
    """Prescribed obstacle positions at the end of step `step` (0-based) for
    moving_plate scenes: the plate moves along -z at constant speed."""
    x = scene.x0.copy()
    ids = scene.meta["plate_vertices"]
    x[ids, 2] -= scene.meta["plate_speed"] * scene.params.dt * (step + 1)
    return x[scene.dirichlet == 1]


def _fibonacci_dirs(n: int, rng) -> np.ndarray:
    """n roughly uniform unit directions (Fibonacci sphere), jittered"""
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    r = np.sqrt(1.0 - z * z)
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1) + rng.normal(0.0, 0.08, size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _grid_kuhn_mesh(inside, cell: float, origin):
    """Tets of the grid cells whose centre is inside (boolean array over
    cells, indexed [i, j, k] along x, y, z), keeping the largest face-
    connected group of cells; Kuhn split with one diagonal for every cell.
    Returns (vertices, tets) with unused grid vertices dropped."""
    from scipy import ndimage
    lab, n = ndimage.label(inside)
    if n > 1:
        sizes = ndimage.sum(inside, lab, index=np.arange(1, n + 1))
        inside = lab == 1 + int(np.argmax(sizes))
    ci, cj, ck = np.nonzero(inside)
    nx, ny, nz = (np.array(inside.shape) + 1)
    vid = lambda i, j, k: (i * ny + j) * nz + k
    corners = []
    for c in range(8):
        corners.append(vid(ci + (c & 1), cj + ((c >> 1) & 1), ck + ((c >> 2) & 1)))
    corners = np.stack(corners, axis=1)  # (ncell, 8)
    tets = corners[:, _KUHN].reshape(-1, 4)
    used, tets = np.unique(tets, return_inverse=True)
    tets = tets.reshape(-1, 4).astype(np.int32)
    i = used // (ny * nz)
    j = (used // nz) % ny
    k = used % nz
    verts = np.stack([i, j, k], axis=1) * cell + np.asarray(origin, dtype=np.float64)
    d = verts[tets[:, 1:]] - verts[tets[:, :1]]
    neg = np.linalg.det(d) < 0
    tets[neg] = tets[neg][:, [0, 2, 1, 3]]
    return verts, tets


def spiky_ball(rng, center, radius=0.1, n_spikes=64, l_lo=0.02, l_hi=0.05, base=0.012, cell=0.0038):
    """A ball with conical spikes, tetrahedralised on a regular grid: the
    solid is the sphere of `radius` united with n_spikes cones (directions
    from a jittered Fibonacci sphere, lengths U(l_lo, l_hi), base radius
    `base` at the sphere, apex at radius + length); the grid cells (size
    `cell`) whose centres are inside are kept (largest connected group),
    each split into 6 tets."""
    dirs = _fibonacci_dirs(n_spikes, rng)
    lens = rng.uniform(l_lo, l_hi, size=n_spikes)
    ext = radius + l_hi
    n = int(math.ceil(2 * ext / cell))
    g = (np.arange(n) + 0.5) * cell - n * cell / 2
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    inside = (P * P).sum(1) <= radius * radius
    for d, L in zip(dirs, lens):
        t = P @ d
        rho2 = (P * P).sum(1) - t * t
        cand = (t >= radius - base) & (t <= radius + L)
        rr = base * np.clip((radius + L - t) / L, 0.0, None)
        inside |= cand & (rho2 <= rr * rr)
    inside = inside.reshape(n, n, n)
    org = np.asarray(center, dtype=np.float64) - n * cell / 2
    v, t = _grid_kuhn_mesh(inside, cell, org)
    return v + rng.uniform(-0.02 * cell, 0.02 * cell, size=v.shape), t  # no exactly parallel edges


def spiky_balls(seed: int = 0, cell: float = 0.0039, precision: int = 1, n_steps: int = 60) -> Scene:
    """Five spiky balls (radius 0.1 m, 64 spikes of 0.02-0.05 m) in a
    0.7 x 0.7 m open box, four on the floor in a 2 x 2 grid and one on top,
    compressed by a plate that starts 0.02 m above the top ball and moves
    down at 0.5 m/s to 30 % of its initial height, then back up at 0.5 m/s;
    E = 5e4 Pa, nu = 0.45, rho = 1000 kg/m^3, h = 1/60 s.  With the default
    cell of 3.9 mm each ball has about 4.6e5 tets; vertices are jittered by
    up to 2 % of a cell (rest shape too)."""
    rng = np.random.default_rng(seed)
    ext = 0.1 + 0.05
    b = _Builder()
    gap = 0.004
    centres = [(sx * (ext + gap), sy * (ext + gap), ext + gap) for sx in (-1, 1) for sy in (-1, 1)]
    centres.append((0.0, 0.0, ext + gap + 2 * ext + gap))
    for c in centres:
        v, t = spiky_ball(rng, c, cell=cell)
        b.add_solid(v, t, 0)
    half = 2 * (ext + gap) + 0.02
    bv, bt = open_box(half, 0.9)
    b.add_obstacle(bv, bt)
    z0 = centres[-1][2] + ext + 0.02
    pv, pt = ground_quad(half - 0.005, z=z0)
    b.add_obstacle(pv, pt[:, [0, 2, 1]])
    s = b.build(f"spiky_balls_seed{seed}", [[5e4, 0.45, 1000.0]], Params(dt=1.0 / 60.0, precision=precision),
                n_steps, {"seed": seed, "cell": cell, "plate_speed": 0.5, "plate_z0": z0,
                          "plate_z_min": 0.3 * z0})
    s.meta["plate_vertices"] = np.arange(s.nv - 4, s.nv)
    return s


def plate_schedule_z(scene: Scene, step: int) -> float:
    """plate height at the end of step `step` (0-based) for spiky_balls:
    down at plate_speed to plate_z_min, then back up at the same speed"""
    z0, zmin, v, h = scene.meta["plate_z0"], scene.meta["plate_z_min"], scene.meta["plate_speed"], scene.params.dt
    t = (step + 1) * h
    t_down = (z0 - zmin) / v
    return z0 - v * t if t <= t_down else min(z0, zmin + v * (t - t_down))


def plate_targets_schedule(scene: Scene, step: int) -> np.ndarray:
    """Prescribed obstacle positions at the end of step `step` for
    spiky_balls (the plate follows plate_schedule_z)"""
    x = scene.x0.copy()
    ids = scene.meta["plate_vertices"]
    x[ids, 2] = plate_schedule_z(scene, step)
    return x[scene.dirichlet == 1]


CONFIGS = {
    "two_cubes": two_cubes,
    "eight_cubes": eight_cubes,
}
