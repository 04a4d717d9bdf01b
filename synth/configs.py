"""Seeded synthetic workloads sized like the paper's 2D, mechanical and docking cases.

Each builder returns a :class:`Workload`: two solids (fixed S1, moving S2), each
as oriented boundary samples plus the query points where its SDF is sampled,
the translation grid (N points per axis over a periodic box of side L), the
rotation set and the SDF parameters.  The paper's own shapes (Section 6 figures,
PDB 1A2K) are not available, so these stand in for them:

* ``peg_in_hole_2d``   - square peg (side 1) and a 4x4 plate with a 1.05 hole,
  512 boundary samples each, 64x64 jittered query cells, 128^2 grid,
  64 planar rotations, FP64.
* ``peg_in_bore_3d``   - cylinder (r=1, length 3) and a 6x6x4 block with a blind
  bore (r=1.02, depth 2.5), 20,000 boundary samples each, ~50,000 query points
  each in a 0.3 band, 128^3 grid, 576 Hopf rotations, top-10.
* ``docking_pair``     - unions of 2,000 and 500 spheres (radii U[1.2, 2.0]),
  surface at 2 samples per unit area, ~40 query points per sphere, 192^3 grid at
  spacing 0.8, 54,000 super-Fibonacci rotations, top-100.
* ``tiny_2d`` / ``tiny_3d`` - reduced versions for exhaustive checks.

SDF parameters default to the values of the paper's validation (Section 6):
lambda1 = 1, lambda2 = 3, sigma = 0.5, eps = 1.5.
"""

from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field

import numpy as np

from . import rotations as rot
from . import shapes as sh


@dataclass
class ShapeInput:
    name: str
    boundary: sh.Boundary
    query: sh.QuerySet


@dataclass
class Workload:
    name: str
    dim: int
    fixed: ShapeInput
    moving: ShapeInput
    N: int
    L: float
    sigma_g: float
    quats: np.ndarray
    top_k: int = 1
    precision: str = "f32"
    lam1: float = 1.0
    lam2: float = 3.0
    sigma_t: float = 0.5
    eps: float = 1.5
    alpha: int = 2
    w: int = 6
    extra: dict = field(default_factory=dict)

    @property
    def h(self) -> float:
        return self.L / self.N

    @property
    def n_rot(self) -> int:
        return int(self.quats.shape[0])

    def sdf_params(self) -> dict:
        return dict(lam1=self.lam1, lam2=self.lam2, sigma_t=self.sigma_t, eps=self.eps)


# ---------------------------------------------------------------------------

def _peg_hole_shapes(n_b, cells, seed, side=1.0, hole=1.05):
    peg_b = sh.square_peg_boundary(side, n_b)
    plate_b = sh.plate_with_hole_boundary(4.0, hole, n_b)
    m = 0.3
    hp = side / 2 + m
    peg_q = sh.query_points(lambda p: sh.sd_square(p, side / 2), [-hp, -hp], [hp, hp],
                            2 * hp / cells, peg_b.spacing, None, seed)
    plate_q = sh.query_points(lambda p: sh.sd_plate(p, 4.0, hole), [-2.3, -2.3], [2.3, 2.3],
                              4.6 / cells, plate_b.spacing, None, seed + 1000)
    return ShapeInput("plate", plate_b, plate_q), ShapeInput("peg", peg_b, peg_q)


@functools.lru_cache(maxsize=None)
def peg_in_hole_2d(n_rot: int = 64, peg_side: float = 1.0) -> Workload:
    fixed, moving = _peg_hole_shapes(512, 64, 0, side=peg_side)
    return Workload("peg_in_hole_2d", 2, fixed, moving, N=128, L=6.6, sigma_g=0.02,
                    quats=rot.planar(n_rot), top_k=1, precision="f64")


@functools.lru_cache(maxsize=None)
def tiny_2d(N: int = 32, n_rot: int = 16) -> Workload:
    fixed, moving = _peg_hole_shapes(128, 24, 10)
    return Workload("tiny_2d", 2, fixed, moving, N=N, L=6.6, sigma_g=0.12,
                    quats=rot.planar(n_rot), top_k=1, precision="f64")


def _peg_bore_shapes(n_b, target, seed, band=0.3):
    cyl_b = sh.cylinder_boundary(1.0, 3.0, n_b, seed)
    blk_b = sh.block_with_bore_boundary((6.0, 6.0, 4.0), 1.02, 2.5, n_b, seed)
    m = 0.3
    cyl_q = sh.query_points_target(lambda p: sh.sd_cylinder(p, 1.0, 3.0),
                                   [-1 - m, -1 - m, -1.5 - m], [1 + m, 1 + m, 1.5 + m],
                                   target, cyl_b.spacing, band, seed)
    blk_q = sh.query_points_target(lambda p: sh.sd_block_with_bore(p),
                                   [-3 - m, -3 - m, -2 - m], [3 + m, 3 + m, 2 + m],
                                   target, blk_b.spacing, band, seed + 1000)
    return ShapeInput("block_with_bore", blk_b, blk_q), ShapeInput("cylinder", cyl_b, cyl_q)


@functools.lru_cache(maxsize=None)
def peg_in_bore_3d() -> Workload:
    fixed, moving = _peg_bore_shapes(20000, 50000, 1)
    return Workload("peg_in_bore_3d", 3, fixed, moving, N=128, L=10.9, sigma_g=0.03,
                    quats=rot.hopf_grid(2, 12), top_k=10, precision="f32")


@functools.lru_cache(maxsize=None)
def tiny_3d(N: int = 32, n_rot: int = 12) -> Workload:
    fixed, moving = _peg_bore_shapes(3000, 1500, 11, band=0.5)
    q = rot.super_fibonacci(n_rot)
    q[0] = [1.0, 0.0, 0.0, 0.0]
    return Workload("tiny_3d", 3, fixed, moving, N=N, L=10.9, sigma_g=0.25,
                    quats=q, top_k=3, precision="f32")


# ---------------------------------------------------------------------------

def _sphere_shape(name, n_spheres, seed, per_sphere=40, band=2.0, density=2.0):
    su = sh.sphere_union(n_spheres, seed)
    b = sh.sphere_union_boundary(su, density, seed)
    try:
        from scipy.spatial import cKDTree
        tree = cKDTree(su.centers)
        kq = min(16, n_spheres)
        # Spheres farther than band + max radius cannot decide a kept point
        # (|d| <= band); points with none nearer get d = inf and are dropped.
        bound = band + float(su.radii.max())
        radii = np.append(su.radii, 0.0)

        def sdist(p):
            d, i = tree.query(p, k=kq, distance_upper_bound=bound, workers=-1)
            d = np.atleast_2d(d.T).T if kq == 1 else d
            i = np.atleast_2d(i.T).T if kq == 1 else i
            return (d - radii[i]).min(axis=1)
    except ImportError:  # pragma: no cover - scipy is present on both machines
        def sdist(p):
            return sh.sd_sphere_union(p, su)
    lo = su.centers.min(0) - su.radii.max() - band
    hi = su.centers.max(0) + su.radii.max() + band
    q = sh.query_points_target(sdist, lo, hi, per_sphere * n_spheres, b.spacing, band, seed + 77)
    s = ShapeInput(name, b, q)
    s.query.info["spheres"] = su
    return s


@functools.lru_cache(maxsize=None)
def large_sphere_shape(n_spheres: int = 5000, seed: int = 4) -> ShapeInput:
    """One shape at the top of the uneven batch's size range (5,000 spheres:
    ~2e5 SDF samples against ~2e5 boundary samples), built by the same rules."""
    return _sphere_shape(f"spheres{n_spheres}", n_spheres, seed * 1000 + 999)


@functools.lru_cache(maxsize=None)
def docking_pair(n_rec: int = 2000, n_lig: int = 500, seed: int = 2) -> tuple[ShapeInput, ShapeInput]:
    return _sphere_shape("receptor", n_rec, seed), _sphere_shape("ligand", n_lig, seed)


@functools.lru_cache(maxsize=None)
def docking_2000_500(n_rot: int = 54000) -> Workload:
    fixed, moving = docking_pair()
    return Workload("docking_2000_500", 3, fixed, moving, N=192, L=153.6, sigma_g=0.6,
                    quats=rot.super_fibonacci(n_rot), top_k=100, precision="f32",
                    extra={"rot_per_launch": 3000})


@functools.lru_cache(maxsize=None)
def refine_poses_256(n_pose: int = 256):
    """Starting poses for gradient refinement on the docking pair: random rotations,
    translations uniform in a ball of radius 10 around the receptor centre (the origin)."""
    return rot.random_uniform(n_pose, 3), rot.random_ball(n_pose, 10.0, 3)


def grid_for_pair(fixed: ShapeInput, moving: ShapeInput, choices=(64, 96, 128, 192, 256),
                  hmax=0.8, pad=2.0):
    """Box side L >= D1 + D2 (plus ``pad``) and the smallest N with L/N <= hmax."""
    r1 = float(np.linalg.norm(fixed.query.pos, axis=1).max())
    r2 = float(np.linalg.norm(moving.query.pos, axis=1).max())
    L = 2 * (r1 + r2) + pad
    for N in choices:
        if L / N <= hmax:
            return N, L
    return choices[-1], L


def uneven_batch(n_pairs: int = 64, seed: int = 4, n_rot: int = 3000):
    """Pairs with sphere counts log-uniform in [50, 5000] (receptor and ligand drawn independently)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 9]))
    counts = np.exp(rng.uniform(math.log(50), math.log(5000), (n_pairs, 2))).astype(int)
    out = []
    for k, (a, b) in enumerate(counts):
        fx = _sphere_shape(f"rec{k}", int(a), seed * 1000 + 2 * k)
        mv = _sphere_shape(f"lig{k}", int(b), seed * 1000 + 2 * k + 1)
        N, L = grid_for_pair(fx, mv)
        out.append(Workload(f"uneven_{k}", 3, fx, mv, N=N, L=L, sigma_g=0.6,
                            quats=rot.super_fibonacci(n_rot), top_k=1))
    return out
