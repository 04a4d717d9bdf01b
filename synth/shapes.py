"""Synthetic solids for the workloads: oriented boundary samples and query points.

Every function here is seeded and deterministic.  The module holds geometry only:
where boundary samples sit, their unit outward normals and area (2D: length)
weights, and where the query points of a shape's skeletal density function (SDF)
are placed.  It computes nothing of the SDF or of the score; the analytic
distance helpers exist only to keep query points off the boundary and inside a
band, never to stand in for the signed distance of Eq. 10A.

Conventions
-----------
* Positions are float64 arrays of shape (n, d) with d = 2 or 3.
* ``normals`` are unit outward normals of the solid (Section 4: a consistent
  manifold orientation, averaged where two smooth pieces meet).
* ``area`` holds the boundary measure carried by each sample; it sums to the
  boundary's length (2D) or area (3D).
* Query points carry a cell volume ``vol`` (2D: cell area), the weight of the
  sample when the SDF is represented as a weighted point set.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Boundary:
    pos: np.ndarray      # (n_b, d)
    normal: np.ndarray   # (n_b, d) unit outward normals
    area: np.ndarray     # (n_b,)   boundary measure per sample

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def dim(self) -> int:
        return int(self.pos.shape[1])

    @property
    def spacing(self) -> float:
        """Mean sample spacing h_b: |dS|/n_b in 2D, sqrt(|dS|/n_b) in 3D."""
        tot = float(self.area.sum())
        return tot / self.n if self.dim == 2 else math.sqrt(tot / self.n)


@dataclass
class QuerySet:
    pos: np.ndarray      # (m, d)
    vol: np.ndarray      # (m,)
    inside: np.ndarray   # (m,) bool, analytic membership (test aid only)
    info: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.pos.shape[0])


# ---------------------------------------------------------------------------
# 2D polygons (square peg, plate with a square hole)
# ---------------------------------------------------------------------------

def _square_loop(half: float, count: int, hole: bool) -> Boundary:
    """``count`` equally spaced samples on the square [-half, half]^2.

    Samples sit at arclengths (k + 1/2) * P / count from the corner (-half, -half),
    walking counter-clockwise.  A sample that lands on a corner takes the
    normalised mean of the two face normals.  ``hole=True`` flips the normals
    so they point into the hole, i.e. out of the surrounding solid.
    """
    side = 2.0 * half
    perim = 4.0 * side
    ds = perim / count
    s = (np.arange(count) + 0.5) * ds
    corners = np.array([[-half, -half], [half, -half], [half, half], [-half, half]])
    face_n = np.array([[0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])
    pos = np.zeros((count, 2))
    nrm = np.zeros((count, 2))
    for i, si in enumerate(s):
        f = min(int(si // side), 3)
        u = si - f * side
        a, b = corners[f], corners[(f + 1) % 4]
        pos[i] = a + (b - a) * (u / side)
        tol = 1e-12 * side
        if abs(u) < tol:
            v = face_n[f] + face_n[(f - 1) % 4]
        elif abs(u - side) < tol:
            v = face_n[f] + face_n[(f + 1) % 4]
        else:
            v = face_n[f]
        nrm[i] = v / np.linalg.norm(v)
    if hole:
        nrm = -nrm
    return Boundary(pos, nrm, np.full(count, ds))


def square_peg_boundary(side: float = 1.0, n_b: int = 512) -> Boundary:
    return _square_loop(side / 2.0, n_b, hole=False)


def plate_with_hole_boundary(outer: float = 4.0, hole: float = 1.05, n_b: int = 512) -> Boundary:
    """Outer square and a centred square hole share ``n_b`` samples in proportion to length."""
    p_out, p_in = 4.0 * outer, 4.0 * hole
    n_out = int(round(n_b * p_out / (p_out + p_in)))
    n_in = n_b - n_out
    a = _square_loop(outer / 2.0, n_out, hole=False)
    b = _square_loop(hole / 2.0, n_in, hole=True)
    return Boundary(np.vstack([a.pos, b.pos]), np.vstack([a.normal, b.normal]),
                    np.concatenate([a.area, b.area]))


def sd_square(p: np.ndarray, half: float) -> np.ndarray:
    """Exact signed distance to the square [-half, half]^2 (negative inside)."""
    q = np.abs(p) - half
    out = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
    ins = np.minimum(np.max(q, axis=-1), 0.0)
    return out + ins


def sd_plate(p: np.ndarray, outer: float = 4.0, hole: float = 1.05) -> np.ndarray:
    return np.maximum(sd_square(p, outer / 2.0), -sd_square(p, hole / 2.0))


# ---------------------------------------------------------------------------
# 3D: cylinder peg and block with a blind bore
# ---------------------------------------------------------------------------

def _disc(rng, cnt, r, z, nz):
    rr = r * np.sqrt(rng.random(cnt))
    th = 2 * np.pi * rng.random(cnt)
    pos = np.stack([rr * np.cos(th), rr * np.sin(th), np.full(cnt, z)], 1)
    nrm = np.tile([0.0, 0.0, nz], (cnt, 1))
    return pos, nrm


def cylinder_boundary(radius=1.0, length=3.0, n_b=20000, seed=1) -> Boundary:
    """Area-uniform random samples on a closed cylinder (axis z, centred at 0)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 1]))
    a_side = 2 * np.pi * radius * length
    a_cap = np.pi * radius ** 2
    tot = a_side + 2 * a_cap
    face = rng.choice(3, size=n_b, p=[a_side / tot, a_cap / tot, a_cap / tot])
    pos = np.zeros((n_b, 3))
    nrm = np.zeros((n_b, 3))
    m = face == 0
    th = 2 * np.pi * rng.random(m.sum())
    z = length * (rng.random(m.sum()) - 0.5)
    pos[m] = np.stack([radius * np.cos(th), radius * np.sin(th), z], 1)
    nrm[m] = np.stack([np.cos(th), np.sin(th), np.zeros_like(th)], 1)
    for f, zc, nz in ((1, length / 2, 1.0), (2, -length / 2, -1.0)):
        m = face == f
        pos[m], nrm[m] = _disc(rng, m.sum(), radius, zc, nz)
    return Boundary(pos, nrm, np.full(n_b, tot / n_b))


def sd_cylinder(p, radius=1.0, length=3.0):
    """Exact signed distance to a closed finite cylinder (axis z, centred)."""
    dr = np.hypot(p[..., 0], p[..., 1]) - radius
    dz = np.abs(p[..., 2]) - length / 2
    out = np.hypot(np.maximum(dr, 0), np.maximum(dz, 0))
    return out + np.minimum(np.maximum(dr, dz), 0.0)


def block_with_bore_boundary(size=(6.0, 6.0, 4.0), bore_r=1.02, bore_depth=2.5,
                             n_b=20000, seed=1) -> Boundary:
    """Area-uniform samples on a centred box with a blind cylindrical bore.

    The bore has axis z, opens on the top face z = +size_z/2 and ends at depth
    ``bore_depth``.  Its wall normals point at the bore axis and its floor normal
    points up (+z): both point out of the solid.
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 2]))
    hx, hy, hz = (s / 2 for s in size)
    z_floor = hz - bore_depth
    a_top = 4 * hx * hy - np.pi * bore_r ** 2
    a_bot = 4 * hx * hy
    a_sx = 4 * hy * hz      # each of the two x faces
    a_sy = 4 * hx * hz
    a_wall = 2 * np.pi * bore_r * bore_depth
    a_floor = np.pi * bore_r ** 2
    areas = np.array([a_top, a_bot, a_sx, a_sx, a_sy, a_sy, a_wall, a_floor])
    tot = areas.sum()
    face = rng.choice(8, size=n_b, p=areas / tot)
    pos = np.zeros((n_b, 3))
    nrm = np.zeros((n_b, 3))
    # top: uniform on the square, outside the bore disc (rejection)
    m = np.flatnonzero(face == 0)
    pts = []
    while sum(len(x) for x in pts) < len(m):
        c = np.stack([hx * (2 * rng.random(len(m)) - 1), hy * (2 * rng.random(len(m)) - 1)], 1)
        pts.append(c[np.hypot(c[:, 0], c[:, 1]) > bore_r])
    c = np.vstack(pts)[: len(m)]
    pos[m] = np.column_stack([c, np.full(len(m), hz)])
    nrm[m] = [0, 0, 1]
    m = np.flatnonzero(face == 1)
    pos[m] = np.column_stack([hx * (2 * rng.random(len(m)) - 1), hy * (2 * rng.random(len(m)) - 1),
                              np.full(len(m), -hz)])
    nrm[m] = [0, 0, -1]
    for f, sgn in ((2, 1.0), (3, -1.0)):
        m = np.flatnonzero(face == f)
        pos[m] = np.column_stack([np.full(len(m), sgn * hx), hy * (2 * rng.random(len(m)) - 1),
                                  hz * (2 * rng.random(len(m)) - 1)])
        nrm[m] = [sgn, 0, 0]
    for f, sgn in ((4, 1.0), (5, -1.0)):
        m = np.flatnonzero(face == f)
        pos[m] = np.column_stack([hx * (2 * rng.random(len(m)) - 1), np.full(len(m), sgn * hy),
                                  hz * (2 * rng.random(len(m)) - 1)])
        nrm[m] = [0, sgn, 0]
    m = np.flatnonzero(face == 6)
    th = 2 * np.pi * rng.random(len(m))
    z = z_floor + bore_depth * rng.random(len(m))
    pos[m] = np.column_stack([bore_r * np.cos(th), bore_r * np.sin(th), z])
    nrm[m] = np.column_stack([-np.cos(th), -np.sin(th), np.zeros(len(m))])
    m = np.flatnonzero(face == 7)
    pos[m], nrm[m] = _disc(rng, len(m), bore_r, z_floor, 1.0)
    return Boundary(pos, nrm, np.full(n_b, tot / n_b))


def sd_block_with_bore(p, size=(6.0, 6.0, 4.0), bore_r=1.02, bore_depth=2.5):
    """Signed distance bound: exact inside the solid, a lower bound on |d| outside."""
    h = np.array(size) / 2
    q = np.abs(p) - h
    box = np.linalg.norm(np.maximum(q, 0), axis=-1) + np.minimum(q.max(-1), 0)
    # bore region: cylinder r <= bore_r, z in [z_floor, top + 1] (open through the top)
    z_floor = h[2] - bore_depth
    zc = 0.5 * (z_floor + h[2] + 1.0)
    hl = 0.5 * (h[2] + 1.0 - z_floor)
    dr = np.hypot(p[..., 0], p[..., 1]) - bore_r
    dz = np.abs(p[..., 2] - zc) - hl
    bore = np.hypot(np.maximum(dr, 0), np.maximum(dz, 0)) + np.minimum(np.maximum(dr, dz), 0)
    return np.maximum(box, -bore)


# ---------------------------------------------------------------------------
# 3D: unions of spheres placed by a confined self-avoiding walk
# ---------------------------------------------------------------------------

def self_avoiding_walk(n: int, seed: int, step=3.8, min_sep=2.8, conf_scale=3.0,
                       tries=100) -> np.ndarray:
    """Centres of a self-avoiding walk confined to a ball of radius conf_scale * n^(1/3).

    Each step is ``step`` long in a uniformly random direction; non-bonded
    centres stay at least ``min_sep`` apart.  After ``tries`` failed attempts
    the walk backtracks one step.  The returned centres are shifted so their
    mean is the origin.

    Centres are kept in a hash grid of cells wider than step + min_sep, so a
    trial step is compared only with the centres of the 27 cells around the
    previous centre: every other centre is farther than min_sep from any
    point on the step sphere, and the accepted walk is the one an all-pairs
    comparison gives.
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 3, n]))
    rc = conf_scale * n ** (1.0 / 3.0)
    cen = np.zeros((n, 3))
    cell = step + min_sep + 1e-6
    grid: dict = {}

    def key(i):
        return tuple(int(v) for v in np.floor(cen[i] / cell))

    def add(i):
        grid.setdefault(key(i), []).append(i)

    add(0)
    offsets = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
    k = 1
    guard = 0
    while k < n:
        guard += 1
        if guard > 200 * n:
            raise RuntimeError("self-avoiding walk did not converge")
        d = rng.standard_normal((tries, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        cand = cen[k - 1] + step * d
        ok = np.linalg.norm(cand, axis=1) <= rc
        if k >= 2:
            kx, ky, kz = key(k - 1)
            near = [i for a, b, c in offsets for i in grid.get((kx + a, ky + b, kz + c), ()) if i < k - 1]
            if near:
                dd = np.linalg.norm(cand[:, None, :] - cen[None, near, :], axis=2)
                ok &= (dd >= min_sep).all(axis=1)
        idx = np.flatnonzero(ok)
        if len(idx):
            cen[k] = cand[idx[0]]
            add(k)
            k += 1
        else:
            if k >= 2:
                grid[key(k - 1)].remove(k - 1)
            k = max(1, k - 1)
    return cen - cen.mean(0)


@dataclass
class SphereUnion:
    centers: np.ndarray
    radii: np.ndarray


def sphere_union(n: int, seed: int, rmin=1.2, rmax=2.0) -> SphereUnion:
    cen = self_avoiding_walk(n, seed)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 4, n]))
    return SphereUnion(cen, rmin + (rmax - rmin) * rng.random(n))


def sphere_union_boundary(su: SphereUnion, density=2.0, seed=2) -> Boundary:
    """Samples at ``density`` points per unit area on each sphere, radial normals.

    Samples buried inside another sphere are dropped, so what is left samples the
    union's surface; each keeps the area share of its own sphere.  Only spheres
    whose centre lies within the largest radius of a sample can bury it; a k-d
    tree finds them (centres are at least 2.8 apart, so a few neighbours cover
    every such sphere), and the test itself is the exact distance comparison.
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 5, len(su.radii)]))
    pos, nrm, area = [], [], []
    for c, r in zip(su.centers, su.radii):
        a = 4 * np.pi * r * r
        cnt = max(4, int(round(density * a)))
        v = rng.standard_normal((cnt, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        pos.append(c + r * v)
        nrm.append(v)
        area.append(np.full(cnt, a / cnt))
    pos = np.vstack(pos)
    nrm = np.vstack(nrm)
    area = np.concatenate(area)
    keep = np.ones(len(pos), bool)
    rmax = float(su.radii.max())
    ns = len(su.radii)
    try:
        from scipy.spatial import cKDTree
    except ImportError:  # pragma: no cover - scipy is present on both machines
        cKDTree = None
    if cKDTree is not None and ns > 16:
        tree = cKDTree(su.centers)
        _, nb = tree.query(pos, k=16, distance_upper_bound=rmax * (1 + 1e-9) + 1e-9)
        # a full row of 16 neighbours would mean more may exist: fall back for those
        full = nb[:, -1] < ns
        for s in range(0, len(pos), 65536):
            sl = slice(s, s + 65536)
            j = np.where(nb[sl] < ns, nb[sl], 0)
            d = np.linalg.norm(pos[sl, None, :] - su.centers[j], axis=2) - su.radii[j]
            keep[sl] = np.where(nb[sl] < ns, d >= -1e-6, True).all(axis=1)
        for i in np.flatnonzero(full):
            d = np.linalg.norm(pos[i, None, :] - su.centers, axis=1) - su.radii
            keep[i] = (d >= -1e-6).all()
    else:
        for s in range(0, len(pos), 4096):
            d = np.linalg.norm(pos[s:s + 4096, None, :] - su.centers[None], axis=2) - su.radii[None]
            keep[s:s + 4096] = (d >= -1e-6).all(axis=1)
    return Boundary(pos[keep], nrm[keep], area[keep])


def sd_sphere_union(p, su: SphereUnion, chunk=2048):
    """min_k(|p - c_k| - r_k): exact outside the union, |d| underestimated inside."""
    out = np.empty(p.shape[0])
    for s in range(0, len(p), chunk):
        d = np.linalg.norm(p[s:s + chunk, None, :] - su.centers[None], axis=2) - su.radii[None]
        out[s:s + chunk] = d.min(axis=1)
    return out


# ---------------------------------------------------------------------------
# Query points: jittered grids, kept in a band around the boundary
# ---------------------------------------------------------------------------

def jittered_grid(lo, hi, cell, seed) -> np.ndarray:
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    cnt = np.maximum(1, np.floor((hi - lo) / cell + 1e-9).astype(int))
    axes = [lo[i] + cell * np.arange(cnt[i]) for i in range(len(lo))]
    g = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, len(lo))
    rng = np.random.default_rng(np.random.SeedSequence([seed, 6]))
    return g + cell * rng.random(g.shape)


def query_points(sdist, lo, hi, cell, h_b, band=None, seed=0) -> QuerySet:
    """Jittered grid over [lo, hi], dropping points with |d| < h_b or |d| > band.

    ``sdist`` is the analytic signed distance of the solid (negative inside).
    The h_b rule keeps the discrete sums of Eq. 13 away from the single-sample
    singularity at the boundary; ``band`` optionally limits the samples to a
    shell around the boundary.
    """
    p = jittered_grid(lo, hi, cell, seed)
    d = sdist(p)
    keep = np.abs(d) >= h_b
    if band is not None:
        keep &= np.abs(d) <= band
    p = p[keep]
    d = d[keep]
    dim = p.shape[1]
    return QuerySet(p, np.full(len(p), cell ** dim), d < 0,
                    {"cell": cell, "h_b": h_b, "band": band, "grid_count": int(keep.size)})


def query_points_target(sdist, lo, hi, target, h_b, band, seed, iters=6) -> QuerySet:
    """Tune the jittered-grid cell so that about ``target`` points are kept."""
    dim = len(lo)
    vol = float(np.prod(np.asarray(hi) - np.asarray(lo)))
    cell = (vol / target) ** (1.0 / dim)
    qs = query_points(sdist, lo, hi, cell, h_b, band, seed)
    for _ in range(iters):
        if qs.m == 0:
            cell *= 0.5
        else:
            cell *= (qs.m / target) ** (1.0 / dim)
        qs = query_points(sdist, lo, hi, cell, h_b, band, seed)
        if abs(qs.m - target) <= 0.02 * target:
            break
    return qs
