"""Oracle: adaptive octree (quadtree in 2D) sampling of a solid's SDF (Section 5).

TEST INFRASTRUCTURE.  Plain FP64 NumPy, used only by tests; shares no code with
the library's tree.

Section 5 observes that the skeletal density varies most near the shape's
skeleton, so a uniform grid of SDF samples wastes points where it is flat; it
proposes sampling the SDF on a tree that is subdivided deepest where the
skeletal density is high, and evaluating the score of those nonequispaced
samples with a nonequispaced FFT.  The paper gives no subdivision rule.  The
reading restated here:

* the root is the cube [lo, lo + size]^d, first cut uniformly into 2^d_min
  cells per axis; a cell at depth D has side h = size / 2^D and integer
  coordinates k in [0, 2^D)^d, centre lo + (k + 1/2) h;
* a cell at depth D < d_max is split into its 2^d children when the boundary
  sample nearest its centre lies closer than half the cell's diagonal (the
  cell may cross the boundary, where the SDF is singular), or otherwise when
  its weight |rho(centre)| h^d reaches tau (the cell would carry a large share
  of the density as one sample);
* every cell not split is a leaf with position its centre and volume h^d,
  except that a leaf whose centre lies closer than ``clearance`` to a boundary
  sample is dropped (the same rule that keeps uniform query points off the
  boundary's single-sample singularity);
* optionally the samples are kept to a band around the boundary, like the
  uniform query sets: a leaf whose centre lies farther than ``band`` from the
  boundary is dropped, and a cell whose centre lies farther than ``band`` plus
  half its diagonal (so that all of it lies beyond the band, the distance to
  the boundary being 1-Lipschitz) is dropped without being split or evaluated;
* leaves are listed by depth, then by the linear index
  k_x + 2^D (k_y + 2^D k_z) of their coordinates.

tau = 0 gives the uniform grid at depth d_max; tau = inf gives the tree the
boundary alone forces.
"""

from __future__ import annotations

import math

import numpy as np


def _sorted_level(k, D):
    dim = k.shape[1]
    lin = np.zeros(len(k), np.int64)
    for a in reversed(range(dim)):
        lin = lin * (1 << D) + k[:, a]
    return k[np.argsort(lin, kind="stable")]


def octree_leaves(rho_fn, xi_fn, lo, size, dim, d_min, d_max, tau, clearance, band=np.inf):
    """Leaves of the adaptive tree, level by level.

    ``rho_fn(points) -> complex rho`` and ``xi_fn(points) -> |xi|`` (distance to
    the nearest boundary sample) are evaluated at cell centres.  Returns
    (centres (m, dim), volumes (m,), coords (m, dim) int, depths (m,) int, asked)
    where ``asked`` lists, per level, the centres at which rho was evaluated.
    """
    lo = np.asarray(lo, float)[:dim]
    axes = [np.arange(1 << d_min)] * dim
    k = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, dim).astype(np.int64)
    k = _sorted_level(k, d_min)
    child = np.stack(np.meshgrid(*([np.arange(2)] * dim), indexing="ij"), -1).reshape(-1, dim)
    cen, vol, crd, dep, asked = [], [], [], [], []
    for D in range(d_min, d_max + 1):
        if len(k) == 0:
            break
        h = size / (1 << D)
        c = lo + (k + 0.5) * h
        xi = xi_fn(c)
        half_diag = 0.5 * h * math.sqrt(dim)
        beyond = xi - half_diag > band
        split = np.zeros(len(k), bool)
        if D < d_max:
            split = xi < half_diag
            ask = ~split & ~beyond
            asked.append(c[ask])
            if ask.any():
                split[ask] = np.abs(rho_fn(c[ask])) * h ** dim >= tau
        leaf = ~split & ~beyond & (xi >= clearance) & (xi <= band)
        cen.append(c[leaf])
        vol.append(np.full(int(leaf.sum()), h ** dim))
        crd.append(k[leaf])
        dep.append(np.full(int(leaf.sum()), D))
        k = (2 * k[split][:, None, :] + child[None]).reshape(-1, dim)
        k = _sorted_level(k, D + 1)
    cat = np.concatenate
    return (np.vstack(cen) if cen else np.zeros((0, dim)), cat(vol), np.vstack(crd).astype(np.int64),
            cat(dep).astype(np.int64), asked)
