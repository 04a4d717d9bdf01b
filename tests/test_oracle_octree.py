"""Pins for the oracle's adaptive tree sampling (Section 5's octree of SDF samples).

The level-by-level tree is held to a depth-first restatement, to the uniform
grid it must reduce to, to a tiling of the root cube and to the midpoint-rule
error bound of the density it samples.
"""

import math

import numpy as np
import pytest

from oracle import octree as ooct


def _far(p):
    return np.full(len(p), np.inf)


def test_tau_zero_is_the_uniform_grid():
    lo, size, D = np.array([-1.0, 0.5]), 2.0, 3
    c, v, k, d, asked = ooct.octree_leaves(lambda p: np.ones(len(p)), _far, lo, size, 2, 1, D, 0.0, 0.0)
    h = size / 8
    want = [(lo[0] + (i + 0.5) * h, lo[1] + (j + 0.5) * h) for j in range(8) for i in range(8)]
    assert np.allclose(c, want, rtol=0, atol=1e-15)
    assert np.all(v == h * h) and np.all(d == D)
    assert [a.shape[0] for a in asked] == [4, 16]


def _dfs(rho_fn, xi_fn, lo, size, dim, d_min, d_max, tau, clear):
    leaves = set()

    def visit(k, D):
        h = size / (1 << D)
        c = lo + (np.array(k) + 0.5) * h
        xi = float(xi_fn(c[None])[0])
        split = False
        if D < d_max:
            split = xi < 0.5 * h * math.sqrt(dim) or abs(rho_fn(c[None])[0]) * h ** dim >= tau
        if split:
            for off in np.ndindex(*([2] * dim)):
                visit(tuple(2 * a + b for a, b in zip(k, off)), D + 1)
        elif xi >= clear:
            leaves.add((D,) + tuple(k))

    for k in np.ndindex(*([1 << d_min] * dim)):
        visit(k, d_min)
    return leaves


@pytest.mark.parametrize("dim", [2, 3])
def test_levels_equal_depth_first_tree(dim):
    rng = np.random.default_rng(5 + dim)
    q = rng.normal(size=(60, dim))
    q /= np.linalg.norm(q, axis=1, keepdims=True) * 1.3         # samples on a sphere of radius 1/1.3
    lo, size = np.full(dim, -1.1), 2.23

    def xi_fn(p):
        return np.linalg.norm(p[:, None, :] - q[None], axis=2).min(1)

    def rho_fn(p):
        return np.exp(-np.linalg.norm(p, axis=1) ** 2 / 0.1) * (1 + 2j)

    args = (rho_fn, xi_fn, lo, size, dim, 1, 4 if dim == 3 else 6, 1e-3 if dim == 2 else 3e-3, 0.05)
    c, v, k, d, _ = ooct.octree_leaves(*args)
    got = {(int(a),) + tuple(int(x) for x in b) for a, b in zip(d, k)}
    assert len(got) == len(d)
    assert got == _dfs(*args)
    assert len(set(d.tolist())) >= 3                             # the tree is genuinely adaptive
    # listing order: depth, then linear index
    lin = [(int(a), sum(int(b[i]) << (a * i) for i in range(dim))) for a, b in zip(d, k)]
    assert lin == sorted(lin)
    # leaves tile the root, up to the dropped cells next to the boundary
    pts = lo + size * rng.random((4000, dim))
    hits = np.zeros(len(pts), int)
    for cc, hh in zip(c, v ** (1 / dim)):
        hits += np.all(np.abs(pts - cc) < hh / 2, axis=1)
    assert hits.max() == 1
    miss = pts[hits == 0]
    hmax = size / 2 ** 1
    assert np.all(xi_fn(miss) < 0.05 + hmax * math.sqrt(dim))
    assert abs(v.sum() - size ** dim) < size ** dim and v.sum() <= size ** dim + 1e-12


def test_midpoint_rule_is_exact_for_affine_density():
    # the midpoint rule integrates an affine density exactly on every cell, so any
    # tiling with the right centres and volumes reproduces its integral
    dim = 3
    lo, size = np.array([-2.0, 1.0, 0.5]), 4.0
    a, b = -6.3, np.array([3.0, 0.5, -0.4])                     # changes sign inside the cube

    def rho_fn(p):
        return a + (p - lo) @ b

    c, v, k, d, _ = ooct.octree_leaves(rho_fn, _far, lo, size, dim, 1, 5, 0.5, 0.0)
    assert len(set(d.tolist())) >= 3
    exact = size ** dim * (a + b.sum() * size / 2)
    assert abs((rho_fn(c) * v).sum() - exact) < 1e-13 * (np.abs(rho_fn(c)) * v).sum()
    assert v.sum() == size ** dim
    # where the density is large the cube is sampled deeper
    w = np.abs(rho_fn(c))
    assert np.mean(d[w > np.median(w)]) > np.mean(d[w < np.median(w)])


@pytest.mark.parametrize("dim", [2, 3])
def test_band_keeps_exactly_the_leaves_within_it(dim):
    # a cell dropped as lying wholly beyond the band has only descendants beyond it,
    # so the banded tree is the full tree's leaves filtered by centre distance
    rng = np.random.default_rng(21 + dim)
    q = rng.normal(size=(80, dim))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    lo, size, band = np.full(dim, -2.3), 4.7, 0.35

    def xi_fn(p):
        return np.linalg.norm(p[:, None, :] - q[None], axis=2).min(1)

    def rho_fn(p):
        return 1.0 / (0.05 + np.abs(np.linalg.norm(p, axis=1) - 1.0)) + 0j

    args = (rho_fn, xi_fn, lo, size, dim, 1, 6 if dim == 2 else 4, 4e-3, 0.05)
    c0, v0, k0, d0, a0 = ooct.octree_leaves(*args)
    c1, v1, k1, d1, a1 = ooct.octree_leaves(*args, band=band)
    keep = xi_fn(c0) <= band
    assert 0 < keep.sum() < len(keep)
    assert np.array_equal(c1, c0[keep]) and np.array_equal(d1, d0[keep]) and np.array_equal(k1, k0[keep])
    assert np.all(xi_fn(c1) <= band) and np.all(xi_fn(c1) >= 0.05)
    assert sum(len(a) for a in a1) < sum(len(a) for a in a0)
