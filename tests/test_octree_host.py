"""The library's host-side sampling tree (sd_octree_*) against the oracle's tree (no GPU needed).

Both trees are driven with the oracle's rho at the centres they ask for, so every
subdivision decision is taken on the same FP64 values; the leaves (integer
coordinates, depths, centres, volumes) must agree exactly.
"""

import ctypes as ct

import numpy as np
import pytest

from oracle import octree as ooct
from oracle import sdf as osdf
from paper_1712_00238_gb300 import build as pbuild
from paper_1712_00238_gb300 import sdfdock as sd
from synth import configs


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return sd.load()


def _box(s, pad=0.2):
    lo = s.query.pos.min(0) - pad
    return lo, float((s.query.pos.max(0) - s.query.pos.min(0)).max() + 2 * pad)


def _drive(tree, rho_fn, dim):
    asked = []
    while True:
        cen, vol = tree.pending()
        if len(cen) == 0:
            break
        assert np.all(cen[:, 3] == 0) and np.all(vol == vol[0])
        asked.append(cen[:, :dim])
        tree.feed(rho_fn(cen[:, :dim]))
    return asked


INF = float("inf")


@pytest.mark.parametrize("case", [("tiny_2d", "moving", 2, 7, 2e-3, 0.2, INF), ("tiny_2d", "fixed", 2, 7, 2e-2, 0.2, INF),
                                  ("tiny_3d", "moving", 1, 4, 2e-2, 0.2, INF),
                                  ("tiny_2d", "moving", 0, 8, 2e-3, 3.0, INF),   # root far larger than the shape
                                  ("tiny_2d", "fixed", 1, 7, 2e-2, 1.0, 0.5),     # samples kept to a band
                                  ("tiny_3d", "moving", 1, 5, 5e-3, 0.5, 0.3)])
def test_tree_equals_oracle_tree(lib, case):
    name, which, d_min, d_max, tau, pad, band = case
    w = getattr(configs, name)()
    s = getattr(w, which)
    b = s.boundary
    sp = w.sdf_params()

    def rho_fn(p):
        return osdf.sdf_rho(p, b.pos, b.normal, b.area, **sp)

    def xi_fn(p):
        return osdf.nearest_distance(p, b.pos)

    lo, size = _box(s, pad)
    c, v, k, d, asked = ooct.octree_leaves(rho_fn, xi_fn, lo, size, w.dim, d_min, d_max, tau, b.spacing, band)
    tree = sd.Octree(w.dim, b.pos, lo, size, d_min, d_max, tau, b.spacing, band)
    got_asked = _drive(tree, rho_fn, w.dim)
    cen, vol, crd = tree.leaves()
    tree.close()
    assert len(set(d.tolist())) >= 2
    want_asked = [a for a in asked if len(a)]
    assert len(got_asked) == len(want_asked)
    for g, a in zip(got_asked, want_asked):
        assert np.array_equal(g, a)
    assert np.array_equal(crd[:, :w.dim], k) and np.array_equal(crd[:, 3], d)
    assert np.array_equal(cen[:, :w.dim], c) and np.array_equal(vol, v)


def test_uniform_limit_and_no_boundary(lib):
    tree = sd.Octree(3, np.zeros((0, 4)), [0.5, -1.0, 2.0], 2.0, 1, 3, 0.0, 0.0)
    _drive(tree, lambda p: np.ones(len(p)), 3)
    cen, vol, crd = tree.leaves()
    h = 2.0 / 8
    ii = np.arange(8)
    want = np.stack(np.meshgrid(ii, ii, ii, indexing="ij"), -1).reshape(-1, 3)[:, ::-1]   # x fastest
    assert np.array_equal(crd[:, :3], want) and np.all(crd[:, 3] == 3)
    assert np.allclose(cen[:, :3], np.array([0.5, -1.0, 2.0]) + (want + 0.5) * h, rtol=0, atol=1e-15)
    assert np.all(vol == h ** 3)


def test_argument_errors(lib):
    h = ct.c_void_p()
    lo = np.zeros(3)
    b = np.zeros((4, 4))
    b[:, 0] = np.arange(4)

    def create(dim=3, bp=b.ctypes.data, n=4, size=1.0, dmin=1, dmax=3, tau=0.1, clear=0.0, band=INF):
        return lib.sd_octree_create(dim, bp, n, lo.ctypes.data, size, dmin, dmax, tau, clear, band, ct.byref(h))

    assert create() == sd.SD_OK
    lib.sd_octree_free(h)
    for bad in (dict(dim=4), dict(n=-1), dict(bp=None), dict(size=0.0), dict(size=float("inf")), dict(dmin=4),
                dict(dmax=21), dict(tau=float("nan")), dict(tau=-1.0), dict(clear=-0.1), dict(band=-1.0),
                dict(band=float("nan"))):
        assert create(**bad) == sd.SD_ERR_ARG, bad
        assert not h.value
    assert create(dmin=10, dmax=12) == sd.SD_ERR_OOM
    b2 = b.copy()
    b2[2, 1] = np.nan
    assert lib.sd_octree_create(3, b2.ctypes.data, 4, lo.ctypes.data, 1.0, 1, 3, 0.1, 0.0, INF, ct.byref(h)) \
        == sd.SD_ERR_NONFINITE
    # a tree waiting for rho: wrong count, non-finite values and early leaves are refused
    tree = sd.Octree(3, np.zeros((0, 4)), lo, 1.0, 1, 3, 1e-3, 0.0)
    cen, vol = tree.pending()
    m = ct.c_int64()
    assert lib.sd_octree_leaves(tree.handle, ct.byref(m), None, None, None) == sd.SD_ERR_ARG
    r = np.ones((len(cen), 2))
    assert lib.sd_octree_feed(tree.handle, r.ctypes.data, len(cen) - 1) == sd.SD_ERR_ARG
    r[3, 1] = np.inf
    assert lib.sd_octree_feed(tree.handle, r.ctypes.data, len(cen)) == sd.SD_ERR_NONFINITE
    cen2, _ = tree.pending()
    assert np.array_equal(cen, cen2)
    _drive(tree, lambda p: np.ones(len(p)), 3)
    c3, v3, k3 = tree.leaves()
    assert np.all(k3[:, 3] == 3) and v3.sum() == 1.0
    assert lib.sd_octree_feed(tree.handle, r.ctypes.data, 0) == sd.SD_ERR_ARG
    tree.close()
    assert lib.sd_octree_free(None) == sd.SD_OK
