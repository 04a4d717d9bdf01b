"""Adaptive tree sampling of the SDF (Section 5) through the library against the oracle's tree.

The library builds the tree on the host and evaluates rho at the cells it asks
for with sd_sdf_build on the device; the oracle builds the same tree with its
FP64 rho.  A subdivision decision is a float comparison |rho| h^d >= tau, so
leaves are compared exactly except below cells whose oracle weight lies within
the device path's tolerance of tau (none in the FP64 cases).
"""

import numpy as np
import pytest
import torch

from helpers import oracle_maps, rel_err
from oracle import octree as ooct
from oracle import sdf as osdf
from paper_1712_00238_gb300 import sdfdock as sd
from synth import configs

pytestmark = pytest.mark.gpu


def make_ctx(w, precision):
    return sd.Context(w.dim, precision, 0, lambda1=w.lam1, lambda2=w.lam2, sigma_t=w.sigma_t, eps=w.eps,
                      sigma_g=w.sigma_g, w=w.w)


def quats_dev(q):
    return torch.as_tensor(np.asarray(q, float), dtype=torch.float64, device="cuda").contiguous()


def _setup(name, which, pad=0.2):
    w = getattr(configs, name)()
    s = getattr(w, which)
    b = s.boundary
    sp = w.sdf_params()

    def rho_fn(p):
        return osdf.sdf_rho(p, b.pos, b.normal, b.area, **sp)

    def xi_fn(p):
        return osdf.nearest_distance(p, b.pos)

    lo = s.query.pos.min(0) - pad
    size = float((s.query.pos.max(0) - s.query.pos.min(0)).max() + 2 * pad)
    return w, s, rho_fn, xi_fn, lo, size


def _fragile(asked, rho_fn, lo, size, dim, d_min, tau, rel):
    """(depth, coords) of asked cells whose weight is within rel * (level max) of tau."""
    out = []
    for i, a in enumerate(asked):
        if not len(a):
            continue
        D = d_min + i
        h = size / (1 << D)
        wt = np.abs(rho_fn(a)) * h ** dim
        near = np.abs(wt - tau) <= rel * wt.max()
        k = np.rint((a[near] - lo) / h - 0.5).astype(np.int64)
        out += [(D, tuple(x)) for x in k]
    return out


def _under(leaf_d, leaf_k, cells):
    """Mask of leaves lying in (or equal to) any of the given cells."""
    m = np.zeros(len(leaf_d), bool)
    for D, k in cells:
        deep = leaf_d >= D
        anc = leaf_k[deep] >> (leaf_d[deep] - D)[:, None]
        m[np.flatnonzero(deep)[np.all(anc == np.array(k), axis=1)]] = True
    return m


@pytest.mark.parametrize("name,d_min,d_max,tau,band", [("tiny_2d", 2, 7, 2e-3, np.inf), ("tiny_3d", 1, 4, 2e-2, np.inf),
                                                        ("tiny_2d", 2, 7, 2e-3, 0.3), ("tiny_3d", 1, 4, 2e-2, 0.5)])
def test_tree_and_samples_match_oracle_fp64(name, d_min, d_max, tau, band):
    # band < inf keeps only the leaves within `band` of the nearest boundary
    # sample and drops whole cells beyond band + half their diagonal unevaluated
    w, s, rho_fn, xi_fn, lo, size = _setup(name, "moving")
    b = s.boundary
    c, v, k, d, asked = ooct.octree_leaves(rho_fn, xi_fn, lo, size, w.dim, d_min, d_max, tau, b.spacing, band)
    assert not _fragile(asked, rho_fn, lo, size, w.dim, d_min, tau, 1e-7)
    if np.isfinite(band):
        assert np.all(xi_fn(c) <= band)
    ctx = make_ctx(w, "f64")
    shape, (cen, vol, crd, rho) = ctx.sdf_build_octree(b.pos, b.normal, b.area, lo, size, d_min, d_max, tau,
                                                       b.spacing, return_leaves=True, band=band)
    assert np.array_equal(crd[:, :w.dim], k) and np.array_equal(crd[:, 3], d)
    assert np.allclose(cen[:, :w.dim], c, rtol=0, atol=1e-12 * size) and np.array_equal(vol, v)
    got = rho.cpu().numpy()
    ref = rho_fn(c)
    assert rel_err(got[:, 0] + 1j * got[:, 1], ref) < 1e-9
    assert shape.m == len(c) and len(set(d.tolist())) >= 2
    if w.dim == 2:
        # the tree's samples score like any others: maps against the oracle's
        fb = w.fixed.boundary
        p1 = w.fixed.query.pos
        c1 = osdf.sdf_rho(p1, fb.pos, fb.normal, fb.area, **w.sdf_params()) * w.fixed.query.vol
        fixed = ctx.sdf_build(fb.pos, fb.normal, fb.area, p1, w.fixed.query.vol)
        quats = w.quats[[0, 3]]
        grid = sd.Grid(w.N, w.L)
        maps = ctx.score_maps(fixed, shape, quats_dev(quats), grid).cpu().numpy()
        refm = oracle_maps(p1, c1, c, ref * v, quats, w.N, w.L, w.sigma_g)
        for r in range(len(quats)):
            assert rel_err(maps[r], refm[r]) < 2e-5
    ctx.close()


def test_tree_fp32_3d_matches_away_from_threshold():
    name, d_min, d_max, tau = "tiny_3d", 1, 4, 2e-2
    w, s, rho_fn, xi_fn, lo, size = _setup(name, "moving")
    b = s.boundary
    c, v, k, d, asked = ooct.octree_leaves(rho_fn, xi_fn, lo, size, w.dim, d_min, d_max, tau, b.spacing)
    fragile = _fragile(asked, rho_fn, lo, size, w.dim, d_min, tau, 1e-3)
    ctx = make_ctx(w, "f32")
    shape, (cen, vol, crd, rho) = ctx.sdf_build_octree(b.pos, b.normal, b.area, lo, size, d_min, d_max, tau,
                                                       b.spacing, return_leaves=True)
    gd, gk = crd[:, 3].astype(np.int64), crd[:, :w.dim].astype(np.int64)
    keep_o = ~_under(d, k, fragile)
    keep_g = ~_under(gd, gk, fragile)
    assert keep_o.sum() > 0.9 * len(d)
    assert np.array_equal(gd[keep_g], d[keep_o]) and np.array_equal(gk[keep_g], k[keep_o])
    got = rho.cpu().numpy()
    got = got[keep_g, 0] + 1j * got[keep_g, 1]
    assert rel_err(got, rho_fn(c[keep_o])) < 1e-4
    assert shape.m == len(cen)
    ctx.close()
