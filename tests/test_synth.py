"""The sphere-union generators' neighbour lookups make exactly the all-pairs decisions.

The self-avoiding walk compares trial steps only with centres in nearby hash
cells, the buried-sample test only with spheres a k-d tree finds within the
largest radius, and the query-point distance only with spheres within the band
plus the largest radius; each is held here to a brute-force restatement on
small inputs, bit for bit.
"""

import numpy as np

from synth import configs
from synth import shapes as sh


def _walk_all_pairs(n, seed, step=3.8, min_sep=2.8, conf_scale=3.0, tries=100):
    rng = np.random.default_rng(np.random.SeedSequence([seed, 3, n]))
    rc = conf_scale * n ** (1.0 / 3.0)
    cen = np.zeros((n, 3))
    k = 1
    while k < n:
        d = rng.standard_normal((tries, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        cand = cen[k - 1] + step * d
        ok = np.linalg.norm(cand, axis=1) <= rc
        if k >= 2:
            dd = np.linalg.norm(cand[:, None, :] - cen[None, : k - 1, :], axis=2)
            ok &= (dd >= min_sep).all(axis=1)
        idx = np.flatnonzero(ok)
        if len(idx):
            cen[k] = cand[idx[0]]
            k += 1
        else:
            k = max(1, k - 1)
    return cen - cen.mean(0)


def test_walk_equals_all_pairs_walk():
    for n, seed in ((40, 1), (150, 7)):
        assert np.array_equal(sh.self_avoiding_walk(n, seed), _walk_all_pairs(n, seed))


def test_buried_samples_equal_all_pairs_test():
    su = sh.sphere_union(120, 3)
    b = sh.sphere_union_boundary(su, 2.0, 3)
    # regenerate every sample and bury by comparing with every sphere
    rng = np.random.default_rng(np.random.SeedSequence([3, 5, len(su.radii)]))
    pos = []
    for c, r in zip(su.centers, su.radii):
        cnt = max(4, int(round(2.0 * 4 * np.pi * r * r)))
        v = rng.standard_normal((cnt, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        pos.append(c + r * v)
    pos = np.vstack(pos)
    d = np.linalg.norm(pos[:, None, :] - su.centers[None], axis=2) - su.radii[None]
    keep = (d >= -1e-6).all(axis=1)
    assert np.array_equal(b.pos, pos[keep])


def test_query_points_equal_unbounded_distance():
    n, seed, band = 90, 11, 2.0
    s = configs._sphere_shape("x", n, seed)
    su = s.query.info["spheres"]

    def sdist_all(p):  # 16 nearest centres by brute force, no distance bound
        d = np.linalg.norm(p[:, None, :] - su.centers[None], axis=2)
        order = np.argsort(d, axis=1, kind="stable")[:, :16]
        rows = np.arange(len(p))[:, None]
        return (d[rows, order] - su.radii[order]).min(axis=1)

    lo = su.centers.min(0) - su.radii.max() - band
    hi = su.centers.max(0) + su.radii.max() + band
    q = sh.query_points(sdist_all, lo, hi, s.query.info["cell"], s.boundary.spacing, band, seed + 77)
    assert np.array_equal(q.pos, s.query.pos)
    assert np.array_equal(q.inside, s.query.inside)
