"""Table 1 (Section 4) as a golden fixture: the sign and size of the score contribution of overlapping
high-density regions, through the oracle's SDF and its pair score (no conjugate on either density)."""

import math
import os

import numpy as np
import pytest

from oracle import score, sdf

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_overlaps.txt")
SIG = 0.5


def _rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            a, b, sign, f1, f2 = line.split()
            rows.append((a, b, sign, f1, f2))
    return rows


def _centre_density(region, dim, lam1, lam2, n=400, radius=0.9):
    # samples on a sphere / circle: outward normals bound a ball (the centre is interior),
    # inward normals bound a cavity in a surrounding solid (the centre is exterior)
    rng = np.random.default_rng(dim * 10 + n)
    v = rng.standard_normal((n, dim))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    meas = 4 * math.pi * radius ** 2 if dim == 3 else 2 * math.pi * radius
    nrm = v if region == "i" else -v
    rho = sdf.sdf_rho(np.zeros((1, dim)), radius * v, nrm, np.full(n, meas / n), lam1, lam2, SIG, 1.5)
    return rho[0]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("lam1,lam2", [(1.0, 3.0), (2.0, 0.5)])
def test_table1_overlap_contributions(dim, lam1, lam2):
    rows = _rows()
    assert len(rows) == 4
    lam = {"l1": lam1, "l2": lam2}
    dens = {r: _centre_density(r, dim, lam1, lam2) for r in ("e", "i")}
    assert abs(dens["e"] + 1j * lam1 / SIG) < 1e-12 and abs(dens["i"] - 1j * lam2 / SIG) < 1e-12
    sg, vol = 0.2, 0.01
    g0 = (4 * math.pi * sg * sg) ** (-dim / 2)           # G_{sigma_g sqrt 2}(0)
    q = np.array([1.0, 0.0, 0.0, 0.0])
    for a, b, sign, f1, f2 in rows:
        want = (1.0 if sign == "+" else -1.0) * lam[f1] * lam[f2] / SIG ** 2
        # one sample of each solid at the same point: f = c1 c2 G(0)
        f = score.pair_score_fc(np.zeros((1, dim)), np.array([dens[a] * vol]), np.zeros((1, dim)),
                                np.array([dens[b] * vol]), q, np.zeros(dim), sg)
        got = f / (vol * vol * g0)
        assert abs(got.imag) < 1e-9 * abs(want)
        assert abs(got.real - want) < 1e-9 * abs(want), (a, b)
