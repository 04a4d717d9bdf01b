"""Shared test helpers: oracle-side inputs and comparison metrics.

Inputs come from the seeded generators in synth/; expected values come only
from oracle/.  GPU results are produced through the C ABI (via the binding).
"""

from __future__ import annotations

import functools

import numpy as np

from oracle import score as oscore
from oracle import sdf as osdf
from synth import configs


def rel_err(got, ref):
    """Max-norm relative error: max |got - ref| / max |ref|."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.abs(got - ref).max() / np.abs(ref).max())


@functools.lru_cache(maxsize=None)
def oracle_weights(name: str):
    """(p1, c1, p2, c2) with c = rho * vol from the oracle's SDF (small workloads only)."""
    w = getattr(configs, name)()
    out = []
    for s in (w.fixed, w.moving):
        b = s.boundary
        rho = osdf.sdf_rho(s.query.pos, b.pos, b.normal, b.area, **w.sdf_params())
        out += [s.query.pos, rho * s.query.vol]
    return tuple(out)


def synthetic_weights(m: int, seed: int):
    """Seeded complex weights standing in for c_i (shared input, no method arithmetic)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 99]))
    return rng.standard_normal(m) + 1j * rng.standard_normal(m)


def cplx_to_pairs(c):
    c = np.asarray(c)
    return np.stack([c.real, c.imag], 1)


def oracle_maps(p1, c1, p2, c2, quats, N, L, sigma_g):
    F1 = oscore.nudft(p1, c1, N, L, -1)
    return np.array([oscore.score_map_fN(p1, c1, p2, c2, q, N, L, sigma_g, F1=F1).ravel() for q in quats])
