"""Rotation and pose sets, as unit quaternions (w, x, y, z), Hamilton convention.

A quaternion q acts on a point as the active rotation p -> q p q*.  Only the
sets themselves live here; turning a quaternion into a matrix is left to each
consumer.

* planar(n): rotations by 2*pi*r/n about +z, the 2D search of Section 6.
* hopf_grid(nside, n_psi): the Hopf-fibration grid of Yershova et al.
  (IJRR 2010): HEALPix pixel centres on S^2 times a uniform circle.
* super_fibonacci(n): Alexa's super-Fibonacci spiral on S^3 (CVPR 2022).
* random_uniform(n, seed): Shoemake's uniform random rotations.
"""

from __future__ import annotations

import math

import numpy as np


def planar(n: int) -> np.ndarray:
    th = 2.0 * np.pi * np.arange(n) / n
    return np.stack([np.cos(th / 2), np.zeros(n), np.zeros(n), np.sin(th / 2)], 1)


def healpix_centres(nside: int) -> tuple[np.ndarray, np.ndarray]:
    """(theta, phi) of the 12*nside^2 HEALPix pixel centres in ring order (Gorski et al. 2005)."""
    npix = 12 * nside * nside
    ncap = 2 * nside * (nside - 1)
    z = np.empty(npix)
    phi = np.empty(npix)
    for p in range(npix):
        if p < ncap:
            ph = (p + 1) / 2.0
            i = int(math.floor(math.sqrt(ph - math.sqrt(math.floor(ph))))) + 1
            j = p + 1 - 2 * i * (i - 1)
            z[p] = 1.0 - i * i / (3.0 * nside * nside)
            phi[p] = (j - 0.5) * math.pi / (2.0 * i)
        elif p < npix - ncap:
            ip = p - ncap
            i = ip // (4 * nside) + nside
            j = ip % (4 * nside) + 1
            s = (i - nside + 1) % 2
            z[p] = (2.0 * nside - i) * 2.0 / (3.0 * nside)
            phi[p] = (j - s / 2.0) * math.pi / (2.0 * nside)
        else:
            ip = npix - p
            ph = ip / 2.0
            i = int(math.floor(math.sqrt(ph - math.sqrt(math.floor(ph))))) + 1
            j = 4 * i + 1 - (ip - 2 * i * (i - 1))
            z[p] = -1.0 + i * i / (3.0 * nside * nside)
            phi[p] = (j - 0.5) * math.pi / (2.0 * i)
    return np.arccos(np.clip(z, -1, 1)), phi


def hopf_grid(nside: int = 2, n_psi: int = 12) -> np.ndarray:
    """Hopf coordinates: S^2 from HEALPix (12*nside^2 points) times n_psi circle points.

    nside=2, n_psi=12 gives 48 x 12 = 576 rotations.
    """
    th, ph = healpix_centres(nside)
    psi = 2.0 * np.pi * (np.arange(n_psi) + 0.5) / n_psi
    T, S = np.meshgrid(th, psi, indexing="ij")   # theta, psi
    P, _ = np.meshgrid(ph, psi, indexing="ij")   # phi
    T, P, S = T.ravel(), P.ravel(), S.ravel()
    q = np.stack([np.cos(T / 2) * np.cos(S / 2), np.cos(T / 2) * np.sin(S / 2),
                  np.sin(T / 2) * np.cos(P + S / 2), np.sin(T / 2) * np.sin(P + S / 2)], 1)
    # rows of q above are (theta, phi) outer, psi inner
    return q / np.linalg.norm(q, axis=1, keepdims=True)


_SF_PHI = math.sqrt(2.0)
_SF_PSI = 1.533751168755204288118041  # real root of x^4 = x + 4


def super_fibonacci(n: int) -> np.ndarray:
    s = np.arange(n) + 0.5
    r = np.sqrt(s / n)
    R = np.sqrt(1.0 - s / n)
    a = 2.0 * np.pi * s / _SF_PHI
    b = 2.0 * np.pi * s / _SF_PSI
    q = np.stack([r * np.sin(a), r * np.cos(a), R * np.sin(b), R * np.cos(b)], 1)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def random_uniform(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(np.random.SeedSequence([seed, 7]))
    u1, u2, u3 = rng.random((3, n))
    q = np.stack([np.sqrt(1 - u1) * np.sin(2 * np.pi * u2), np.sqrt(1 - u1) * np.cos(2 * np.pi * u2),
                  np.sqrt(u1) * np.sin(2 * np.pi * u3), np.sqrt(u1) * np.cos(2 * np.pi * u3)], 1)
    return q


def random_ball(n: int, radius: float, seed: int, dim: int = 3) -> np.ndarray:
    rng = np.random.default_rng(np.random.SeedSequence([seed, 8]))
    v = rng.standard_normal((n, dim))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * radius * rng.random(n)[:, None] ** (1.0 / dim)
