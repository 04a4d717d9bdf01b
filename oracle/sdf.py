"""Oracle: the skeletal density function (SDF) of a solid from oriented boundary samples.

TEST INFRASTRUCTURE.  A deliberately plain FP64 NumPy restatement of the paper's
definitions, used only by tests, by the smoke check and by the benchmark's CPU
baseline.  It shares no code with the CUDA path.

Definitions followed (Section 4):

* Eq. 10A  xi(p) = pmc(p) * min_q eta(p, q), eta = ||p - q||.
* PMC      the solid's membership from its consistent outward normals: the
           generalised winding number w(p) = sum_j a_j (q_j - p).n_j / (S ||q_j - p||^d)
           with S = 2*pi (2D) or 4*pi (3D); pmc = -1 where w > 1/2, else +1.
* Eq. 11   zeta = xi + i*eta (the "+" convention).
* Eq. 12a  cos(theta) = (p - q).n / eta.
* Eq. 13   rho(p) = integral over the boundary of phi(zeta) cos(theta) ds,
           taken as a midpoint sum over the samples (weights a_j).
* Eq. 15   phi(zeta) = lambda / sqrt(2 pi) * zeta^-2 * g_sigma(|tan angle(zeta)| - 1),
           g_sigma(x) = exp(-x^2 / (2 sigma^2)) / (sqrt(2 pi) sigma), |tan angle zeta| = eta/|xi|.
* Eq. 16c  lambda = +lambda1 outside (xi > 0), -lambda2 inside (xi < 0).
* Eq. 17t  truncation: only samples with eta <= (1 + eps)|xi| contribute
           (the contact region of Def. 1, Eq. 10b); eps = inf keeps all.

Planar shapes (d = 2): Eq. 17 measures each boundary element by the solid angle
it subtends over 4*pi.  In the plane the same construction uses the planar angle
cos(theta) ds / eta over 2*pi, which multiplies the 3D summand by 2*eta.  That
reading keeps rho scale-invariant in 2D as it is in 3D.
"""

from __future__ import annotations

import math

import numpy as np


def nearest_distance(p, q, chunk=1024):
    """|xi(p)| = min_j ||p - q_j|| (Eq. 10A without the sign)."""
    p = np.asarray(p, float)
    q = np.asarray(q, float)
    out = np.empty(len(p))
    for s in range(0, len(p), chunk):
        d = np.linalg.norm(p[s:s + chunk, None, :] - q[None, :, :], axis=2)
        out[s:s + chunk] = d.min(axis=1)
    return out


def winding_number(p, q, nrm, area, chunk=1024):
    """Generalised winding number of the sampled boundary seen from each p."""
    p = np.asarray(p, float)
    d = p.shape[1]
    S = 2.0 * math.pi if d == 2 else 4.0 * math.pi
    out = np.empty(len(p))
    for s in range(0, len(p), chunk):
        v = q[None, :, :] - p[s:s + chunk, None, :]          # q - p
        r = np.linalg.norm(v, axis=2)
        dot = (v * nrm[None, :, :]).sum(axis=2)
        out[s:s + chunk] = (area[None, :] * dot / (S * r ** d)).sum(axis=1)
    return out


def pmc(p, q, nrm, area):
    """Point membership: -1 inside (winding number > 1/2), +1 outside."""
    return np.where(winding_number(p, q, nrm, area) > 0.5, -1.0, 1.0)


def signed_distance(p, q, nrm, area):
    return pmc(p, q, nrm, area) * nearest_distance(p, q)


def sdf_rho(p, q, nrm, area, lam1=1.0, lam2=3.0, sigma_t=0.5, eps=1.5, pmc_values=None,
            chunk=512):
    """rho(p) of Eq. 13 with the kernel of Eq. 15, truncated as in Eq. 17t.

    Returns the complex SDF value at every query point.  ``pmc_values`` may
    supply the membership (+1 / -1) instead of the winding-number rule.
    """
    p = np.asarray(p, float)
    q = np.asarray(q, float)
    nrm = np.asarray(nrm, float)
    area = np.asarray(area, float)
    dim = p.shape[1]
    if pmc_values is None:
        pmc_values = pmc(p, q, nrm, area)
    rho = np.empty(len(p), complex)
    for s in range(0, len(p), chunk):
        ps = p[s:s + chunk]
        diff = ps[:, None, :] - q[None, :, :]                 # p - q
        eta = np.linalg.norm(diff, axis=2)
        xi = pmc_values[s:s + chunk] * eta.min(axis=1)         # Eq. 10A
        lam = np.where(xi > 0, lam1, -lam2)                    # Eq. 16c
        ratio = eta / np.abs(xi)[:, None]                      # |tan angle zeta|
        cos_t = (diff * nrm[None, :, :]).sum(axis=2) / eta     # Eq. 12a
        g = np.exp(-0.5 * ((ratio - 1.0) / sigma_t) ** 2) / (math.sqrt(2 * math.pi) * sigma_t)
        g = np.where(ratio - 1.0 <= eps, g, 0.0)               # Eq. 17t
        zeta = xi[:, None] + 1j * eta                          # Eq. 11
        phi = lam[:, None] / math.sqrt(2 * math.pi) * g / zeta ** 2   # Eq. 15
        if dim == 2:
            phi = phi * 2.0 * eta                              # planar angle measure
        rho[s:s + chunk] = (phi * cos_t * area[None, :]).sum(axis=1)   # Eq. 13
    return rho


PHI_SDF, PHI_PROXIMAL, PHI_RADIAL, PHI_SKIN = 0, 1, 2, 3


def rho_variant(p, q, nrm, area, phi, radius=1.0, lam1=1.0, lam2=3.0, sigma_t=0.5, pmc_values=None, chunk=512):
    """rho(p) for the other phi-kernels Section 4 sets beside Eq. 15 (their Section 3 analogues).

    Eq. 13 with a different phi, or the pointwise skin/core form:
      PHI_PROXIMAL  phi(zeta) = lambda zeta^-2 / sqrt(2 pi), lambda of Eq. 16c (the proximal
                    factor of Eq. 15 alone: inverse-square, no characteristic size, no
                    truncation); in 2D the planar angle measure as for Eq. 15;
      PHI_RADIAL    phi(zeta) = c g(eta / R - 1), c = lam1 outside and i lam2 inside
                    (skin real, core imaginary), g the normalised Gaussian of width sigma_t:
                    only eta = Im zeta is used, like the radial-basis double-skin affinity;
      PHI_SKIN      rho(p) = lam1 g(xi / R - 1) + i lam2 g(xi / R + 1), the swept-volume
                    skin / core layers of the signed distance (no boundary integral);
    with R = ``radius``.
    """
    p = np.asarray(p, float)
    q = np.asarray(q, float)
    nrm = np.asarray(nrm, float)
    area = np.asarray(area, float)
    dim = p.shape[1]
    if pmc_values is None:
        pmc_values = pmc(p, q, nrm, area)

    def gauss(x):
        return np.exp(-0.5 * (x / sigma_t) ** 2) / (math.sqrt(2 * math.pi) * sigma_t)

    rho = np.empty(len(p), complex)
    for s in range(0, len(p), chunk):
        ps = p[s:s + chunk]
        diff = ps[:, None, :] - q[None, :, :]
        eta = np.linalg.norm(diff, axis=2)
        xi = pmc_values[s:s + chunk] * eta.min(axis=1)
        if phi == PHI_SKIN:
            rho[s:s + chunk] = lam1 * gauss(xi / radius - 1.0) + 1j * lam2 * gauss(xi / radius + 1.0)
            continue
        cos_t = (diff * nrm[None, :, :]).sum(axis=2) / eta
        if phi == PHI_PROXIMAL:
            lam = np.where(xi > 0, lam1, -lam2)
            zeta = xi[:, None] + 1j * eta
            f = lam[:, None] / math.sqrt(2 * math.pi) / zeta ** 2
            if dim == 2:
                f = f * 2.0 * eta
        elif phi == PHI_RADIAL:
            c = np.where(xi > 0, lam1 + 0j, 1j * lam2)
            f = c[:, None] * gauss(eta / radius - 1.0)
        else:
            raise ValueError(phi)
        rho[s:s + chunk] = (f * cos_t * area[None, :]).sum(axis=1)
    return rho


def sdf_weights(rho, vol):
    """Weights of the sampled representation: c_i = rho_i * v_i."""
    return np.asarray(rho) * np.asarray(vol)
