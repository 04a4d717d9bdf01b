"""Pins for the oracle's other phi-kernels of Section 4 (Eq. 13 with a different phi).

Each is held to a closed form: the value at the centre of a sphere or circle,
where every boundary element is seen at the same distance and angle, and the
skin / core layers above a flat plate.
"""

import numpy as np
import pytest

from oracle import sdf as osdf


def _sphere(r, n, dim):
    """Equal-area samples of a circle / Fibonacci sphere of radius r, outward normals."""
    if dim == 2:
        th = 2 * np.pi * (np.arange(n) + 0.5) / n
        u = np.stack([np.cos(th), np.sin(th)], 1)
        return r * u, u, np.full(n, 2 * np.pi * r / n)
    k = np.arange(n) + 0.5
    z = 1 - 2 * k / n
    ph = np.pi * (1 + 5 ** 0.5) * k
    u = np.stack([np.sqrt(1 - z * z) * np.cos(ph), np.sqrt(1 - z * z) * np.sin(ph), z], 1)
    return r * u, u, np.full(n, 4 * np.pi * r * r / n)


@pytest.mark.parametrize("dim", [3, 2])
def test_proximal_and_radial_kernels_at_the_centre_of_a_sphere(dim):
    lam1, lam2, st, R = 1.0, 3.0, 0.5, 0.8
    for r in (0.5, 1.7):
        q, n, a = _sphere(r, 400, dim)
        p = np.zeros((1, dim))
        # every element: eta = r = |xi|, zeta = -r + i r, cos theta = -1, lambda = -lam2
        prox = osdf.rho_variant(p, q, n, a, osdf.PHI_PROXIMAL, R, lam1, lam2, st, pmc_values=np.array([-1]))
        assert abs(prox[0] - 1j * lam2 * np.sqrt(2 * np.pi)) < 1e-12
        rad = osdf.rho_variant(p, q, n, a, osdf.PHI_RADIAL, R, lam1, lam2, st, pmc_values=np.array([-1]))
        g = np.exp(-0.5 * ((r / R - 1) / st) ** 2) / (np.sqrt(2 * np.pi) * st)
        total = 4 * np.pi * r * r if dim == 3 else 2 * np.pi * r
        assert abs(rad[0] - (-1j * lam2 * g * total)) < 1e-12 * max(1.0, abs(rad[0]))


def test_skin_core_kernel_over_a_plate():
    # a flat boundary sampled on a unit grid at z = 0, normals +z: at height h above a
    # sample the nearest distance is exactly h and the point is outside
    g1 = np.arange(-6, 7, dtype=float)
    X, Y = np.meshgrid(g1, g1)
    q = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    n = np.tile([0.0, 0.0, 1.0], (len(q), 1))
    a = np.ones(len(q))
    lam1, lam2, st, R = 1.5, 2.5, 0.4, 0.6
    for h in (0.2, 0.55, 0.9):
        rho = osdf.rho_variant(np.array([[0.0, 0.0, h]]), q, n, a, osdf.PHI_SKIN, R, lam1, lam2, st,
                               pmc_values=np.array([1]))
        g = lambda x: np.exp(-0.5 * (x / st) ** 2) / (np.sqrt(2 * np.pi) * st)  # noqa: E731
        assert abs(rho[0] - (lam1 * g(h / R - 1) + 1j * lam2 * g(h / R + 1))) < 1e-13
