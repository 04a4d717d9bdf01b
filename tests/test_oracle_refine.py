"""Pins for the oracle's pose-maximisation updates (Section 6's force model and CG).

Each update rule is held to a closed form or to finite differences of the score,
never to a retyping of itself.
"""

import numpy as np
import pytest

from oracle import refine as orf
from oracle import score as oscore


def _rz(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def test_left_rotation_is_the_axis_angle_rotation():
    q = orf.rotate_left(np.array([1.0, 0, 0, 0]), [0.0, 0.0, 0.7])
    assert np.allclose(oscore.rotation_matrix(q), _rz(0.7), atol=1e-14)
    # left multiplication: R <- Rz(a) R; angles about one axis add
    q0 = np.array([0.9, 0.1, -0.3, 0.2])
    q1 = orf.rotate_left(orf.rotate_left(q0, [0, 0, 0.3]), [0, 0, 0.45])
    assert np.allclose(oscore.rotation_matrix(q1), _rz(0.75) @ oscore.rotation_matrix(q0), atol=1e-13)
    assert abs(np.linalg.norm(q1) - 1.0) < 1e-15


@pytest.mark.parametrize("dim", [3, 2])
def test_force_and_torque_match_finite_differences(dim):
    rng = np.random.default_rng(40 + dim)
    m1, m2, N, L, sg = 40, 25, 8, 4.0, 0.45
    p1 = rng.uniform(-0.8, 0.8, (m1, dim))
    p2 = rng.uniform(-0.6, 0.6, (m2, dim))
    c1 = rng.standard_normal(m1) + 1j * rng.standard_normal(m1)
    c2 = rng.standard_normal(m2) + 1j * rng.standard_normal(m2)
    q = np.array([0.8, 0.2, -0.1, 0.3]) if dim == 3 else np.array([np.cos(0.4), 0, 0, np.sin(0.4)])
    t = np.array([0.1, -0.2, 0.05])[:dim]
    f, F, T, dq = orf.force_torque_fN(p1, c1, p2, c2, q, t, N, L, sg)
    eps = 1e-5

    def score(qq, tt):
        return oscore.pair_score_fN(p1, c1, p2, c2, qq, tt, N, L, sg).real

    assert abs(f - score(q, t)) < 1e-12 * abs(f)
    for a in range(dim):
        e = np.zeros(dim)
        e[a] = eps
        fd = (score(q, t + e) - score(q, t - e)) / (2 * eps)
        assert abs(fd - F[a]) < 1e-6 * np.abs(F).max()
    axes = range(3) if dim == 3 else [2]
    for a in axes:
        e = np.zeros(3)
        e[a] = eps
        fd = (score(orf.rotate_left(q, e), t) - score(orf.rotate_left(q, -e), t)) / (2 * eps)
        assert abs(fd - T[a]) < 1e-6 * np.abs(T).max()
    if dim == 2:
        assert T[0] == 0.0 and T[1] == 0.0 and F[2] == 0.0


def _field(F0=None, T0=None, bowl=None):
    """grad(q, t) of an analytic field: constant force / torque, or f = -|t - bowl|^2."""
    def grad(q, t):
        if bowl is not None:
            F = -2.0 * (t - bowl)
            return -float((t - bowl) @ (t - bowl)), F, np.zeros(3), np.zeros(4)
        return 0.0, np.asarray(F0, float), np.asarray(T0, float), np.zeros(4)
    return grad


def test_cg_moves_straight_in_a_constant_field_and_down_a_bowl():
    F0 = np.array([0.3, -0.4, 1.2])
    q, t, _ = orf.refine(_field(F0, [0, 0, 2.0]), [1, 0, 0, 0], [0, 0, 0], 5, orf.CG, lr_t=0.1, lr_q=0.05)
    assert np.allclose(t, 5 * 0.1 * F0 / np.linalg.norm(F0), atol=1e-14)
    assert np.allclose(oscore.rotation_matrix(q), _rz(5 * 0.05), atol=1e-13)
    # radial bowl: successive gradients are parallel and shrinking, so beta clips to 0
    star = np.array([2.0, 1.0, -1.0])
    q, t, hist = orf.refine(_field(bowl=star), [1, 0, 0, 0], [0, 0, 0], 6, orf.CG, lr_t=0.25)
    assert np.allclose(t, 6 * 0.25 * star / np.linalg.norm(star), atol=1e-13)
    assert np.all(np.diff(hist) > 0)


@pytest.mark.parametrize("gamma", [0.0, 0.2])
def test_dynamics_under_constant_force_and_torque(gamma):
    F0, Tz, m, inertia, h, k = np.array([0.5, -1.0, 0.25]), 0.8, 2.0, 3.0, 0.1, 7
    q, t, _ = orf.refine(_field(F0, [0, 0, Tz]), [1, 0, 0, 0], [0, 0, 0], k, orf.DYNAMICS,
                         mass=m, inertia=inertia, damping=gamma, h=h)
    # v_i = (h F / m) sum_{j<i} (1 - gamma)^j,  t_k = h sum_{i=1..k} v_i (same for the angle)
    s = [sum((1 - gamma) ** j for j in range(i)) for i in range(1, k + 1)]
    assert np.allclose(t, h * h * F0 / m * sum(s), atol=1e-14)
    assert np.allclose(oscore.rotation_matrix(q), _rz(h * h * Tz / inertia * sum(s)), atol=1e-13)

