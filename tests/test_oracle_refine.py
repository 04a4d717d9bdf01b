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



def _scripted(Fs, Ts, dqs=None):
    """grad(q, t) that returns the k-th scripted (F, T, dq) on its k-th call, whatever the pose."""
    calls = []

    def grad(q, t):
        k = len(calls)
        calls.append(k)
        dq = np.zeros(4) if dqs is None else np.asarray(dqs[k], float)
        return 0.0, np.asarray(Fs[k], float), np.asarray(Ts[k], float), dq
    return grad


def _expm_rot(theta):
    """Rotation matrix of the rotation vector theta as the matrix exponential of its skew matrix."""
    from scipy.linalg import expm
    x, y, z = theta
    return expm(np.array([[0.0, -z, y], [z, 0.0, -x], [-y, x, 0.0]]))


def test_cg_polak_ribiere_beta_and_its_clip():
    # Scripted gradients, so every direction is worked out by hand:
    #   translation block, lr_t = 0.5 from t = 0:
    #     F0 = (3, 4, 0): d0 = F0, |d0| = 5, t1 = (0.3, 0.4, 0)
    #     F1 = (0, 5, 0): beta = F1.(F1 - F0) / |F0|^2 = 5/25 = 1/5 (Polak-Ribiere;
    #       Fletcher-Reeves would give 1), d1 = (3/5, 29/5, 0), |d1| = sqrt(34),
    #       t2 = t1 + (0.3, 2.9, 0) / sqrt(34)
    #     F2 = (0, 1, 0): F2.(F2 - F1) = -4 < 0, so beta clips to 0 and d2 = F2,
    #       t3 = t2 + (0, 0.5, 0)
    #   rotation block, lr_q = 0.1 rad:
    #     T0 = (0, 0, 2): turn 0.1 about z
    #     T1 = (1, 0, 3): beta = (1, 0, 3).(1, 0, 1) / 4 = 1, d1 = (1, 0, 5): turn 0.1
    #       about (1, 0, 5)/sqrt(26)
    #     T2 = (0, 0, 1): T2.(T2 - T1) = -2 < 0, clipped: turn 0.1 about z
    Fs = [(3, 4, 0), (0, 5, 0), (0, 1, 0), (0, 0, 0)]
    Ts = [(0, 0, 2), (1, 0, 3), (0, 0, 1), (0, 0, 0)]
    q0 = np.array([0.9, 0.1, -0.3, 0.2]) / np.linalg.norm([0.9, 0.1, -0.3, 0.2])
    q, t, _ = orf.refine(_scripted(Fs, Ts), q0, [0, 0, 0], 3, orf.CG, lr_t=0.5, lr_q=0.1)
    r34 = np.sqrt(34.0)
    assert np.allclose(t, [0.3 + 0.3 / r34, 0.4 + 2.9 / r34 + 0.5, 0.0], atol=1e-14)
    axis = np.array([1.0, 0.0, 5.0]) / np.sqrt(26.0)
    want = (_expm_rot([0, 0, 0.1]) @ _expm_rot(0.1 * axis) @ _expm_rot([0, 0, 0.1])
            @ oscore.rotation_matrix(q0))
    assert np.allclose(oscore.rotation_matrix(q), want, atol=1e-13)


def test_ascent_step_is_normalised_by_the_largest_entry():
    # Scripted gradients, lr_t = 0.1, lr_q = 0.05 from t = (1, 1, 1), q = 1:
    #   F0 = (0.5, -2, 1) -> step (0.25, -1, 0.5) * 0.1;  dq0 = (0.1, 0.4, -0.2, 0) ->
    #   q1 = (1.0125, 0.05, -0.025, 0) / sqrt(1.02828125)
    #   F1 = (0, 0, -4) -> step (0, 0, -0.1);  dq1 = (0, 0, 0, 3) -> q2 = (q1 + (0, 0, 0, 0.05)) / |.|
    Fs = [(0.5, -2, 1), (0, 0, -4), (0, 0, 0)]
    dqs = [(0.1, 0.4, -0.2, 0), (0, 0, 0, 3), (0, 0, 0, 0)]
    q, t, _ = orf.refine(_scripted(Fs, [(0, 0, 0)] * 3, dqs), [1, 0, 0, 0], [1, 1, 1], 2, orf.ASCENT,
                         lr_t=0.1, lr_q=0.05)
    assert np.allclose(t, [1.025, 0.9, 0.95], atol=1e-15)
    q1 = np.array([1.0125, 0.05, -0.025, 0.0]) / np.sqrt(1.02828125)
    q2 = q1 + np.array([0, 0, 0, 0.05])
    assert np.allclose(q, q2 / np.linalg.norm(q2), atol=1e-15)
    assert abs(np.linalg.norm(q) - 1.0) < 1e-15


@pytest.mark.parametrize("method", [orf.ASCENT, orf.CG])
def test_small_steps_climb_the_pair_sum_score(method):
    # a steepest-ascent (or conjugate) step short enough for the field to be
    # locally linear raises the score: f_N rises at every step from a pose near a peak
    rng = np.random.default_rng(5)
    p1 = rng.uniform(-0.7, 0.7, (30, 3))
    p2 = rng.uniform(-0.5, 0.5, (20, 3))
    c1 = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    c2 = np.conj(c1[:20]) * 0.5
    N, L, sg = 8, 4.0, 0.5

    def grad(q, t):
        return orf.force_torque_fN(p1, c1, p2, c2, q, t, N, L, sg)

    q0 = np.array([0.95, 0.1, 0.2, -0.1])
    _, _, hist = orf.refine(grad, q0 / np.linalg.norm(q0), [0.1, -0.05, 0.08], 6, method, lr_t=0.005, lr_q=0.003)
    assert np.all(np.diff(hist) > 0), hist
