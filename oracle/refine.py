"""Oracle: local maximisation of the score from starting poses (Section 6).

TEST INFRASTRUCTURE.  Plain FP64 NumPy, used only by tests; shares no code with
the CUDA path.

Section 6 treats the score as the negative of a virtual energy, E(tau) ~ -f(tau),
so that the fixed solid exerts on the moving one the force F = -grad E, which
points up the score.  It uses that field two ways: a damped rigid-body dynamics
simulation (with inertia and damping coefficients it does not print) and
conjugate-gradient maximisation from many random starts.  The paper gives
neither update in formulas; the readings restated here are:

* the pose is (q, t), R = R(q / |q|) acting as x -> R x + t on the moving
  solid's samples about its frame origin;
* the generalised force is (F, T): F = d Re f / dt and the torque
  T = sum_j (R p2_j) x g_j, g_j = d Re f / dy at y_j = R p2_j + t, which is
  d Re f / d omega for the left perturbation R <- exp([omega]x) R;
* a rotation by the vector theta multiplies q on the left by the unit
  quaternion (cos |theta|/2, sin |theta|/2 theta/|theta|);
* ascent (the plain gradient step): t += lr_t F / max|F|, q += lr_q dq / max|dq|
  with dq = d Re f / dq, then q is normalised;
* conjugate gradient: Polak-Ribiere with restart (beta clipped at 0), kept
  separately for the translation block and the rotation block so that no
  length-to-angle scale is needed; each block moves a fixed length along its
  direction (lr_t for t, lr_q radians for R);
* dynamics: semi-implicit Euler with mass m, scalar moment of inertia I,
  damping factor gamma per step and time step h:
  v <- (1 - gamma) v + h F / m,  w <- (1 - gamma) w + h T / I,
  t <- t + h v,  q <- exp(h w) (x) q, starting at rest.
"""

from __future__ import annotations

import numpy as np

from . import score as oscore

ASCENT, CG, DYNAMICS = 0, 1, 2


def force_torque_fN(p1, c1, p2, c2, q, t, N, L, sigma_g, chunk=256):
    """Re f_N, the force dRe f/dt, the torque sum_j (R p2_j) x g_j and dRe f/dq, by pair sums."""
    p1 = np.asarray(p1, float)
    dim = p1.shape[1]
    R = oscore.rotation_matrix(q, dim)
    dR = oscore.rotation_matrix_grad(q, dim)
    p2 = np.asarray(p2, float)
    rp = p2 @ R.T
    y = rp + np.asarray(t, float)[:dim]
    f = 0j
    gy = np.zeros_like(y)
    for s in range(0, len(y), chunk):
        d = y[s:s + chunk, None, :] - p1[None, :, :]
        K1 = [oscore.kernel_1d(d[:, :, a], N, L, sigma_g) for a in range(dim)]
        dK1 = [oscore.kernel_1d(d[:, :, a], N, L, sigma_g, deriv=True) for a in range(dim)]
        cc = c2[s:s + chunk, None] * c1[None, :]
        f += (cc * np.prod(K1, axis=0)).sum()
        for a in range(dim):
            g = dK1[a]
            for b in range(dim):
                if b != a:
                    g = g * K1[b]
            gy[s:s + chunk, a] = np.real(cc * g).sum(1)
    F = np.zeros(3)
    F[:dim] = gy.sum(0)
    r3 = np.zeros((len(y), 3))
    g3 = np.zeros((len(y), 3))
    r3[:, :dim] = rp
    g3[:, :dim] = gy
    T = np.cross(r3, g3).sum(0)
    dq = np.array([(gy * (p2 @ dR[a].T)).sum() for a in range(4)])
    return f.real, F, T, dq


def quat_mul(a, b):
    """Hamilton product a (x) b of (w, x, y, z) quaternions."""
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw])


def rotate_left(q, theta):
    """exp(theta) (x) q for a rotation vector theta (3), normalised."""
    theta = np.asarray(theta, float)
    a = float(np.linalg.norm(theta))
    if a == 0.0:
        out = np.asarray(q, float)
    else:
        e = np.concatenate([[np.cos(a / 2)], np.sin(a / 2) * theta / a])
        out = quat_mul(e, q)
    return out / np.linalg.norm(out)


def refine(grad, q0, t0, steps, method, lr_t=0.05, lr_q=0.02, mass=1.0, inertia=1.0, damping=0.1, h=0.1):
    """Run `steps` updates from (q0, t0) with `grad(q, t) -> (f, F, T, dq)`.

    Returns (q, t, history of f before each step and after the last)."""
    q = np.asarray(q0, float).copy()
    t = np.zeros(3)
    t[:len(t0)] = t0
    hist = []
    g_prev = d_prev = None
    v = np.zeros(3)
    w = np.zeros(3)
    for k in range(steps + 1):
        f, F, T, dq = grad(q, t)
        hist.append(f)
        if k == steps:
            break
        if method == ASCENT:
            t = t + lr_t * F / max(np.abs(F).max(), 1e-30)
            q = q + lr_q * dq / max(np.abs(dq).max(), 1e-30)
            q = q / np.linalg.norm(q)
        elif method == CG:
            g = (F, T)
            if g_prev is None:
                d = g
            else:
                d = []
                for gb, gp, dp in zip(g, g_prev, d_prev):
                    den = float(gp @ gp)
                    beta = max(0.0, float(gb @ (gb - gp)) / den) if den > 0 else 0.0
                    d.append(gb + beta * dp)
                d = tuple(d)
            g_prev, d_prev = g, d
            nt, nr = np.linalg.norm(d[0]), np.linalg.norm(d[1])
            if nt > 0:
                t = t + lr_t * d[0] / nt
            if nr > 0:
                q = rotate_left(q, lr_q * d[1] / nr)
        elif method == DYNAMICS:
            v = (1.0 - damping) * v + h * F / mass
            w = (1.0 - damping) * w + h * T / inertia
            t = t + h * v
            q = rotate_left(q, h * w)
        else:
            raise ValueError(method)
    return q, t, np.array(hist)
