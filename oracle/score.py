"""Oracle: the complementarity score over rigid poses, its search and its gradient.

TEST INFRASTRUCTURE.  A plain FP64 NumPy restatement used only by tests, by the
smoke check and by the benchmark's CPU baseline; it shares no code with the CUDA
path and is deliberately slow.

Score (Eq. 1 / Eq. 8): f(tau) = integral of rho1(p) rho2(tau^-1 p) dv, with no
conjugate.  Each shape's SDF is carried by weighted samples (p_i, c_i) and
represented as rho(x) = sum_i c_i G_s(x - p_i) with the normalised isotropic
Gaussian G_s(x) = (2 pi s^2)^(-d/2) exp(-|x|^2 / (2 s^2)).  A pose tau = (R, t)
moves S2 as x -> R x + t.  Because G_s * G_s = G_{s sqrt 2}:

    f_c(R, t) = sum_ij c1_i c2_j G_{s sqrt 2}(R p2_j + t - p1_i).

The translation search of Section 5 evaluates, per rotation, the score on a
periodic grid with an FFT.  What that computes exactly is the band-limited
periodic score

    f_N(R, t) = sum_ij c1_i c2_j K_N(R p2_j + t - p1_i),
    K_N(x) = prod_d K_1(x_d),
    K_1(x) = (1/L) [1 + 2 sum_{m=1}^{N/2-1} exp(-s^2 (2 pi m / L)^2) cos(2 pi m x / L)],

i.e. the Gaussian's Fourier series on a box of side L truncated to |m| < N/2
(the Nyquist mode is left out so that K_1 is real and even).  In Fourier terms,
with k = 2 pi kappa / L:

    F1(kappa) = sum_i c1_i exp(-i k.p1_i),   F2(kappa) = sum_j c2_j exp(+i k.R p2_j),
    f_N(t) = L^-d sum_kappa exp(-s^2 |k|^2) F1 F2 exp(i k.t).

The score compared everywhere is Re f.  Translations are t_m = (i - N/2) h,
h = L/N, i in [0, N) per axis; arrays are indexed [iz, iy, ix] (3D) or [iy, ix]
(2D), so the C-order flat index is the translation index.
"""

from __future__ import annotations

import math

import numpy as np


# ---------------------------------------------------------------------------
# rotations (Hamilton quaternions (w, x, y, z), active)
# ---------------------------------------------------------------------------

def _quad_form(q):
    """M(q): the rotation matrix of q / |q| times |q|^2 (quadratic in q)."""
    w, x, y, z = q
    return np.array([
        [w * w + x * x - y * y - z * z, 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), w * w - x * x + y * y - z * z, 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), w * w - x * x - y * y + z * z]])


def rotation_matrix(q, dim=3):
    q = np.asarray(q, float)
    R = _quad_form(q) / float(q @ q)
    return R[:dim, :dim]


def rotation_matrix_grad(q, dim=3):
    """dR/dq_a for R(q / |q|), a = 0..3, from R = M(q)/|q|^2 with M quadratic."""
    q = np.asarray(q, float)
    n2 = float(q @ q)
    M = _quad_form(q)
    out = []
    for a in range(4):
        e = np.zeros(4)
        e[a] = 1.0
        dM = 0.5 * (_quad_form(q + e) - _quad_form(q - e))   # exact for a quadratic
        out.append((dM / n2 - 2.0 * q[a] * M / n2 ** 2)[:dim, :dim])
    return np.array(out)


# ---------------------------------------------------------------------------
# continuous score (closed form of two Gaussians)
# ---------------------------------------------------------------------------

def gauss(x2, s, dim):
    """Normalised isotropic Gaussian of width s at squared distance x2."""
    return (2 * math.pi * s * s) ** (-dim / 2) * np.exp(-x2 / (2 * s * s))


def pair_score_fc(p1, c1, p2, c2, q, t, sigma_g, chunk=2048):
    """Complex f_c(R, t) by direct pair sums."""
    p1 = np.asarray(p1, float)
    dim = p1.shape[1]
    y = np.asarray(p2, float) @ rotation_matrix(q, dim).T + np.asarray(t, float)[:dim]
    s2 = sigma_g * math.sqrt(2.0)
    tot = 0j
    for s in range(0, len(y), chunk):
        d = y[s:s + chunk, None, :] - p1[None, :, :]
        tot += (c2[s:s + chunk, None] * c1[None, :] * gauss((d * d).sum(2), s2, dim)).sum()
    return tot


def pair_grad_fc(p1, c1, p2, c2, q, t, sigma_g, chunk=1024):
    """Re f_c and its gradient w.r.t. t (dim) and the raw quaternion q (4)."""
    p1 = np.asarray(p1, float)
    dim = p1.shape[1]
    R = rotation_matrix(q, dim)
    dR = rotation_matrix_grad(q, dim)
    p2 = np.asarray(p2, float)
    y = p2 @ R.T + np.asarray(t, float)[:dim]
    s2 = sigma_g * math.sqrt(2.0)
    f = 0j
    gy = np.zeros_like(y)                  # d Re f / d y_j
    for s in range(0, len(y), chunk):
        d = y[s:s + chunk, None, :] - p1[None, :, :]
        G = c2[s:s + chunk, None] * c1[None, :] * gauss((d * d).sum(2), s2, dim)
        f += G.sum()
        gy[s:s + chunk] = (np.real(G)[:, :, None] * (-d / (s2 * s2))).sum(1)
    dt = gy.sum(0)
    dq = np.array([(gy * (p2 @ dR[a].T)).sum() for a in range(4)])
    return f.real, dt, dq


# ---------------------------------------------------------------------------
# band-limited periodic score
# ---------------------------------------------------------------------------

def kernel_1d(x, N, L, sigma_g, deriv=False):
    """K_1(x) (or dK_1/dx) as its cosine series."""
    m = np.arange(1, N // 2)
    k = 2 * math.pi * m / L
    a = np.exp(-(sigma_g * k) ** 2)
    x = np.asarray(x, float)[..., None]
    if deriv:
        return -(2.0 / L) * (a * k * np.sin(k * x)).sum(-1)
    return (1.0 / L) * (1.0 + 2.0 * (a * np.cos(k * x)).sum(-1))


def pair_score_fN(p1, c1, p2, c2, q, t, N, L, sigma_g, chunk=512):
    """Complex f_N(R, t) by direct pair sums over K_N (the second, definition route)."""
    p1 = np.asarray(p1, float)
    dim = p1.shape[1]
    y = np.asarray(p2, float) @ rotation_matrix(q, dim).T + np.asarray(t, float)[:dim]
    tot = 0j
    for s in range(0, len(y), chunk):
        d = y[s:s + chunk, None, :] - p1[None, :, :]
        K = np.ones(d.shape[:2])
        for a in range(dim):
            K = K * kernel_1d(d[:, :, a], N, L, sigma_g)
        tot += (c2[s:s + chunk, None] * c1[None, :] * K).sum()
    return tot


def pair_grad_fN(p1, c1, p2, c2, q, t, N, L, sigma_g, chunk=256):
    """Re f_N and its gradient w.r.t. t and the raw quaternion, by pair sums."""
    p1 = np.asarray(p1, float)
    dim = p1.shape[1]
    R = rotation_matrix(q, dim)
    dR = rotation_matrix_grad(q, dim)
    p2 = np.asarray(p2, float)
    y = p2 @ R.T + np.asarray(t, float)[:dim]
    f = 0j
    gy = np.zeros_like(y)
    for s in range(0, len(y), chunk):
        d = y[s:s + chunk, None, :] - p1[None, :, :]
        K1 = [kernel_1d(d[:, :, a], N, L, sigma_g) for a in range(dim)]
        dK1 = [kernel_1d(d[:, :, a], N, L, sigma_g, deriv=True) for a in range(dim)]
        cc = c2[s:s + chunk, None] * c1[None, :]
        K = np.prod(K1, axis=0)
        f += (cc * K).sum()
        for a in range(dim):
            g = dK1[a]
            for b in range(dim):
                if b != a:
                    g = g * K1[b]
            gy[s:s + chunk, a] = np.real(cc * g).sum(1)
    dt = gy.sum(0)
    dq = np.array([(gy * (p2 @ dR[a].T)).sum() for a in range(4)])
    return f.real, dt, dq


def _axis_modes(N):
    """Integer frequencies kappa at array positions 0..N-1 (kappa mod N order)."""
    return np.fft.fftfreq(N, d=1.0 / N).astype(int)


def nudft(points, c, N, L, sign):
    """F(kappa) = sum_j c_j exp(sign * i k.x_j), kappa in [-N/2, N/2)^d, k = 2 pi kappa / L.

    Direct sum (separable exponentials).  Output indexed [kz, ky, kx] (3D) or
    [ky, kx] (2D), each axis in kappa-mod-N order.
    """
    x = np.asarray(points, float)
    dim = x.shape[1]
    k = 2 * math.pi * _axis_modes(N) / L
    E = [np.exp(sign * 1j * np.outer(x[:, a], k)) for a in range(dim)]   # (M, N) each
    c = np.asarray(c, complex)
    if dim == 2:
        return (c[:, None] * E[1]).T @ E[0]
    out = np.empty((N, N, N), complex)
    for kz in range(N):
        out[kz] = ((c * E[2][:, kz])[:, None] * E[1]).T @ E[0]
    return out


def spectral_weight(N, L, sigma_g, dim):
    """exp(-s^2 |k|^2) / L^d on the mode grid, zero wherever a component is -N/2."""
    kap = _axis_modes(N)
    k = 2 * math.pi * kap / L
    g1 = np.exp(-(sigma_g * k) ** 2)
    g1[kap == -N // 2] = 0.0
    G = g1
    for _ in range(dim - 1):
        G = np.multiply.outer(G, g1)
    return G / L ** dim


def score_map_fN(p1, c1, p2, c2, q, N, L, sigma_g, F1=None, inverse="fft"):
    """Complex f_N on the translation grid for one rotation (spectral route).

    ``inverse="fft"`` uses numpy's FFT as the inverse DFT; ``"naive"`` evaluates
    the inverse DFT as a dense matrix product (small N only).
    """
    p1 = np.asarray(p1, float)
    dim = p1.shape[1]
    if F1 is None:
        F1 = nudft(p1, c1, N, L, -1)
    y = np.asarray(p2, float) @ rotation_matrix(q, dim).T
    F2 = nudft(y, c2, N, L, +1)
    P = spectral_weight(N, L, sigma_g, dim) * F1 * F2
    i = np.arange(N)
    kap = _axis_modes(N)
    if inverse == "fft":
        sgn = (-1.0) ** np.arange(N)
        S = sgn
        for _ in range(dim - 1):
            S = np.multiply.outer(S, sgn)
        return np.fft.ifftn(P * S) * N ** dim
    # naive: E[i, kappa] = exp(2 pi i kappa (i - N/2) / N), applied along every axis
    E = np.exp(2j * math.pi * np.outer(i - N // 2, kap) / N)
    out = P
    for ax in range(dim):
        out = np.moveaxis(np.tensordot(E, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out


def translations(N, L, dim):
    """t_m for every grid index, shaped like the map, last axis = (x, y[, z])."""
    h = L / N
    v = (np.arange(N) - N // 2) * h
    g = np.meshgrid(*([v] * dim), indexing="ij")    # g[0] varies along axis 0
    # axis 0 of the map is the slowest coordinate (z in 3D, y in 2D)
    return np.stack(g[::-1], -1)


def translation_of_index(idx, N, L, dim):
    h = L / N
    out = []
    for _ in range(dim):
        out.append((idx % N - N // 2) * h)
        idx //= N
    return np.array(out)


# ---------------------------------------------------------------------------
# search: per-rotation argmax and global top-k (Section 4, the argmax over T)
# ---------------------------------------------------------------------------

def rotation_best(re_map):
    """(max Re f, flat index), lowest index on ties."""
    flat = np.asarray(re_map).ravel()
    i = int(np.argmax(flat))
    return float(flat[i]), i


def global_top_k(scores, idxs, k):
    """Order (score desc, rotation asc, index asc) over per-rotation maxima; first k."""
    scores = np.asarray(scores, float)
    idxs = np.asarray(idxs)
    order = np.lexsort((idxs, np.arange(len(scores)), -scores))
    return [(int(r), float(scores[r]), int(idxs[r])) for r in order[:k]]


def score_rotations(p1, c1, p2, c2, quats, N, L, sigma_g, return_maps=False):
    """Per rotation: Re f_N map argmax.  Returns (best scores, best indices[, maps])."""
    p1 = np.asarray(p1, float)
    F1 = nudft(p1, c1, N, L, -1)
    best, idx, maps = [], [], []
    for q in quats:
        m = score_map_fN(p1, c1, p2, c2, q, N, L, sigma_g, F1=F1).real
        s, i = rotation_best(m)
        best.append(s)
        idx.append(i)
        if return_maps:
            maps.append(m)
    if return_maps:
        return np.array(best), np.array(idx), np.array(maps)
    return np.array(best), np.array(idx)
