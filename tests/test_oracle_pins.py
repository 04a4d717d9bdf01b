"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form
derived from the definitions, an invariance the paper states, a textbook
identity, a numerical integral of the defining integral, or brute force.
"""

import math

import numpy as np
import pytest
from scipy import integrate

from oracle import score, sdf
from synth import configs, rotations

LAM1, LAM2, SIG, EPS = 1.0, 3.0, 0.5, 1.5


def _sphere_samples(n, radius, rng, dim):
    v = rng.standard_normal((n, dim))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    meas = (4 * math.pi * radius ** 2) if dim == 3 else (2 * math.pi * radius)
    return radius * v, v, np.full(n, meas / n)


# --- Eq. 13/15/16c: centre of a sphere or circle ---------------------------------

@pytest.mark.parametrize("dim,radius,n", [(3, 1.7, 2000), (3, 0.3, 517), (2, 0.8, 300), (2, 2.5, 77)])
def test_centre_of_sphere_is_i_lambda2_over_sigma(dim, radius, n):
    # every sample is a nearest neighbour (r = 1, E = 1, cos(theta) = -1), so
    # rho = i * lambda2 / sigma exactly for any sampling density and radius
    rng = np.random.default_rng(n)
    q, nrm, a = _sphere_samples(n, radius, rng, dim)
    rho = sdf.sdf_rho(np.zeros((1, dim)), q, nrm, a, LAM1, LAM2, SIG, EPS)
    assert abs(rho[0] - 1j * LAM2 / SIG) < 1e-12


# --- Prop. 1 (Eq. 17B/17C): flat boundary, closed radial integral ----------------

def _plate_integral(eps, dim):
    # exterior value; the interior one is (lambda2/lambda1) * conj(exterior)
    up = 1 + eps if np.isfinite(eps) else 1 + 12 * SIG
    if dim == 3:
        f = lambda r, part: part(np.exp(-0.5 * ((r - 1) / SIG) ** 2) * np.exp(-2j * np.arctan(r)) / (1 + r * r))
        re = integrate.quad(lambda r: f(r, np.real), 1, up, limit=200)[0]
        im = integrate.quad(lambda r: f(r, np.imag), 1, up, limit=200)[0]
        return LAM1 / SIG * (re + 1j * im)
    # planar: gamma(r) = 2 arccos(1/r), so rho = (2 lambda/(pi sigma)) int E r e^{-2i atan r} /
    # ((1 + r^2) sqrt(r^2 - 1)) dr; r = cosh(u) removes the 1/sqrt singularity
    g = lambda u, part: part(np.exp(-0.5 * ((np.cosh(u) - 1) / SIG) ** 2) * np.cosh(u)
                             * np.exp(-2j * np.arctan(np.cosh(u))) / (1 + np.cosh(u) ** 2))
    umax = np.arccosh(up)
    re = integrate.quad(lambda u: g(u, np.real), 0, umax, limit=200)[0]
    im = integrate.quad(lambda u: g(u, np.imag), 0, umax, limit=200)[0]
    return 2 * LAM1 / (math.pi * SIG) * (re + 1j * im)


@pytest.mark.parametrize("eps", [np.inf, EPS])
def test_flat_plate_3d_matches_radial_integral(eps):
    hg = 0.04
    xs = np.arange(-12, 12, hg) + hg / 2
    X, Y = np.meshgrid(xs, xs)
    q = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1)
    nrm = np.tile([0.0, 0.0, 1.0], (len(q), 1))
    a = np.full(len(q), hg * hg)
    ext = _plate_integral(eps, 3)
    for h in (0.4, 0.8):
        r_out = sdf.sdf_rho(np.array([[0.013, -0.007, h]]), q, nrm, a, LAM1, LAM2, SIG, eps,
                            pmc_values=np.array([1.0]))[0]
        r_in = sdf.sdf_rho(np.array([[0.013, -0.007, -h]]), q, nrm, a, LAM1, LAM2, SIG, eps,
                           pmc_values=np.array([-1.0]))[0]
        assert abs(r_out - ext) < 4e-3 * abs(ext)
        assert abs(r_in - (LAM2 / LAM1) * np.conj(ext)) < 4e-3 * abs(ext) * LAM2
        # Table 1 phases: exterior ~ -i lambda1, interior ~ +i lambda2
        assert r_out.imag < 0 < r_in.imag


@pytest.mark.parametrize("eps", [np.inf, EPS])
def test_flat_line_2d_matches_planar_integral(eps):
    hg = 0.0005
    xs = np.arange(-40, 40, hg) + hg / 2
    q = np.stack([xs, np.zeros_like(xs)], 1)
    nrm = np.tile([0.0, 1.0], (len(q), 1))
    a = np.full(len(q), hg)
    ext = _plate_integral(eps, 2)
    r_out = sdf.sdf_rho(np.array([[0.0, 1.0]]), q, nrm, a, LAM1, LAM2, SIG, eps,
                        pmc_values=np.array([1.0]))[0]
    assert abs(r_out - ext) < 3e-3 * abs(ext)


# --- Prop. 2 (Eq. 18b): truncation error bound -----------------------------------

def test_truncation_error_bound():
    w = configs.tiny_3d()
    b = w.moving.boundary
    p = w.moving.query.pos[::7]
    full = sdf.sdf_rho(p, b.pos, b.normal, b.area, LAM1, LAM2, SIG, np.inf)
    for eps in (0.5, 1.0, 1.5):
        cut = sdf.sdf_rho(p, b.pos, b.normal, b.area, LAM1, LAM2, SIG, eps)
        d = p[:, None, :] - b.pos[None]
        eta = np.linalg.norm(d, axis=2)
        cos = np.abs((d * b.normal[None]).sum(2)) / eta
        gamma_abs = (cos * b.area[None] / eta ** 2).sum(1)      # unsigned solid angle (sr)
        bound = LAM2 / (2 * math.pi * SIG) * math.exp(-0.5 * (eps / SIG) ** 2) * gamma_abs
        assert np.all(np.abs(full - cut) <= bound * (1 + 1e-9))
        assert np.any(np.abs(full - cut) > 0)


# --- Section 4: invariance of rho under rigid motion, and membership -------------

def test_rho_equivariant_under_rigid_motion():
    w = configs.tiny_3d()
    b = w.fixed.boundary
    p = w.fixed.query.pos[::11]
    Q = score.rotation_matrix(np.array([0.3, -0.5, 0.7, 0.2]))
    a = np.array([1.5, -2.0, 0.25])
    r0 = sdf.sdf_rho(p, b.pos, b.normal, b.area, LAM1, LAM2, SIG, EPS)
    r1 = sdf.sdf_rho(p @ Q.T + a, b.pos @ Q.T + a, b.normal @ Q.T, b.area, LAM1, LAM2, SIG, EPS)
    assert np.max(np.abs(r1 - r0)) < 1e-12 * np.max(np.abs(r0))


@pytest.mark.parametrize("which", ["tiny_2d", "tiny_3d"])
def test_membership_matches_analytic_solid(which):
    w = getattr(configs, which)()
    for s in (w.fixed, w.moving):
        pm = sdf.pmc(s.query.pos, s.boundary.pos, s.boundary.normal, s.boundary.area)
        assert np.array_equal(pm < 0, s.query.inside)


def test_nearest_distance_bounds_true_distance():
    rng = np.random.default_rng(3)
    q, nrm, a = _sphere_samples(4000, 1.0, rng, 3)
    p = rng.standard_normal((50, 3)) * 2
    d = sdf.nearest_distance(p, q)
    true = np.abs(np.linalg.norm(p, axis=1) - 1.0)
    assert np.all(d >= true - 1e-12)
    assert np.all(d <= true + 0.08)


# --- Eq. 8 with Gaussian-represented SDFs ---------------------------------------

def test_gaussian_self_correlation_is_wider_gaussian():
    s = 0.3
    hg = 0.01
    xs = np.arange(-4, 4, hg)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    for a, b in (([0.0, 0.0], [0.0, 0.0]), ([0.2, -0.1], [-0.3, 0.4]), ([0.5, 0.5], [-0.2, 0.0])):
        g1 = score.gauss((X - a[0]) ** 2 + (Y - a[1]) ** 2, s, 2)
        g2 = score.gauss((X - b[0]) ** 2 + (Y - b[1]) ** 2, s, 2)
        num = (g1 * g2).sum() * hg * hg
        ref = math.exp(-((a[0] - b[0]) ** 2 + (a[1] - b[1]) ** 2) / (4 * s * s)) / (4 * math.pi * s * s)
        assert abs(num - ref) < 1e-9 * ref


def test_pair_score_matches_eq8_integral_2d():
    # f(tau) = integral of rho1(p) rho2(tau^-1 p) dv, tau^-1 p = R^T (p - t)
    rng = np.random.default_rng(5)
    s = 0.25
    p1 = rng.uniform(-1, 1, (4, 2))
    c1 = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    p2 = rng.uniform(-1, 1, (3, 2))
    c2 = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    th = 0.7
    q = np.array([math.cos(th / 2), 0, 0, math.sin(th / 2)])
    t = np.array([0.3, -0.2])
    hg = 0.01
    xs = np.arange(-4, 4, hg)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    P = np.stack([X, Y], -1)
    rho1 = sum(c * score.gauss(((P - pi) ** 2).sum(-1), s, 2) for pi, c in zip(p1, c1))
    Rm = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    Pb = (P - t) @ Rm          # rows: R^T (p - t)
    rho2 = sum(c * score.gauss(((Pb - pj) ** 2).sum(-1), s, 2) for pj, c in zip(p2, c2))
    num = (rho1 * rho2).sum() * hg * hg
    ref = score.pair_score_fc(p1, c1, p2, c2, q, t, s)
    assert abs(num - ref) < 1e-8 * abs(ref)


def test_pair_score_invariant_under_joint_motion():
    rng = np.random.default_rng(6)
    p1 = rng.standard_normal((40, 3))
    c1 = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    p2 = rng.standard_normal((30, 3))
    c2 = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    q = np.array([0.9, 0.1, -0.3, 0.2])
    t = np.array([0.2, 0.1, -0.4])
    Qq = np.array([0.4, 0.5, -0.1, 0.7])
    Q = score.rotation_matrix(Qq)
    a = np.array([3.0, -1.0, 2.0])
    f0 = score.pair_score_fc(p1, c1, p2, c2, q, t, 0.4)
    # moving S1 by (Q, a) and composing the pose with it leaves f unchanged
    qc = np.array([Qq[0] * q[0] - Qq[1:] @ q[1:], *(Qq[0] * q[1:] + q[0] * Qq[1:] + np.cross(Qq[1:], q[1:]))])
    f1 = score.pair_score_fc(p1 @ Q.T + a, c1, p2, c2, qc, Q @ t + a, 0.4)
    assert abs(f1 - f0) < 1e-12 * abs(f0)


# --- band-limited periodic score (the FFT search) --------------------------------

def _rand_pair(w, n1, n2, seed):
    rng = np.random.default_rng(seed)
    p1 = w.fixed.query.pos[rng.choice(w.fixed.query.m, n1, replace=False)]
    p2 = w.moving.query.pos[rng.choice(w.moving.query.m, n2, replace=False)]
    c1 = rng.standard_normal(n1) + 1j * rng.standard_normal(n1)
    c2 = rng.standard_normal(n2) + 1j * rng.standard_normal(n2)
    return p1, c1, p2, c2


@pytest.mark.parametrize("which,N", [("tiny_2d", 16), ("tiny_2d", 24), ("tiny_3d", 8), ("tiny_3d", 12)])
def test_score_map_routes_agree(which, N):
    w = getattr(configs, which)()
    p1, c1, p2, c2 = _rand_pair(w, 60, 40, N)
    q = w.quats[3]
    dim = w.dim
    m_fft = score.score_map_fN(p1, c1, p2, c2, q, N, w.L, 0.4)
    m_naive = score.score_map_fN(p1, c1, p2, c2, q, N, w.L, 0.4, inverse="naive")
    scale = np.abs(m_fft).max()
    assert np.abs(m_fft - m_naive).max() < 1e-12 * scale
    rng = np.random.default_rng(0)
    for idx in rng.choice(N ** dim, 6, replace=False):
        t = score.translation_of_index(int(idx), N, w.L, dim)
        direct = score.pair_score_fN(p1, c1, p2, c2, q, t, N, w.L, 0.4)
        assert abs(m_fft.ravel()[idx] - direct) < 1e-11 * scale


def test_band_limited_score_converges_to_continuous():
    w = configs.tiny_3d()
    p1, c1, p2, c2 = _rand_pair(w, 50, 40, 2)
    q, t = w.quats[5], np.array([0.3, -0.2, 0.1])
    # box side 40 >> support, Gaussian resolved (sigma/h = 1.6 at N = 64)
    fc = score.pair_score_fc(p1, c1, p2, c2, q, t, 1.0)
    errs = [abs(score.pair_score_fN(p1, c1, p2, c2, q, t, N, 40.0, 1.0) - fc) for N in (16, 32, 64)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-9 * abs(fc)


def test_nudft_on_grid_nodes_is_the_dft():
    rng = np.random.default_rng(9)
    N, L = 12, 3.0
    h = L / N
    g = rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))   # [iz, iy, ix]
    iz, iy, ix = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    pts = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], 1) * h
    F = score.nudft(pts, g.ravel(), N, L, -1)
    assert np.abs(F - np.fft.fftn(g)).max() < 1e-10 * np.abs(F).max()
    assert abs(F[0, 0, 0] - g.sum()) < 1e-10 * abs(g.sum())
    Fp = score.nudft(pts, g.ravel(), N, L, +1)
    assert np.abs(Fp - np.fft.ifftn(g) * N ** 3).max() < 1e-10 * np.abs(Fp).max()
    # Parseval
    assert abs((np.abs(g) ** 2).sum() - (np.abs(F) ** 2).sum() / N ** 3) < 1e-9 * (np.abs(g) ** 2).sum()


def test_score_map_shift_equivariance():
    w = configs.tiny_2d()
    p1, c1, p2, c2 = _rand_pair(w, 50, 30, 4)
    N = 16
    h = w.L / N
    q = w.quats[2]
    m0 = score.score_map_fN(p1, c1, p2, c2, q, N, w.L, 0.4)
    m1 = score.score_map_fN(p1 + np.array([2 * h, -3 * h]), c1, p2, c2, q, N, w.L, 0.4)
    # moving S1 by a grid vector shifts the map by the same number of cells
    assert np.abs(np.roll(m0, (-3, 2), axis=(0, 1)) - m1).max() < 1e-12 * np.abs(m0).max()


# --- gradients -------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_gradients_match_central_differences(dim):
    w = configs.tiny_3d() if dim == 3 else configs.tiny_2d()
    p1, c1, p2, c2 = _rand_pair(w, 40, 30, 7)
    q = np.array([0.8, 0.0, 0.0, 0.6]) if dim == 2 else np.array([0.7, 0.3, -0.4, 0.5])
    t = np.array([0.2, -0.1, 0.05])[:dim]
    N, L, s = 16, w.L, 0.5
    for fn, gfn in ((lambda qq, tt: score.pair_score_fc(p1, c1, p2, c2, qq, tt, s).real,
                     lambda: score.pair_grad_fc(p1, c1, p2, c2, q, t, s)),
                    (lambda qq, tt: score.pair_score_fN(p1, c1, p2, c2, qq, tt, N, L, s).real,
                     lambda: score.pair_grad_fN(p1, c1, p2, c2, q, t, N, L, s))):
        f, dt, dq = gfn()
        assert abs(f - fn(q, t)) < 1e-12 * max(1.0, abs(f))
        e = 1e-5
        for a in range(dim):
            dd = np.zeros(dim)
            dd[a] = e
            fd = (fn(q, t + dd) - fn(q, t - dd)) / (2 * e)
            assert abs(fd - dt[a]) < 1e-6 * (np.abs(dt).max() + 1e-30)
        for a in range(4):
            dd = np.zeros(4)
            dd[a] = e
            fd = (fn(q + dd, t) - fn(q - dd, t)) / (2 * e)
            assert abs(fd - dq[a]) < 1e-6 * (np.abs(dq).max() + 1e-30)
        assert abs(dq @ q) < 1e-10 * np.abs(dq).max()    # scale invariance of R(q/|q|)


# --- search ----------------------------------------------------------------------

def test_global_top_k_order_brute_force():
    rng = np.random.default_rng(1)
    s = rng.integers(0, 5, 200).astype(float)       # many exact ties
    idx = rng.integers(0, 1000, 200)
    got = score.global_top_k(s, idx, 50)
    ref = sorted(range(200), key=lambda r: (-s[r], r, idx[r]))[:50]
    assert [g[0] for g in got] == ref


def test_peg_in_hole_top1_is_the_inserted_pose():
    # Section 6 behaviour: the correct pairing is the global maximum.  For the
    # square peg and hole it is t = 0 at a multiple of 90 degrees.
    w = configs.peg_in_hole_2d()
    cs = []
    for s in (w.fixed, w.moving):
        b = s.boundary
        rho = sdf.sdf_rho(s.query.pos, b.pos, b.normal, b.area, **w.sdf_params())
        cs.append((s.query.pos, rho * s.query.vol))
    (p1, c1), (p2, c2) = cs
    best, idx = score.score_rotations(p1, c1, p2, c2, w.quats, w.N, w.L, w.sigma_g)
    r, sc, i = score.global_top_k(best, idx, 1)[0]
    assert r % 16 == 0
    assert np.allclose(score.translation_of_index(i, w.N, w.L, 2), 0.0)
    # a 45-degree peg cannot enter the hole and scores lower
    assert best[8] < 0.9 * sc


# --- rotation sets -----------------------------------------------------------------

def test_rotation_sets():
    th, ph = rotations.healpix_centres(2)
    z = np.cos(th)
    assert len(z) == 48 and abs(z.sum()) < 1e-12
    # equal-area rings: 4*nside-1 = 7 distinct latitudes
    assert len(np.unique(np.round(z, 12))) == 7
    for q in (rotations.hopf_grid(2, 12), rotations.super_fibonacci(500), rotations.random_uniform(300, 3)):
        assert np.allclose(np.linalg.norm(q, axis=1), 1.0)
    g = rotations.hopf_grid(2, 12)
    assert len(g) == 576
    ang = 2 * np.arccos(np.clip(np.abs(g @ g.T), 0, 1)) + 4 * np.eye(len(g))
    assert ang.min() > np.deg2rad(10)        # distinct rotations, none repeated


def test_optimum_score_trends_of_section_6():
    # Section 6's parameter study, as loose behaviour checks on the 2D peg-in-hole pair at
    # the inserted pose: the optimal score scales roughly like 1 / sigma_t, and at a fixed
    # product lambda1 lambda2 it hardly depends on the penalty factor lambda2 / lambda1 >= 3
    w = configs.peg_in_hole_2d()

    def f_opt(lam1, lam2, st):
        cs = []
        for s in (w.fixed, w.moving):
            b = s.boundary
            cs.append(sdf.sdf_rho(s.query.pos, b.pos, b.normal, b.area, lam1, lam2, st, 1.5) * s.query.vol)
        return score.pair_score_fc(w.fixed.query.pos, cs[0], w.moving.query.pos, cs[1],
                                    np.array([1.0, 0, 0, 0]), np.zeros(2), w.sigma_g).real

    f = {st: f_opt(1.0, 3.0, st) for st in (0.25, 0.5, 1.0)}
    assert 1.5 < f[0.25] / f[0.5] < 2.5 and 1.5 < f[0.5] / f[1.0] < 2.5
    base = f[0.5]
    for pen in (6.0, 12.0):
        g = f_opt(np.sqrt(3.0 / pen), np.sqrt(3.0 * pen), 0.5)
        assert abs(g - base) <= 0.01 * abs(base)
