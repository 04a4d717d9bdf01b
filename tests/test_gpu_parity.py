"""CUDA path (through the C ABI) against the CPU FP64 oracle, element by element.

Tolerances (max-norm relative error, max |gpu - oracle| / max |oracle|):
* FP32 path: 1e-4 for SDF values, score maps, scores and gradients.
* FP64 path: 1e-9 for SDF values; 2e-5 for maps and gradients, where the
  exponential-of-semicircle kernel of width 6 bounds the nonuniform FFT at ~2e-6.
Top-1 poses must be identical wherever the oracle's best and second-best scores
differ by more than 1e-4 of the map's maximum.
"""

import math

import numpy as np
import pytest
import torch

from helpers import cplx_to_pairs, oracle_maps, oracle_weights, rel_err, synthetic_weights
from oracle import score as oscore
from oracle import sdf as osdf
from paper_1712_00238_gb300 import sdfdock as sd
from synth import configs, rotations

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "f64": 2e-5}
LAM_DEFAULT = (1.0, 3.0, 0.5, 1.5)  # lambda1, lambda2, sigma_t, eps (Section 6)


def make_ctx(w, precision=None, **kw):
    prm = dict(lambda1=w.lam1, lambda2=w.lam2, sigma_t=w.sigma_t, eps=w.eps, sigma_g=w.sigma_g, w=w.w)
    prm.update(kw)
    return sd.Context(w.dim, precision or w.precision, 0, **prm)


def gpu_shape(ctx, s, return_rho=False):
    b, q = s.boundary, s.query
    return ctx.sdf_build(b.pos, b.normal, b.area, q.pos, q.vol, return_rho=return_rho)


def quats_dev(q):
    return torch.as_tensor(np.asarray(q, float), dtype=torch.float64, device="cuda").contiguous()


def grid_of(w, N=None):
    return sd.Grid(N or w.N, w.L)


def top1_margin_ok(ref_map):
    flat = np.sort(np.asarray(ref_map).ravel())[::-1]
    return flat[0] - flat[1] > 1e-4 * np.abs(flat).max()


# ---------------------------------------------------------------------------
# SDF (Eq. 10A-17t)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,prec,eps", [("tiny_2d", "f64", 1.5), ("tiny_2d", "f32", 1.5),
                                           ("tiny_3d", "f32", 1.5), ("tiny_3d", "f64", 1.5),
                                           ("tiny_3d", "f64", math.inf)])
def test_sdf_values_match_oracle(name, prec, eps):
    w = getattr(configs, name)()
    ctx = make_ctx(w, prec, eps=eps)
    for s in (w.fixed, w.moving):
        shape, rho = gpu_shape(ctx, s, return_rho=True)
        got = rho.cpu().numpy()
        got = got[:, 0] + 1j * got[:, 1]
        b = s.boundary
        ref = osdf.sdf_rho(s.query.pos, b.pos, b.normal, b.area, w.lam1, w.lam2, w.sigma_t, eps)
        tol = 1e-9 if prec == "f64" else 1e-4
        assert rel_err(got, ref) < tol
        assert shape.m == s.query.m
        assert abs(shape.radius - np.linalg.norm(s.query.pos, axis=1).max()) < 1e-5 * shape.radius
    ctx.close()


@pytest.mark.parametrize("name,prec", [("tiny_2d", "f64"), ("tiny_3d", "f32"), ("tiny_3d", "f64")])
@pytest.mark.parametrize("phi", ["proximal", "radial", "skin"])
def test_other_phi_kernels_match_oracle(name, prec, phi):
    # the proximal, radial and skin / core kernels of Section 4 through the same build
    w = getattr(configs, name)()
    code = {"proximal": sd.PHI_PROXIMAL, "radial": sd.PHI_RADIAL, "skin": sd.PHI_SKIN}[phi]
    radius = 0.35
    ctx = make_ctx(w, prec, phi=code, phi_radius=radius)
    for s in (w.fixed, w.moving):
        _, rho = gpu_shape(ctx, s, return_rho=True)
        got = rho.cpu().numpy()
        got = got[:, 0] + 1j * got[:, 1]
        b = s.boundary
        ref = osdf.rho_variant(s.query.pos, b.pos, b.normal, b.area, code, radius, w.lam1, w.lam2, w.sigma_t)
        assert rel_err(got, ref) < (1e-9 if prec == "f64" else 1e-4), phi
    ctx.close()
    with pytest.raises(sd.SdError):
        make_ctx(w, prec, phi=9)
    with pytest.raises(sd.SdError):
        make_ctx(w, prec, phi=code, phi_radius=0.0)


def test_sdf_full_size_sampled_points():
    # 3D peg-in-bore shapes at full size (20,000 boundary samples, ~50,000 query
    # points); the oracle evaluates a seeded sample of the query points.
    w = configs.peg_in_bore_3d()
    ctx = make_ctx(w)
    rng = np.random.default_rng(0)
    for s in (w.fixed, w.moving):
        _, rho = gpu_shape(ctx, s, return_rho=True)
        got = rho.cpu().numpy()
        sel = rng.choice(s.query.m, 300, replace=False)
        b = s.boundary
        ref = osdf.sdf_rho(s.query.pos[sel], b.pos, b.normal, b.area, **w.sdf_params())
        assert rel_err(got[sel, 0] + 1j * got[sel, 1], ref) < 1e-4
    ctx.close()


# ---------------------------------------------------------------------------
# score maps and per-rotation argmax
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,prec,N", [("tiny_2d", "f64", 32), ("tiny_2d", "f32", 48), ("tiny_3d", "f32", 16),
                                         ("tiny_3d", "f32", 24), ("tiny_3d", "f64", 32)])
def test_maps_match_oracle_all_rotations(name, prec, N):
    w = getattr(configs, name)()
    p1, c1, p2, c2 = oracle_weights(name)
    ctx = make_ctx(w, prec)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    q = quats_dev(w.quats)
    g = grid_of(w, N)
    maps = ctx.score_maps(fx, mv, q, g).cpu().numpy()
    ref = oracle_maps(p1, c1, p2, c2, w.quats, N, w.L, w.sigma_g)
    for r in range(w.n_rot):
        assert rel_err(maps[r], ref[r]) < TOL[prec], r
    cand = ctx.score_rotations(fx, mv, q, g)
    s, rot, idx = (t.cpu().numpy() for t in sd.decode_cands(cand))
    assert np.array_equal(rot, np.arange(w.n_rot))
    # the argmax pass runs the same transforms as the map pass; spreading
    # accumulates with float atomics, so two runs agree to rounding only
    run_tol = 1e-12 if prec == "f64" else 1e-6
    for r in range(w.n_rot):
        mr = maps[r].real
        assert abs(s[r] - mr.max()) <= run_tol * np.abs(mr).max()
        top2 = np.sort(mr)[-2:]
        if top2[1] - top2[0] > 10 * run_tol * np.abs(mr).max():
            assert idx[r] == int(np.argmax(mr))
        if top1_margin_ok(ref[r].real):
            assert idx[r] == int(np.argmax(ref[r].real))
    ctx.close()


@pytest.mark.parametrize("name,N,swap", [("tiny_2d", 48, False), ("tiny_3d", 16, False), ("tiny_3d", 32, False),
                                         ("tiny_3d", 8, True)])
def test_binned_spreading_matches_oracle(name, N, swap):
    # spread by 8^d-cell bins with warp-cooperative shared-memory tiles; with the
    # block as the moving shape on the 8^3 grid the sub-box is the whole periodic
    # 16^3 grid, so tiles wrap around its faces
    w = getattr(configs, name)()
    p1, c1, p2, c2 = oracle_weights(name)
    if swap:
        p1, c1, p2, c2 = p2, c2, p1, c1
    ctx = make_ctx(w, "f32")
    ctx.set_option("spread_direct", 0)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    q = quats_dev(w.quats)
    g = grid_of(w, N)
    maps = ctx.score_maps(fx, mv, q, g).cpu().numpy()
    ref = oracle_maps(p1, c1, p2, c2, w.quats, N, w.L, w.sigma_g)
    for r in range(w.n_rot):
        assert rel_err(maps[r], ref[r]) < TOL["f32"], r
    s, rot, idx = (t.cpu().numpy() for t in sd.decode_cands(ctx.score_rotations(fx, mv, q, g)))
    for r in range(w.n_rot):
        assert abs(s[r] - maps[r].real.max()) <= 1e-6 * np.abs(maps[r].real).max()
        if top1_margin_ok(ref[r].real):
            assert idx[r] == int(np.argmax(ref[r].real))
    ctx.close()


@pytest.mark.parametrize("name,N,swap", [("tiny_2d", 48, False), ("tiny_3d", 16, False), ("tiny_3d", 48, False),
                                         ("tiny_3d", 8, True)])
def test_box_spreading_matches_oracle(name, N, swap):
    # each CTA spreads 128 Morton-consecutive samples into a shared box; with the
    # block as the moving shape on the 8^3 grid the sub-box is the whole periodic
    # grid and boxes that wrap take the global-atomic path
    w = getattr(configs, name)()
    p1, c1, p2, c2 = oracle_weights(name)
    if swap:
        p1, c1, p2, c2 = p2, c2, p1, c1
    ctx = make_ctx(w, "f32")
    ctx.set_option("spread_box", 1)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    q = quats_dev(w.quats)
    g = grid_of(w, N)
    assert ctx.search_plan(mv, g, w.n_rot)["spread_bins"] == 2
    maps = ctx.score_maps(fx, mv, q, g).cpu().numpy()
    ref = oracle_maps(p1, c1, p2, c2, w.quats, N, w.L, w.sigma_g)
    for r in range(w.n_rot):
        assert rel_err(maps[r], ref[r]) < TOL["f32"], r
    s, rot, idx = (t.cpu().numpy() for t in sd.decode_cands(ctx.score_rotations(fx, mv, q, g)))
    for r in range(w.n_rot):
        assert abs(s[r] - maps[r].real.max()) <= 1e-6 * np.abs(maps[r].real).max()
        if top1_margin_ok(ref[r].real):
            assert idx[r] == int(np.argmax(ref[r].real))
    ctx.close()


def _sub_box(radius, N, L, w):
    # side of the moving shape's sub-box on the oversampled grid n = 2N
    n = 2 * N
    s_h = int(math.floor(radius * n / L + 0.5 * w)) + 2
    return n if 2 * s_h >= n else 2 * s_h


@pytest.mark.parametrize("name,prec,N", [("tiny_3d", "f32", 48), ("tiny_3d", "f64", 64), ("tiny_2d", "f64", 32),
                                         ("tiny_2d", "f32", 64), ("tiny_3d", "f32", 64)])
def test_pruned_and_full_forward_passes_agree(name, prec, N):
    # The pruned forward passes read the sub-box unshifted and compute only the
    # kept modes, applying the shift as a phase in the product table; the full
    # passes read the shifted sub-box and compute every mode; the narrow and wide
    # plans are the pruned one with half / twice the columns per CTA (FP32, n
    # from 128 to 384).  Same maps,
    # and all equal the oracle's.  (tiny_3d at N = 48 has s = N exactly, the
    # largest sub-box the pruned path takes; n = 96 ends with radix 12, n = 64 /
    # 128 with 8.)
    w = getattr(configs, name)()
    p1, c1, p2, c2 = oracle_weights(name)
    s = _sub_box(float(np.linalg.norm(p2, axis=1).max()), N, w.L, w.w)
    assert s <= N, "the pruned path needs the sub-box in the low half of a line"
    ctx = make_ctx(w, prec)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    q = quats_dev(w.quats)
    g = grid_of(w, N)
    alt = prec == "f32" and 128 <= 2 * N <= 384
    got = {}
    for plan in (1, 0, 2, 3):
        ctx.set_option("fft_plan", plan)
        # a plan that does not apply falls back to the pruned default
        assert ctx.search_plan(mv, g, w.n_rot)["fft_plan"] == (plan if plan < 2 or alt else 1)
        got[plan] = ctx.score_maps(fx, mv, q, g).cpu().numpy()
    ctx.set_option("fft_plan", -1)
    ref = oracle_maps(p1, c1, p2, c2, w.quats, N, w.L, w.sigma_g)
    for r in range(w.n_rot):
        assert rel_err(got[1][r], got[0][r]) < (1e-12 if prec == "f64" else 2e-6), r
        for alt_plan in (2, 3):
            assert rel_err(got[alt_plan][r], got[1][r]) < (1e-12 if prec == "f64" else 2e-6), (alt_plan, r)
        assert rel_err(got[1][r], ref[r]) < TOL[prec], r
    ctx.close()


@pytest.mark.parametrize("N", [48, 64])
def test_fused_spreading_matches_oracle(N):
    # spreading fused with the forward x transform: each CTA accumulates whole
    # x rows of a (y, z) block in shared memory and transforms them there
    # (tiny_3d: N = 48 puts the sub-box at s = N, the edge of the pruned path)
    w = configs.tiny_3d()
    p1, c1, p2, c2 = oracle_weights("tiny_3d")
    ctx = make_ctx(w, "f32")
    ctx.set_option("spread_fused", 1)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    q = quats_dev(w.quats)
    g = grid_of(w, N)
    assert ctx.search_plan(mv, g, w.n_rot)["spread_bins"] == 1
    maps = ctx.score_maps(fx, mv, q, g).cpu().numpy()
    ref = oracle_maps(p1, c1, p2, c2, w.quats, N, w.L, w.sigma_g)
    for r in range(w.n_rot):
        assert rel_err(maps[r], ref[r]) < TOL["f32"], r
    s, rot, idx = (t.cpu().numpy() for t in sd.decode_cands(ctx.score_rotations(fx, mv, q, g)))
    for r in range(w.n_rot):
        assert abs(s[r] - maps[r].real.max()) <= 1e-6 * np.abs(maps[r].real).max()
        if top1_margin_ok(ref[r].real):
            assert idx[r] == int(np.argmax(ref[r].real))
    # the same maps as the other spreading paths (fixed point, so exact up to FP32 rounding of the passes)
    ctx.set_option("spread_fused", 0)
    other = ctx.score_maps(fx, mv, q, g).cpu().numpy()
    for r in range(w.n_rot):
        assert rel_err(maps[r], other[r]) < 2e-6, r
    ctx.close()


@pytest.mark.parametrize("N", [32, 48, 64, 96])
def test_cluster_inverse_matches_oracle(N):
    # inverse y and x of each z-plane in one kernel (a cluster of CTAs sharing the
    # plane through distributed shared memory) against the oracle's maps and the
    # two-pass inverse; the argmax candidates come from the same kernel
    w = configs.tiny_3d()
    p1, c1, p2, c2 = oracle_weights("tiny_3d")
    ctx = make_ctx(w, "f32")
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    q = quats_dev(w.quats)
    g = grid_of(w, N)
    got = {}
    for on in (1, 0):
        ctx.set_option("inverse_cluster", on)
        ctx.set_option("timing", 1)
        ctx.pass_times(reset=True)
        maps = ctx.score_maps(fx, mv, q, g).cpu().numpy()
        cands = [t.cpu().numpy() for t in sd.decode_cands(ctx.score_rotations(fx, mv, q, g))]
        t = ctx.pass_times()
        # the cluster pass ran instead of the inverse y and x passes (and only then)
        assert (t["inv_yx"][0] > 0) == bool(on) and (t["inv_y"][0] > 0) == (not on)
        got[on] = (maps, cands)
    ref = oracle_maps(p1, c1, p2, c2, w.quats, N, w.L, w.sigma_g)
    maps, (s, rot, idx) = got[1]
    for r in range(w.n_rot):
        assert rel_err(maps[r], ref[r]) < TOL["f32"], r
        assert rel_err(maps[r], got[0][0][r]) < 2e-6, r
        assert abs(s[r] - maps[r].real.max()) <= 1e-6 * np.abs(maps[r].real).max()
        if top1_margin_ok(ref[r].real):
            assert idx[r] == int(np.argmax(ref[r].real)) == got[0][1][2][r]
    ctx.close()


def test_maps_full_size_peg_in_bore():
    # 128^3 translations, n = 256 oversampled grid, ~50,000 samples per shape;
    # weights are seeded synthetic values shared by both sides.
    w = configs.peg_in_bore_3d()
    p1, p2 = w.fixed.query.pos, w.moving.query.pos
    c1 = synthetic_weights(len(p1), 1) * 1e-3
    c2 = synthetic_weights(len(p2), 2) * 1e-3
    ctx = make_ctx(w)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    sel = [0, 137, 402]
    q = quats_dev(w.quats[sel])
    maps = ctx.score_maps(fx, mv, q, grid_of(w)).cpu().numpy()
    ref = oracle_maps(p1, c1, p2, c2, w.quats[sel], w.N, w.L, w.sigma_g)
    for r in range(len(sel)):
        assert rel_err(maps[r], ref[r]) < 1e-4
        if top1_margin_ok(ref[r].real):
            assert int(np.argmax(maps[r].real)) == int(np.argmax(ref[r].real))
    ctx.close()


def test_end_to_end_peg_in_hole_2d_fp64():
    # boundary samples -> SDF -> 64 rotations x 128^2 translations, FP64
    w = configs.peg_in_hole_2d()
    ctx = make_ctx(w)
    fx = gpu_shape(ctx, w.fixed)
    mv = gpu_shape(ctx, w.moving)
    q = quats_dev(w.quats)
    g = grid_of(w)
    maps = ctx.score_maps(fx, mv, q, g).cpu().numpy()
    p1, c1, p2, c2 = oracle_weights("peg_in_hole_2d")
    ref = oracle_maps(p1, c1, p2, c2, w.quats, w.N, w.L, w.sigma_g)
    assert max(rel_err(maps[r], ref[r]) for r in range(w.n_rot)) < TOL["f64"]
    cand = ctx.score_rotations(fx, mv, q, g)
    poses = ctx.top_k_poses(cand, 4, fx, mv, q, g, rescore_fp64=True)
    best_r = [oscore.rotation_best(m.real) for m in ref]
    ref_top = oscore.global_top_k([b[0] for b in best_r], [b[1] for b in best_r], 4)
    assert [(p["rot"], p["idx"]) for p in poses] == [(r, i) for r, _, i in ref_top]
    assert poses[0]["rot"] % 16 == 0 and np.allclose(poses[0]["t"], 0.0)
    for p, (r, _, i) in zip(poses, ref_top):
        t = oscore.translation_of_index(i, w.N, w.L, 2)
        fc = oscore.pair_score_fc(p1, c1, p2, c2, w.quats[r], t, w.sigma_g)
        assert abs(p["score_fp64"] - fc.real) < 1e-9 * abs(fc)
    ctx.close()


def test_batching_graph_and_plain_paths_agree():
    w = configs.tiny_3d()
    p1, c1, p2, c2 = oracle_weights("tiny_3d")
    ctx = make_ctx(w)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    q = quats_dev(w.quats)
    g = grid_of(w)
    ref = ctx.score_maps(fx, mv, q, g).cpu().numpy()
    base = sd.decode_cands(ctx.score_rotations(fx, mv, q, g))
    outs = []
    for opt in ({"batch": 5}, {"plain": 1}, {"batch": 4, "graph": 1}):
        for k, v in opt.items():
            ctx.set_option(k, v)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            for _ in range(3):   # eager, then captured, then replayed
                cand = ctx.score_rotations(fx, mv, q, g)
        st.synchronize()
        outs.append(sd.decode_cands(cand))
        for k in opt:
            ctx.set_option(k, 0)
    for s, rot, idx in outs:
        assert torch.equal(rot, base[1])
        assert (s - base[0]).abs().max().item() <= 1e-5 * np.abs(ref.real).max()
        for r in range(w.n_rot):
            if top1_margin_ok(ref[r].real):
                assert idx[r].item() == base[2][r].item()
    ctx.close()


# ---------------------------------------------------------------------------
# top-k and FP64 re-score
# ---------------------------------------------------------------------------

def test_top_k_and_fp64_rescore_tiny_3d():
    w = configs.tiny_3d()
    p1, c1, p2, c2 = oracle_weights("tiny_3d")
    ctx = make_ctx(w)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    q = quats_dev(w.quats)
    g = grid_of(w)
    poses = ctx.top_k_poses(ctx.score_rotations(fx, mv, q, g), 3, fx, mv, q, g)
    ref = oracle_maps(p1, c1, p2, c2, w.quats, w.N, w.L, w.sigma_g)
    best = [oscore.rotation_best(m.real) for m in ref]
    ref_top = oscore.global_top_k([b[0] for b in best], [b[1] for b in best], 3)
    scale = max(abs(b[0]) for b in best)
    for p, (r, sc, i) in zip(poses, ref_top):
        assert abs(p["score"] - sc) < 1e-4 * scale
    gaps = np.diff([-x[1] for x in ref_top])
    if np.all(gaps > 1e-4 * scale):
        assert [(p["rot"], p["idx"]) for p in poses] == [(r, i) for r, _, i in ref_top]
        for p, (r, _, i) in zip(poses, ref_top):
            t = oscore.translation_of_index(i, w.N, w.L, 3)
            fc = oscore.pair_score_fc(p1, c1, p2, c2, w.quats[r], t, w.sigma_g)
            # FP64 sums of the shape's FP32-stored positions and weights
            assert abs(p["score_fp64"] - fc.real) < 1e-6 * abs(fc)
            assert abs(p["score_fp64_im"] - fc.imag) < 1e-6 * abs(fc)
    ctx.close()


# ---------------------------------------------------------------------------
# score and gradient at arbitrary poses (type-2 gather)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,prec,N", [("tiny_3d", "f32", 16), ("tiny_3d", "f64", 24), ("tiny_2d", "f64", 32),
                                         ("tiny_2d", "f32", 32)])
def test_score_grad_matches_oracle(name, prec, N):
    w = getattr(configs, name)()
    p1, c1, p2, c2 = oracle_weights(name)
    ctx = make_ctx(w, prec)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    P = 6
    if w.dim == 3:
        qs = rotations.random_uniform(P, 11)
    else:
        th = np.linspace(0.3, 5.0, P)
        qs = np.stack([np.cos(th / 2), 0 * th, 0 * th, np.sin(th / 2)], 1)
    qs = qs * np.linspace(0.7, 1.3, P)[:, None]          # unnormalised on purpose
    ts = rotations.random_ball(P, 1.0, 12, 3)
    if w.dim == 2:
        ts[:, 2] = 0
    real = torch.float64 if prec == "f64" else torch.float32
    s, dq, dt = ctx.score_grad(fx, mv, grid_of(w, N), torch.tensor(qs, dtype=real, device="cuda"),
                               torch.tensor(ts, dtype=real, device="cuda"))
    s, dq, dt = s.cpu().numpy(), dq.cpu().numpy(), dt.cpu().numpy()
    ref = [oscore.pair_grad_fN(p1, c1, p2, c2, qs[i], ts[i, : w.dim], N, w.L, w.sigma_g) for i in range(P)]
    fs = np.array([r[0] for r in ref])
    rdt = np.array([r[1] for r in ref])
    rdq = np.array([r[2] for r in ref])
    tol = TOL[prec]
    assert rel_err(s, fs) < tol
    assert rel_err(dt, rdt) < tol
    assert rel_err(dq, rdq) < tol
    assert np.abs((dq * qs).sum(1)).max() < 1e-4 * np.abs(dq).max()
    ctx.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_score_grad_at_the_refinement_grid(prec):
    # the refinement workload's grid (docking pair, N = 192 on L = 153.6, n = 384,
    # sigma_g = 0.6) on seeded 64 x 64-sample subsets of its SDF samples with
    # seeded weights: score and gradient at 8 poses against the oracle's pair sums
    # over the band-limited kernel (each axis a cosine series)
    w = configs.docking_2000_500(n_rot=1)
    rng = np.random.default_rng(64)
    p1 = w.fixed.query.pos[np.sort(rng.choice(w.fixed.query.m, 64, replace=False))]
    p2 = w.moving.query.pos[np.sort(rng.choice(w.moving.query.m, 64, replace=False))]
    c1, c2 = synthetic_weights(64, 5), synthetic_weights(64, 6)
    ctx = sd.Context(3, prec, 0, sigma_g=w.sigma_g)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    P = 8
    qs = rotations.random_uniform(P, 21)
    # each pose puts one seeded pair of samples within 0.3 A of each other, so the
    # scores carry Gaussian peaks and not only the band limit's ripple
    a_i, b_i = rng.integers(0, 64, P), rng.integers(0, 64, P)
    off = rotations.random_ball(P, 0.3, 22, 3)
    ts = np.stack([p1[a_i[i]] - oscore.rotation_matrix(qs[i], 3) @ p2[b_i[i]] + off[i] for i in range(P)])
    real = torch.float64 if prec == "f64" else torch.float32
    s, dq, dt = ctx.score_grad(fx, mv, sd.Grid(w.N, w.L), torch.tensor(qs, dtype=real, device="cuda"),
                               torch.tensor(ts, dtype=real, device="cuda"))
    s, dq, dt = s.cpu().numpy(), dq.cpu().numpy(), dt.cpu().numpy()
    ref = [oscore.pair_grad_fN(p1, c1, p2, c2, qs[i], ts[i], w.N, w.L, w.sigma_g) for i in range(P)]
    tol = TOL[prec]
    assert rel_err(s, np.array([r[0] for r in ref])) < tol
    assert rel_err(dt, np.array([r[1] for r in ref])) < tol
    assert rel_err(dq, np.array([r[2] for r in ref])) < tol
    ctx.close()


def test_score_grad_equals_map_on_grid_points():
    w = configs.tiny_3d()
    p1, c1, p2, c2 = oracle_weights("tiny_3d")
    ctx = make_ctx(w, "f64")
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    g = grid_of(w, 16)
    q = quats_dev(w.quats[:2])
    maps = ctx.score_maps(fx, mv, q, g).cpu().numpy()
    idx = np.array([0, 77, 1000, 4095])
    qs = np.repeat(w.quats[:2], len(idx), 0)
    ts = np.array([oscore.translation_of_index(int(i), 16, w.L, 3) for i in idx] * 2)
    s, _, _ = ctx.score_grad(fx, mv, g, torch.tensor(qs, device="cuda"), torch.tensor(ts, device="cuda"))
    want = np.concatenate([maps[0].real[idx], maps[1].real[idx]])
    assert np.abs(s.cpu().numpy() - want).max() < 2e-5 * np.abs(maps.real).max()
    ctx.close()


def test_autograd_function_and_refinement():
    # backward returns the analytic gradient (checked against the oracle above);
    # central differences of the interpolated score agree up to the derivative
    # of the interpolation error (about 1e-3 of the largest gradient at h = 1e-3)
    w = configs.tiny_3d()
    p1, c1, p2, c2 = oracle_weights("tiny_3d")
    ctx = make_ctx(w, "f64")
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    g = grid_of(w, 16)
    q = torch.tensor(rotations.random_uniform(3, 5), device="cuda", requires_grad=True)
    t = torch.tensor(rotations.random_ball(3, 1.0, 6, 3), device="cuda", requires_grad=True)
    s = sd.sdf_score(ctx, fx, mv, g, q, t)
    gq, gt = torch.autograd.grad(s.sum(), (q, t))
    s2, dq2, dt2 = ctx.score_grad(fx, mv, g, q.detach(), t.detach())
    # per-pose sums accumulate across blocks with FP64 atomics: equal to rounding
    for a, b in ((s, s2), (gq, dq2), (gt, dt2)):
        assert (a.detach() - b).abs().max().item() <= 1e-12 * b.abs().max().item()
    h = 1e-3
    for a in range(3):
        e = torch.zeros_like(t)
        e[:, a] = h
        fd = (ctx.score_grad(fx, mv, g, q.detach(), t.detach() + e)[0]
              - ctx.score_grad(fx, mv, g, q.detach(), t.detach() - e)[0]) / (2 * h)
        assert (fd - gt[:, a]).abs().max().item() < 2e-3 * gt.abs().max().item()
    for a in range(4):
        e = torch.zeros_like(q)
        e[:, a] = h
        fd = (ctx.score_grad(fx, mv, g, q.detach() + e, t.detach())[0]
              - ctx.score_grad(fx, mv, g, q.detach() - e, t.detach())[0]) / (2 * h)
        assert (fd - gq[:, a]).abs().max().item() < 2e-3 * gq.abs().max().item()
    q1, t1, hist = sd.refine_poses(ctx, fx, mv, g, q.detach(), t.detach(), steps=20, lr_t=0.02, lr_q=0.01)
    assert (hist[-1] >= hist[0]).all()
    ctx.close()


@pytest.mark.parametrize("name,method", [("tiny_3d", "cg"), ("tiny_3d", "dynamics"), ("tiny_2d", "cg"),
                                         ("tiny_2d", "dynamics")])
def test_refine_rules_match_oracle(name, method):
    # the device's conjugate-gradient and damped-dynamics updates against the
    # oracle's rules driven by the oracle's own pair-sum force and torque
    from oracle import refine as orf

    w = getattr(configs, name)()
    p1, c1, p2, c2 = oracle_weights(name)
    ctx = make_ctx(w, "f64")
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    N = 16
    g = grid_of(w, N)
    P, steps = 2, 4
    if w.dim == 3:
        q0 = rotations.random_uniform(P, 9)
        t0 = rotations.random_ball(P, 0.8, 10, 3)
    else:
        q0 = rotations.planar(7)[[1, 4]]
        t0 = rotations.random_ball(P, 0.8, 10, 2)
    kw = dict(lr_t=0.03, lr_q=0.02) if method == "cg" else dict(mass=2.0, inertia=3.0, damping=0.2, dt=0.05)
    code = sd.REFINE_CG if method == "cg" else sd.REFINE_DYNAMICS
    qd = torch.tensor(q0, device="cuda", dtype=torch.float64)
    td = torch.tensor(t0, device="cuda", dtype=torch.float64)
    qg, tg, hg = ctx.refine(fx, mv, g, qd, td, steps, method=code, **kw)
    qg, tg, hg = qg.cpu().numpy(), tg.cpu().numpy(), hg.cpu().numpy()

    def grad(q, t):
        return orf.force_torque_fN(p1, c1, p2, c2, q, t[: w.dim], N, w.L, w.sigma_g)

    okw = dict(lr_t=kw.get("lr_t", 0), lr_q=kw.get("lr_q", 0), mass=kw.get("mass", 1), inertia=kw.get("inertia", 1),
               damping=kw.get("damping", 0), h=kw.get("dt", 0))
    for i in range(P):
        qo, to, ho = orf.refine(grad, q0[i], t0[i], steps, orf.CG if method == "cg" else orf.DYNAMICS, **okw)
        scale = np.abs(ho).max()
        assert np.abs(hg[:, i] - ho).max() <= 1e-4 * scale, (i, hg[:, i], ho)
        sign = 1.0 if float(qg[i] @ qo) >= 0 else -1.0  # q and -q are one rotation
        assert np.abs(qg[i] - sign * qo).max() < 1e-5
        assert np.abs(tg[i] - to[: w.dim]).max() < 1e-5
    with pytest.raises(sd.SdError) as e:
        ctx.refine(fx, mv, g, qd, td, 1, method=7)
    assert e.value.code == sd.SD_ERR_ARG
    with pytest.raises(sd.SdError) as e:
        ctx.refine(fx, mv, g, qd, td, 1, method=sd.REFINE_DYNAMICS, mass=0.0)
    assert e.value.code == sd.SD_ERR_ARG
    ctx.close()


@pytest.mark.parametrize("name,prec", [("tiny_3d", "f64"), ("tiny_3d", "f32"), ("tiny_2d", "f64"), ("tiny_2d", "f32")])
def test_device_ascent_matches_oracle(name, prec):
    # the device's gradient-ascent rule (sd_refine with SD_REFINE_ASCENT, which
    # sd_refine_poses runs) against the oracle's ascent driven by the oracle's
    # own pair-sum force and dq
    from oracle import refine as orf

    w = getattr(configs, name)()
    p1, c1, p2, c2 = oracle_weights(name)
    ctx = make_ctx(w, prec)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    N = 16
    g = grid_of(w, N)
    P, steps, lr_t, lr_q = 3, 5, 0.03, 0.02
    if w.dim == 3:
        q0 = rotations.random_uniform(P, 19)
        t0 = rotations.random_ball(P, 0.8, 20, 3)
    else:
        q0 = rotations.planar(9)[[1, 4, 7]]
        t0 = rotations.random_ball(P, 0.8, 20, 2)
    real = torch.float64 if prec == "f64" else torch.float32
    qd = torch.tensor(q0, device="cuda", dtype=real)
    td = torch.tensor(t0, device="cuda", dtype=real)
    qg, tg, hg = ctx.refine(fx, mv, g, qd, td, steps, method=sd.REFINE_ASCENT, lr_t=lr_t, lr_q=lr_q)
    qn, tn, hn = ctx.refine_poses(fx, mv, g, qd, td, steps=steps, lr_t=lr_t, lr_q=lr_q)
    qg, tg, hg = qg.cpu().double().numpy(), tg.cpu().double().numpy(), hg.cpu().double().numpy()

    def grad(q, t):
        return orf.force_torque_fN(p1, c1, p2, c2, q, t[: w.dim], N, w.L, w.sigma_g)

    tol, ptol = (2e-5, 1e-5) if prec == "f64" else (1e-4, 1e-4)
    for i in range(P):
        qo, to, ho = orf.refine(grad, q0[i], t0[i], steps, orf.ASCENT, lr_t=lr_t, lr_q=lr_q)
        scale = np.abs(ho).max()
        assert np.abs(hg[:, i] - ho).max() <= tol * scale, (i, hg[:, i], ho)
        sign = 1.0 if float(qg[i] @ qo) >= 0 else -1.0
        assert np.abs(qg[i] - sign * qo).max() < ptol, (i, qg[i], qo)
        assert np.abs(tg[i] - to[: w.dim]).max() < ptol, (i, tg[i], to)
    # sd_refine_poses is the same rule
    assert np.abs(hn.cpu().double().numpy() - hg).max() <= 1e-12 * np.abs(hg).max() + (0 if prec == "f64" else 1e-6)
    ctx.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_native_refinement_follows_autograd_path(prec):
    # sd_refine_poses runs the same ascent rule on the device (update arithmetic
    # in FP64); its trajectory must follow the autograd loop's
    w = configs.tiny_3d()
    p1, c1, p2, c2 = oracle_weights("tiny_3d")
    ctx = make_ctx(w, prec)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    g = grid_of(w, 16)
    real = torch.float64 if prec == "f64" else torch.float32
    q0 = torch.tensor(rotations.random_uniform(4, 7), device="cuda", dtype=real)
    t0 = torch.tensor(rotations.random_ball(4, 1.0, 8, 3), device="cuda", dtype=real)
    steps = 12
    qa, ta, ha = sd.refine_poses(ctx, fx, mv, g, q0, t0, steps=steps, lr_t=0.02, lr_q=0.01)
    qn, tn, hn = ctx.refine_poses(fx, mv, g, q0, t0, steps=steps, lr_t=0.02, lr_q=0.01)
    s0 = ctx.score_grad(fx, mv, g, q0, t0)[0]
    scale = ha.abs().max().item()
    tol = 1e-9 if prec == "f64" else 1e-4
    assert (hn[0] - s0).abs().max().item() <= 1e-12 * scale + (0 if prec == "f64" else 1e-6 * scale)
    assert hn.shape == (steps + 1, 4)
    assert (hn - ha).abs().max().item() <= tol * scale
    assert (qn - qa).abs().max().item() <= (1e-9 if prec == "f64" else 1e-4)
    assert (tn - ta).abs().max().item() <= (1e-9 if prec == "f64" else 1e-4)
    assert torch.allclose(qn.norm(dim=1), torch.ones(4, device="cuda", dtype=real), atol=1e-6)
    assert (hn[-1] >= hn[0]).all()
    # q0 and t0 are inputs only
    assert torch.equal(q0, torch.tensor(rotations.random_uniform(4, 7), device="cuda", dtype=real))
    ctx.close()


# ---------------------------------------------------------------------------
# errors
# ---------------------------------------------------------------------------

def test_degenerate_inputs():
    # an empty rotation list writes nothing; a one-sample moving shape still matches the oracle
    w = configs.tiny_3d()
    rng = np.random.default_rng(91)
    p1 = w.fixed.query.pos
    c1 = rng.standard_normal(len(p1)) + 1j * rng.standard_normal(len(p1))
    p2 = np.array([[0.3, -0.2, 0.1]])
    c2 = np.array([0.7 - 0.4j])
    ctx = make_ctx(w)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    empty = torch.empty((0, 4), dtype=torch.float64, device="cuda")
    assert ctx.score_rotations(fx, mv, empty, grid_of(w, 16)).shape[0] == 0
    quats = rotations.super_fibonacci(40)[[0, 9]]
    maps = ctx.score_maps(fx, mv, quats_dev(quats), grid_of(w, 16)).cpu().numpy()
    ref = oracle_maps(p1, c1, p2, c2, quats, 16, w.L, w.sigma_g)
    for r in range(2):
        assert rel_err(maps[r], ref[r]) < 1e-4
    ctx.close()


@pytest.mark.parametrize("name,prec,N", [("tiny_3d", "f32", 48), ("tiny_3d", "f64", 32), ("tiny_2d", "f32", 64),
                                         ("tiny_2d", "f64", 32)])
def test_ties_go_to_the_lowest_translation_index(name, prec, N):
    # zero moving weights: every translation scores exactly 0, so each rotation's
    # best is translation 0 and its k_r best are 0, 1, 2, ... (ties by index), on
    # every path that ends in an argmax (two-pass inverse, cluster inverse, top-K)
    w = getattr(configs, name)()
    p1, c1, p2, _ = oracle_weights(name)
    ctx = make_ctx(w, prec)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(np.zeros(len(p2), complex)))
    q = quats_dev(w.quats)
    g = grid_of(w, N)
    for cluster in ((0, 1) if (w.dim == 3 and prec == "f32") else (0,)):
        ctx.set_option("inverse_cluster", cluster)
        s, rot, idx = (t.cpu().numpy() for t in sd.decode_cands(ctx.score_rotations(fx, mv, q, g)))
        assert (s == 0).all() and (idx == 0).all(), cluster
    ctx.set_option("inverse_cluster", 0)
    k_r = 5
    s, rot, idx = (t.cpu().numpy() for t in sd.decode_cands(ctx.score_rotations(fx, mv, q, g, k_r=k_r)))
    assert (s == 0).all()
    assert (idx.reshape(-1, k_r) == np.arange(k_r)[None, :]).all()
    ctx.close()


def test_argument_errors_are_reported():
    w = configs.tiny_3d()
    p1, c1, p2, c2 = oracle_weights("tiny_3d")
    ctx = make_ctx(w)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    q = quats_dev(w.quats)
    with pytest.raises(sd.SdError) as e:
        ctx.score_rotations(fx, mv, q, sd.Grid(100, w.L))
    assert e.value.code == sd.SD_ERR_ARG
    for bad_k in (0, 17):
        with pytest.raises(sd.SdError) as e:
            ctx.score_rotations(fx, mv, q, grid_of(w), k_r=bad_k)
        assert e.value.code == sd.SD_ERR_ARG
    with pytest.raises(sd.SdError):
        ctx.score_rotations(fx, mv, q, sd.Grid(32, -1.0))
    other = make_ctx(w)
    ofx = other.shape_from_samples(p1, cplx_to_pairs(c1))
    with pytest.raises(sd.SdError) as e:
        ctx.score_rotations(ofx, mv, q, grid_of(w))
    assert "another context" in str(e.value)
    # the context stays usable after errors
    cand = ctx.score_rotations(fx, mv, q, grid_of(w))
    assert torch.isfinite(sd.decode_cands(cand)[0]).all()
    other.close()
    ctx.close()


# ---------------------------------------------------------------------------
# docking-shaped inputs: grids with radix-3 line lengths (96 -> 192, 192 -> 384)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N,L,n1,n2", [(96, 77.4, 3000, 1200), (192, 153.6, 1500, 600)])
def test_maps_docking_grids(N, L, n1, n2):
    # a small sphere-union pair (200 and 60 spheres); seeded subsets of its SDF
    # sample positions carry seeded synthetic weights
    fx_in, mv_in = configs.docking_pair(200, 60, 5)
    rng = np.random.default_rng(N)
    p1 = fx_in.query.pos[np.sort(rng.choice(fx_in.query.m, n1, replace=False))]
    p2 = mv_in.query.pos[np.sort(rng.choice(mv_in.query.m, n2, replace=False))]
    c1 = synthetic_weights(n1, 3)
    c2 = synthetic_weights(n2, 4)
    sg = 0.6
    ctx = sd.Context(3, "f32", 0, sigma_g=sg)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    quats = rotations.super_fibonacci(40)[[3, 17]]
    q = quats_dev(quats)
    g = sd.Grid(N, L)
    ref = oracle_maps(p1, c1, p2, c2, quats, N, L, sg)
    for direct in (1, 0):  # global vector atomics, then binned shared-memory tiles
        ctx.set_option("spread_direct", direct)
        maps = ctx.score_maps(fx, mv, q, g).cpu().numpy()
        cand = sd.decode_cands(ctx.score_rotations(fx, mv, q, g))
        for r in range(len(quats)):
            assert rel_err(maps[r], ref[r]) < 1e-4, (direct, r)
            if top1_margin_ok(ref[r].real):
                assert cand[2][r].item() == int(np.argmax(ref[r].real)), (direct, r)
    ctx.close()


def test_maps_largest_grid_sampled_translations():
    # N = 256 (512-point lines, the two-CTA register bound): the map at sampled
    # translations, the GPU argmax among them, against the oracle's direct pair sums
    fx_in, mv_in = configs.docking_pair(200, 60, 5)
    rng = np.random.default_rng(256)
    n1, n2 = 700, 300
    p1 = fx_in.query.pos[np.sort(rng.choice(fx_in.query.m, n1, replace=False))]
    p2 = mv_in.query.pos[np.sort(rng.choice(mv_in.query.m, n2, replace=False))]
    c1 = synthetic_weights(n1, 7)
    c2 = synthetic_weights(n2, 8)
    N, L, sg = 256, 204.8, 0.6
    ctx = sd.Context(3, "f32", 0, sigma_g=sg)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    quat = rotations.super_fibonacci(40)[[11]]
    maps = ctx.score_maps(fx, mv, quats_dev(quat), sd.Grid(N, L)).cpu().numpy()[0]
    cand = sd.decode_cands(ctx.score_rotations(fx, mv, quats_dev(quat), sd.Grid(N, L)))
    top = int(cand[2][0].item())
    assert top == int(np.argmax(maps.real))
    # the top and translations within three cells of it (where the map is far from zero)
    tz, ty, tx = top // (N * N), (top // N) % N, top % N
    near = [((tz + dz) % N) * N * N + ((ty + dy) % N) * N + (tx + dx) % N
            for dz, dy, dx in rng.integers(-3, 4, (8, 3))]
    idx = np.concatenate([[top], near])
    h = L / N
    scale = np.abs(maps.real).max()
    for i in idx:
        t = np.array([i % N - N // 2, (i // N) % N - N // 2, i // (N * N) - N // 2], float) * h
        ref = oscore.pair_score_fN(p1, c1, p2, c2, quat[0], t, N, L, sg)
        assert abs(maps[i] - ref) < 1e-4 * scale, i
    ctx.close()


def test_sdf_docking_pair_sampled_points():
    fx_in, mv_in = configs.docking_pair(200, 60, 5)
    ctx = sd.Context(3, "f32", 0, sigma_g=0.6)
    rng = np.random.default_rng(1)
    for s in (fx_in, mv_in):
        _, rho = gpu_shape(ctx, s, return_rho=True)
        got = rho.cpu().numpy()
        sel = rng.choice(s.query.m, 300, replace=False)
        b = s.boundary
        ref = osdf.sdf_rho(s.query.pos[sel], b.pos, b.normal, b.area, LAM_DEFAULT[0], LAM_DEFAULT[1],
                           LAM_DEFAULT[2], LAM_DEFAULT[3])
        assert rel_err(got[sel, 0] + 1j * got[sel, 1], ref) < 1e-4
    ctx.close()


def test_alu_peak_probe_rates_are_plausible():
    # the probe behind the ALU rooflines: rates are positive and ordered as the
    # hardware is built (FP32 FMA far above FP64 FMA; ex2 at least as fast as rsqrt)
    rates = {k: sd.alu_peak(k) for k in sd.PEAK_KINDS}
    assert all(v > 0 for v in rates.values())
    assert rates["fp32_fma"] > 10 * rates["fp64_fma"]
    assert rates["sfu_ex2"] >= 0.5 * rates["sfu_rsqrt"]
    lib = sd.load()
    import ctypes as ct
    v = ct.c_double()
    assert lib.sd_alu_peak(0, 9, ct.byref(v)) == sd.SD_ERR_ARG


def test_sdf_cull_levels_agree_on_a_large_shape():
    # the eps-neighbour restriction of the SDF sums (boundary tiles beyond the
    # truncation radius of a block's queries, 32-sample sub-tiles beyond a warp's)
    # skips only pairs that Eq. 17t drops: the sums are the same to the bit, at
    # the top of the uneven batch's size range (~2e5 queries x ~3e5 samples)
    s = configs.large_sphere_shape()
    w = configs.docking_2000_500()
    ctx = make_ctx(w)
    rhos = {}
    for level in (2, 1, 0):
        ctx.set_option("sdf_cull", level)
        _, rho = gpu_shape(ctx, s, return_rho=True)
        rhos[level] = rho.cpu().numpy()
    assert np.array_equal(rhos[2], rhos[1]) and np.array_equal(rhos[2], rhos[0])
    rng = np.random.default_rng(5)
    sel = rng.choice(s.query.m, 200, replace=False)
    b = s.boundary
    ref = osdf.sdf_rho(s.query.pos[sel], b.pos, b.normal, b.area, **w.sdf_params())
    assert rel_err(rhos[2][sel, 0] + 1j * rhos[2][sel, 1], ref) < 1e-4
    ctx.close()


@pytest.mark.parametrize("name,prec,N,k_r", [("tiny_3d", "f32", 16, 5), ("tiny_3d", "f32", 48, 16),
                                             ("tiny_2d", "f64", 32, 3), ("tiny_2d", "f32", 8, 12)])
def test_several_candidates_per_rotation(name, prec, N, k_r):
    # k_r > 1: the k_r best translations of every rotation, score descending then
    # index ascending, against the same maps and the oracle's
    w = getattr(configs, name)()
    p1, c1, p2, c2 = oracle_weights(name)
    ctx = make_ctx(w, prec)
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    q = quats_dev(w.quats)
    g = grid_of(w, N)
    maps = ctx.score_maps(fx, mv, q, g).cpu().numpy().real
    ref = oracle_maps(p1, c1, p2, c2, w.quats, N, w.L, w.sigma_g).real
    s, rot, idx = (t.cpu().numpy().reshape(w.n_rot, k_r) for t in sd.decode_cands(ctx.score_rotations(fx, mv, q, g,
                                                                                                      k_r=k_r)))
    run_tol = 1e-12 if prec == "f64" else 1e-6
    for r in range(w.n_rot):
        assert np.all(rot[r] == r)
        order = np.lexsort((np.arange(maps[r].size), -maps[r]))[:k_r]
        scale = np.abs(maps[r]).max()
        # the scores are the map's k_r largest, in order
        assert np.all(np.diff(s[r]) <= 0)
        assert np.allclose(s[r], maps[r][order], rtol=0, atol=run_tol * scale)
        # the same translations wherever consecutive values are separated
        srt = maps[r][order]
        gaps = -np.diff(np.append(srt, np.sort(maps[r])[::-1][k_r]))
        for k in range(k_r):
            if gaps[k] > 10 * run_tol * scale and (k == 0 or gaps[k - 1] > 10 * run_tol * scale):
                assert idx[r, k] == order[k], (r, k)
        # and the oracle's, where its margins exceed the path's tolerance
        ro = np.lexsort((np.arange(ref[r].size), -ref[r]))[:k_r + 1]
        rs = ref[r][ro]
        tol = TOL[prec] * np.abs(ref[r]).max()
        for k in range(k_r):
            if rs[k] - rs[k + 1] > 2 * tol and (k == 0 or rs[k - 1] - rs[k] > 2 * tol):
                assert idx[r, k] == ro[k], (r, k)
    # the global top-k over all of them
    cand = ctx.score_rotations(fx, mv, q, g, k_r=k_r)
    s2, rot2, idx2 = (t.cpu().numpy() for t in sd.decode_cands(cand))
    poses = ctx.top_k_poses(cand, 4, fx, mv, q, g, rescore_fp64=False)
    flat = np.lexsort((idx2, rot2, -s2))[:4]
    assert [(p["rot"], p["idx"]) for p in poses] == [(int(rot2[i]), int(idx2[i])) for i in flat]
    ctx.close()
