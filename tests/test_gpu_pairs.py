"""Many shape pairs scored in one launch sequence (sd_score_pairs), autotuned.

Jobs of different grids and sample counts share a context.  Each job's
per-rotation candidates must equal those of sd_score_rotations for the same
pair: rotations identical, scores within FP32 rounding of the spreading's
atomic order (1e-5 of the map's maximum), translations identical wherever the
top-1 margin exceeds 1e-4 of the map's maximum.  This holds on the eager call,
the captured call and the replay of the graph; one job's scores are also held
against the oracle's maps.
"""

import numpy as np
import pytest
import torch

from helpers import cplx_to_pairs, oracle_maps, oracle_weights, rel_err, synthetic_weights
from paper_1712_00238_gb300 import sdfdock as sd
from synth import configs, rotations

pytestmark = pytest.mark.gpu

SIGMA_G = 0.6


def _quats(q):
    return torch.as_tensor(np.asarray(q, float), dtype=torch.float64, device="cuda").contiguous()


def _margin_ok(m):
    flat = np.sort(np.asarray(m).ravel())[::-1]
    return flat[0] - flat[1] > 1e-4 * np.abs(flat).max()


def _jobs(ctx):
    w = configs.tiny_3d()
    p1, c1, p2, c2 = oracle_weights("tiny_3d")
    a_fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    a_mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    fx_in, mv_in = configs.docking_pair(200, 60, 5)
    rng = np.random.default_rng(11)
    d1 = fx_in.query.pos[np.sort(rng.choice(fx_in.query.m, 2000, replace=False))]
    d2 = mv_in.query.pos[np.sort(rng.choice(mv_in.query.m, 800, replace=False))]
    b_fx = ctx.shape_from_samples(d1, cplx_to_pairs(synthetic_weights(2000, 5)))
    b_mv = ctx.shape_from_samples(d2, cplx_to_pairs(synthetic_weights(800, 6)))
    sf = rotations.super_fibonacci(40)
    specs = [  # (fixed, moving, rotations, grid, oracle inputs or None)
        (a_fx, a_mv, w.quats, sd.Grid(32, w.L), (p1, c1, p2, c2)),
        (a_fx, a_mv, sf[:7], sd.Grid(48, w.L), None),
        (b_fx, b_mv, sf[5:14], sd.Grid(96, 77.4), None),
        (b_mv, a_mv, sf[20:25], sd.Grid(64, 40.0), None),
    ]
    return specs


def test_score_pairs_equals_per_pair_search_and_replays():
    ctx = sd.Context(3, "f32", 0, sigma_g=SIGMA_G)
    specs = _jobs(ctx)
    jobs, refs, maps = [], [], []
    for fx, mv, q, g, _ in specs:
        qd = _quats(q)
        jobs.append((fx, mv, qd, g))
        refs.append(sd.decode_cands(ctx.score_rotations(fx, mv, qd, g)))
        maps.append(ctx.score_maps(fx, mv, qd, g).cpu().numpy())
    # the oracle pins job 0's maps (and so its candidates, through the per-pair search)
    p1, c1, p2, c2 = specs[0][4]
    ref0 = oracle_maps(p1, c1, p2, c2, specs[0][2], 32, specs[0][3].L, SIGMA_G)
    for r in range(len(specs[0][2])):
        assert rel_err(maps[0][r], ref0[r]) < 1e-4

    ctx.set_option("autotune", 1)
    outs = [torch.empty((q.shape[0], sd.CAND_BYTES), dtype=torch.uint8, device="cuda") for _, _, q, _ in jobs]
    st = torch.cuda.Stream()
    for call in range(4):  # eager, captured, replayed, replayed without stats
        with torch.cuda.stream(st):
            for o in outs:
                o.fill_(255)
            _, stats = ctx.score_pairs(jobs, outs=outs, stats=call < 3)
        st.synchronize()
        for j, (fx, mv, qd, g) in enumerate(jobs):
            s, rot, idx = sd.decode_cands(outs[j])
            bs, brot, bidx = refs[j]
            assert torch.equal(rot, brot), (call, j)
            scale = np.abs(maps[j].real).max()
            assert (s - bs).abs().max().item() <= 1e-5 * scale, (call, j)
            for r in range(qd.shape[0]):
                if _margin_ok(maps[j][r].real):
                    assert idx[r].item() == bidx[r].item(), (call, j, r)
            if stats is not None:
                x = stats[j]
                assert np.isfinite(x["ms"]) and x["ms"] > 0
                assert 1 <= x["batch"] <= 64 and x["spread_bins"] in (0, 1, 2, 8, 12, 16)
                assert x["n"] == 2 * g.N and 0 < x["s"] <= x["n"] and x["s"] % 2 == 0
    ctx.close()


def test_score_pairs_rejects_bad_jobs():
    ctx = sd.Context(3, "f32", 0, sigma_g=SIGMA_G)
    w = configs.tiny_3d()
    p1, c1, p2, c2 = oracle_weights("tiny_3d")
    fx = ctx.shape_from_samples(p1, cplx_to_pairs(c1))
    mv = ctx.shape_from_samples(p2, cplx_to_pairs(c2))
    empty = torch.empty((0, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(sd.SdError) as e:
        ctx.score_pairs([(fx, mv, _quats(w.quats), sd.Grid(32, w.L)), (fx, mv, empty, sd.Grid(32, w.L))])
    assert e.value.code == sd.SD_ERR_ARG
    with pytest.raises(sd.SdError) as e:
        ctx.score_pairs([(fx, mv, _quats(w.quats), sd.Grid(40, w.L))])
    assert e.value.code == sd.SD_ERR_ARG
    ctx.close()


def test_tuned_plans_export_and_import():
    import json
    import re

    ctx = sd.Context(3, "f32", 0, sigma_g=SIGMA_G)
    fx, mv, q, g, _ = _jobs(ctx)[2]
    qd = _quats(q)
    ctx.set_option("autotune", 1)
    ctx.score_rotations(fx, mv, qd, g)  # times the candidate plans of this geometry once
    plan = ctx.search_plan(mv, g, qd.shape[0])
    text = ctx.tune_export()
    table = json.loads(text)
    assert table["sdfdock_plans"] == 1 and len(table["plans"]) == 1
    assert table["plans"][0]["batch"] >= 1 and table["plans"][0]["spread_bins"] in (0, 1, 2, 8, 12, 16)
    assert table["plans"][0]["fft"] == plan["fft_plan"] and plan["fft_plan"] in (0, 1, 2, 3)

    ctx2 = sd.Context(3, "f32", 0, sigma_g=SIGMA_G)
    fx2, mv2, _, _, _ = _jobs(ctx2)[2]
    ctx2.set_option("autotune", 1)
    before = ctx2.search_plan(mv2, g, qd.shape[0])
    ctx2.tune_import(text)
    assert ctx2.search_plan(mv2, g, qd.shape[0]) == plan
    assert json.loads(ctx2.tune_export()) == table
    # malformed tables are refused and leave the cache as it was
    for bad in ("{}", re.sub(r'"batch": \d+', '"batch": 0', text), re.sub(r'"spread_bins": \d+', '"spread_bins": 7', text),
                re.sub(r'"fft": \d+', '"fft": 4', text)):
        with pytest.raises(sd.SdError) as e:
            ctx2.tune_import(bad)
        assert e.value.code == sd.SD_ERR_ARG
    assert json.loads(ctx2.tune_export()) == table
    assert isinstance(before["batch"], int)
    # a table without the FFT plan (older exports) takes the pruned plan
    ctx2.tune_import(re.sub(r', "fft": \d+', '', text))
    assert ctx2.search_plan(mv2, g, qd.shape[0])["fft_plan"] in (1, plan["fft_plan"])
    ctx.close()
    ctx2.close()


def test_plan_options_reject_bad_values():
    # the plan options take only their documented values; a refused value leaves
    # the option as it was
    ctx = sd.Context(3, "f32", 0, sigma_g=SIGMA_G)
    fx, mv, q, g, _ = _jobs(ctx)[2]
    before = ctx.search_plan(mv, g, 9)
    for key, value in (("fft_plan", 5), ("fft_plan", -2), ("spread_bin_side", 10), ("spread_bin_side", 0)):
        with pytest.raises(sd.SdError) as e:
            ctx.set_option(key, value)
        assert e.value.code == sd.SD_ERR_ARG
    assert ctx.search_plan(mv, g, 9) == before
    ctx.set_option("spread_direct", 0)
    for side in (8, 12, 16):
        ctx.set_option("spread_bin_side", side)
        assert ctx.search_plan(mv, g, 9)["spread_bins"] == side
    ctx.close()
