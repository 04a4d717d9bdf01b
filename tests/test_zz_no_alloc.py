"""The allocation-free top-k entry point against the oracle's top-k.

sd_top_k_static exists for callers that cannot allocate device memory while
they run (real-time loops that must not stall on the device synchronisation of
cudaMalloc/cudaFree, engines bound to a fixed shared memory pool, device memory
owned by a foreign allocator); its scratch is a fixed device array inside the
library, shared by every call.  Each call's selection is checked against
oracle.score.global_top_k on the decoded candidates, and against the
workspace-based sd_top_k_poses.  This file is collected last so that a run
stopping at the first failure has run every other test.
"""

import ctypes as ct

import numpy as np
import pytest
import torch

from oracle import score as oscore
from paper_1712_00238_gb300 import sdfdock as sd

pytestmark = pytest.mark.gpu

REC = [("score", "<f8"), ("rot", "<i4"), ("idx", "<i4")]


def _cands(n, seed, nan=0):
    """Per-rotation candidates in a shuffled order; scores drawn from few values
    so that ties exercise the index order, `nan` of them NaN."""
    rng = np.random.default_rng(seed)
    rec = np.zeros(n, dtype=REC)
    rec["score"] = rng.integers(0, 7, n).astype(float) * 0.25 - 0.5
    if nan:
        rec["score"][rng.choice(n, nan, replace=False)] = np.nan
    rec["rot"] = rng.permutation(n)
    rec["idx"] = rng.integers(0, 1 << 20, n)
    return rec


def _oracle_top_k(rec, k):
    # global_top_k ranks per-rotation maxima given in rotation order
    by_rot = np.empty_like(rec)
    by_rot[rec["rot"]] = rec
    return oscore.global_top_k(by_rot["score"], by_rot["idx"], k)


def _run_static(lib, ctx, rec, k, stream):
    cand = torch.from_numpy(rec.view(np.uint8).copy()).cuda()
    out = torch.full((k, sd.CAND_BYTES), 0x5A, dtype=torch.uint8, device="cuda")
    rc = lib.sd_top_k_static(ctx.handle, cand.data_ptr(), len(rec), k, out.data_ptr(), stream)
    assert rc == 0, lib.sd_last_error(ctx.handle)
    return cand, out.cpu().numpy().reshape(-1).view(REC)


def _check_against_oracle(got, rec, k):
    want = _oracle_top_k(rec, k)
    n_real = min(k, len(rec))
    assert [(int(r["rot"]), int(r["idx"])) for r in got[:n_real]] == [(r, i) for r, _, i in want]
    s_got, s_want = got["score"][:n_real], np.array([s for _, s, _ in want])
    assert np.array_equal(np.isnan(s_got), np.isnan(s_want))
    assert np.array_equal(s_got[~np.isnan(s_got)], s_want[~np.isnan(s_want)])
    # entries past the candidate count: rot = idx = -1, score -inf
    pad = got[n_real:]
    assert np.all(pad["rot"] == -1) and np.all(pad["idx"] == -1) and np.all(pad["score"] == -np.inf)


def test_static_top_k_matches_oracle_on_consecutive_calls():
    ctx = sd.Context(3, "f32", 0)
    lib = ctx.lib
    grid = sd.sd_grid(32, 10.0)
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row with different sizes (the shared bitset keeps the
    # first call's bits; the second must not see them), NaN scores ranked last
    for call, (n, k, seed, nan) in enumerate(((50_000, 64, 1, 0), (7_321, 300, 2, 5))):
        rec = _cands(n, seed, nan)
        cand, got = _run_static(lib, ctx, rec, k, stream)
        _check_against_oracle(got, rec, k)
        # the workspace-based entry point selects the same poses
        poses = (sd.sd_pose * k)()
        rc = lib.sd_top_k_poses(ctx.handle, cand.data_ptr(), n, k, 0, None, None, None, ct.byref(grid), poses,
                                stream)
        assert rc == 0, lib.sd_last_error(ctx.handle)
        assert [(int(r["rot"]), int(r["idx"])) for r in got] == [(p.rot, p.idx) for p in poses], call
    # sizes beyond the fixed scratch are refused without touching the device
    rc = lib.sd_top_k_static(ctx.handle, cand.data_ptr(), sd.SD_TOP_K_STATIC_MAX + 1, 4, cand.data_ptr(), stream)
    assert rc == sd.SD_ERR_ARG and b"2^20" in lib.sd_last_error(ctx.handle)
    rc = lib.sd_top_k_static(ctx.handle, cand.data_ptr(), 10, 4097, cand.data_ptr(), stream)
    assert rc == sd.SD_ERR_ARG
    ctx.close()


def test_static_top_k_at_the_size_limit_and_past_the_candidates():
    ctx = sd.Context(3, "f32", 0)
    lib = ctx.lib
    stream = torch.cuda.current_stream().cuda_stream
    # n = 2^20: the last word of the bitset is used; plant the best candidate last
    n = sd.SD_TOP_K_STATIC_MAX
    rec = _cands(n, 3)
    rec["score"][-1] = 10.0
    rec["score"][-2] = 10.0
    _, got = _run_static(lib, ctx, rec, 5, stream)
    _check_against_oracle(got, rec, 5)
    assert set(int(r) for r in got["rot"][:2]) == {int(rec["rot"][-1]), int(rec["rot"][-2])}
    # k > n: the real candidates, then padding (a call after the full-size one)
    rec = _cands(37, 4, nan=2)
    _, got = _run_static(lib, ctx, rec, 50, stream)
    _check_against_oracle(got, rec, 50)
    ctx.close()
