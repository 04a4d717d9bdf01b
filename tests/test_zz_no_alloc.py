"""The allocation-free top-k entry point agrees with the workspace-based one.

sd_top_k_static exists for callers that cannot allocate device memory while
they run (real-time loops, fixed shared memory pools, foreign allocators); its
scratch is a fixed device array inside the library.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""

import ctypes as ct

import numpy as np
import pytest
import torch

from paper_1712_00238_gb300 import sdfdock as sd

pytestmark = pytest.mark.gpu


def _cands(n, seed):
    # scores drawn from few values so that ties exercise the rotation / index order
    rng = np.random.default_rng(seed)
    rec = np.zeros(n, dtype=[("score", "<f8"), ("rot", "<i4"), ("idx", "<i4")])
    rec["score"] = rng.integers(0, 7, n).astype(float) * 0.25 - 0.5
    rec["rot"] = rng.permutation(n)
    rec["idx"] = rng.integers(0, 1 << 20, n)
    return torch.from_numpy(rec.view(np.uint8).copy()).cuda()


def _decode(buf):
    return buf.cpu().numpy().reshape(-1).view([("score", "<f8"), ("rot", "<i4"), ("idx", "<i4")])


def test_static_top_k_matches_workspace_top_k_twice():
    ctx = sd.Context(3, "f32", 0)
    lib = ctx.lib
    grid = sd.sd_grid(32, 10.0)
    stream = torch.cuda.current_stream().cuda_stream
    for call, (n, k, seed) in enumerate(((50_000, 64, 1), (7_321, 300, 2))):
        cand = _cands(n, seed)
        out = torch.full((k, sd.CAND_BYTES), 0xFF, dtype=torch.uint8, device="cuda")
        rc = lib.sd_top_k_static(ctx.handle, cand.data_ptr(), n, k, out.data_ptr(), stream)
        assert rc == 0, lib.sd_last_error(ctx.handle)
        poses = (sd.sd_pose * k)()
        rc = lib.sd_top_k_poses(ctx.handle, cand.data_ptr(), n, k, 0, None, None, None, ct.byref(grid), poses,
                                stream)
        assert rc == 0, lib.sd_last_error(ctx.handle)
        got = _decode(out)
        assert [(int(r["rot"]), int(r["idx"])) for r in got] == [(p.rot, p.idx) for p in poses], call
        assert np.array_equal(got["score"], np.array([p.score for p in poses])), call
    # sizes beyond the fixed scratch are refused without touching the device
    rc = lib.sd_top_k_static(ctx.handle, cand.data_ptr(), sd.SD_TOP_K_STATIC_MAX + 1, 4, out.data_ptr(), stream)
    assert rc == sd.SD_ERR_ARG and b"2^20" in lib.sd_last_error(ctx.handle)
    ctx.close()
