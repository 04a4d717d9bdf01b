"""Rotation sharding across ranks and the top-k merge, as two gloo processes on CPU.

Rotations are independent, so ranks score contiguous rotation shards with no
data-path collective and only gather their per-rank top-k lists.  The per-rank
candidates here come from the oracle on a small 2D workload; the merged result
must equal the single-process global top-k.
"""

import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import score as oscore
from paper_1712_00238_gb300.sdfdock import merge_top_k, shard_range
from synth import configs

K = 5


def _candidates(lo, hi):
    w = configs.tiny_2d()
    rng = np.random.default_rng(3)
    p1 = w.fixed.query.pos
    p2 = w.moving.query.pos
    c1 = rng.standard_normal(len(p1)) + 1j * rng.standard_normal(len(p1))
    c2 = rng.standard_normal(len(p2)) + 1j * rng.standard_normal(len(p2))
    best, idx = oscore.score_rotations(p1, c1, p2, c2, w.quats[lo:hi], 16, w.L, 0.3)
    # per-rank top-k with global rotation numbers
    local = oscore.global_top_k(best, idx, K)
    return [(s, r + lo, i) for r, s, i in local]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = configs.tiny_2d().n_rot
    lo, hi = shard_range(n, world, rank)
    mine = _candidates(lo, hi)
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    merged = merge_top_k(parts, K)
    out[rank] = merged
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2])
def test_sharded_top_k_equals_single_process(world):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        results = [out[r] for r in range(world)]
    n = configs.tiny_2d().n_rot
    ref = _candidates(0, n)
    for res in results:
        assert [(r, i) for _, r, i in res] == [(r, i) for _, r, i in ref]
        assert np.allclose([s for s, _, _ in res], [s for s, _, _ in ref], rtol=0, atol=1e-12)


def test_merge_order_and_nan():
    parts = [[(1.0, 3, 7), (0.5, 1, 2)], [(1.0, 2, 9), (float("nan"), 0, 0), (2.0, 5, 1)]]
    assert merge_top_k(parts, 4) == [(2.0, 5, 1), (1.0, 2, 9), (1.0, 3, 7), (0.5, 1, 2)]


def test_merge_drops_rank_padding():
    # a rank with fewer than k candidates pads its list with rot = idx = -1, score -inf;
    # the padding must not displace real candidates scoring -inf or NaN
    inf = float("inf")
    parts = [[(0.5, 4, 1), (-inf, -1, -1), (-inf, -1, -1)], [(-inf, 2, 8), (float("nan"), 0, 3), (1.5, 7, 0)]]
    merged = merge_top_k(parts, 4)
    assert [(r, i) for _, r, i in merged] == [(7, 0), (4, 1), (0, 3), (2, 8)]
    assert len(merge_top_k(parts, 10)) == 4
