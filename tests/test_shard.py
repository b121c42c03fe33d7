"""Orbit sharding over ranks: slices cover the batch, and the all-gathered merge
of per-rank rankings equals the oracle's ranking of the whole batch
(world_size 2, gloo on the host)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as O
from paper_2503_08854_gb300 import shard


def test_shard_ranges_cover_batch():
    for n in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            parts = [shard.shard_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))


def test_merge_matches_oracle_ranking():
    rng = np.random.default_rng(0)
    nu = np.round(rng.normal(size=5000), 2)
    nu[rng.integers(0, 5000, 300)] = -np.inf
    k = 200
    parts = [shard.shard_range(len(nu), r, 3) for r in range(3)]
    il, sl = [], []
    for lo, hi in parts:
        i, s = O.topk(nu[lo:hi], k)
        il.append(i + lo)
        sl.append(s)
    idx, snr = shard.merge_ranked(il, sl, k)
    ref_i, ref_s = O.topk(nu, k)
    np.testing.assert_array_equal(idx, ref_i)
    np.testing.assert_array_equal(snr, ref_s)


def _worker(rank, world, port, nu, k, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard.shard_range(len(nu), rank, world)
    i, s = O.topk(nu[lo:hi], k)
    idx, snr = shard.allgather_topk(i, s, lo, k)
    out[rank] = (idx.tolist(), snr.tolist())
    dist.destroy_process_group()


def test_allgather_topk_world_size_two():
    rng = np.random.default_rng(1)
    nu = np.round(rng.normal(size=3001), 1)
    k = 64
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, nu, k, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    ref_i, ref_s = O.topk(nu, k)
    for r in range(2):
        np.testing.assert_array_equal(np.array(out[r][0]), ref_i)
        np.testing.assert_array_equal(np.array(out[r][1]), ref_s)
