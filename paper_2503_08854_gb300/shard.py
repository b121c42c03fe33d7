"""Orbit sharding across ranks (one process per GPU).

Orbits are independent (paper sec. 5.2.1 proposes partitioning the orbits
instead of the images), so each rank stacks its own contiguous slice of the
orbit batch against the full exposure set with no exchange.  The one step
that needs the other ranks is a shared candidate list: every rank ranks its
slice, the k (index, nu) pairs of all ranks are all-gathered and merged with
the same order as the single-GPU ranking (nu descending, global orbit index
ascending).  This module holds only that host-side bookkeeping; the ranking
of each slice runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous slice [lo, hi) of n orbits owned by ``rank``."""
    base, rem = divmod(n, world)
    lo = rank * base + min(rank, rem)
    return lo, lo + base + (1 if rank < rem else 0)


def merge_ranked(idx_lists, snr_lists, k: int):
    """Merge per-rank rankings (global indices) into the top-k of their union,
    ordered by nu descending then index ascending."""
    idx = np.concatenate([np.asarray(i, np.int64) for i in idx_lists])
    snr = np.concatenate([np.asarray(s, np.float64) for s in snr_lists])
    snr = np.where(np.isnan(snr), -np.inf, snr)
    order = np.lexsort((idx, -snr))[:k]
    return idx[order], snr[order]


def allgather_topk(local_idx, local_snr, offset: int, k: int, group=None):
    """All-gather every rank's top-k (local indices + its slice offset) and
    merge; every rank returns the same global top-k.  Uses torch.distributed
    (gloo on the host, or NCCL) on k * 12 bytes per rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = len(local_idx)
    payload = torch.full((k, 2), float("nan"), dtype=torch.float64)
    payload[:n, 0] = torch.as_tensor(np.asarray(local_idx, np.int64) + offset, dtype=torch.float64)
    payload[:n, 1] = torch.as_tensor(np.asarray(local_snr, np.float64))
    bufs = [torch.empty_like(payload) for _ in range(world)]
    dist.all_gather(bufs, payload, group=group)
    idx_l, snr_l = [], []
    for b in bufs:
        ok = ~torch.isnan(b[:, 0])
        idx_l.append(b[ok, 0].numpy().astype(np.int64))
        snr_l.append(b[ok, 1].numpy())
    return merge_ranked(idx_l, snr_l, k)
