"""Sharding events over ranks and merging the per-rank cross sections.

Events are independent (the paper's event-level parallelism, Sec. 3.1), so a
batch splits into contiguous event ranges, one per rank, with no exchange on
the data path.  The only exchange is the sum of the per-rank cross sections
sigma'_p (Eq. 2): each rank contributes its (P+1) (sum, compensation) pairs,
and the merge adds them in rank order with TwoSum compensation, so every rank
gets the same, deterministic total.
"""
from __future__ import annotations

import numpy as np


def shard_range(n_events: int, rank: int, world: int):
    """[start, stop) of rank's contiguous share (sizes differ by at most 1)."""
    if not (0 <= rank < world) or n_events < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_events, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def _two_sum(a, b):
    s = a + b
    bp = s - a
    return s, (a - (s - bp)) + (b - bp)


def merge_pairs(sums, comps) -> np.ndarray:
    """Compensated sum over ranks (rows, in rank order) of per-rank
    (sum, compensation) pairs: the sums are added with TwoSum and every
    rank's compensation term joins the running compensation."""
    sums = np.asarray(sums, dtype=np.float64)
    comps = np.asarray(comps, dtype=np.float64)
    s = np.zeros(sums.shape[1])
    c = np.zeros(sums.shape[1])
    for row_s, row_c in zip(sums, comps):
        s, e = _two_sum(s, row_s)
        c += row_c + e
    return s + c


def merge_sums(per_rank) -> np.ndarray:
    """Compensated sum over ranks (rows, in rank order) of per-rank value vectors."""
    per_rank = np.asarray(per_rank, dtype=np.float64)
    s = np.zeros(per_rank.shape[1])
    c = np.zeros(per_rank.shape[1])
    for row in per_rank:
        s, e = _two_sum(s, row)
        c += e
    return s + c


def allreduce_sums(values, device=None) -> np.ndarray:
    """All ranks of the default torch.distributed group exchange their value
    vectors (all_gather) and return the same compensated, rank-ordered sum."""
    import torch
    import torch.distributed as dist
    v = torch.as_tensor(np.asarray(values, dtype=np.float64), device=device)
    world = dist.get_world_size()
    parts = [torch.empty_like(v) for _ in range(world)]
    dist.all_gather(parts, v)
    return merge_sums([p.cpu().numpy() for p in parts])


def allreduce_pairs(sums, comps, device=None) -> np.ndarray:
    """All ranks exchange their (sum, compensation) pairs (one all_gather of
    both rows) and return the same rank-ordered compensated total."""
    import torch
    import torch.distributed as dist
    v = torch.as_tensor(np.stack([np.asarray(sums, np.float64), np.asarray(comps, np.float64)]), device=device)
    world = dist.get_world_size()
    parts = [torch.empty_like(v) for _ in range(world)]
    dist.all_gather(parts, v)
    got = [p.cpu().numpy() for p in parts]
    return merge_pairs([g[0] for g in got], [g[1] for g in got])
