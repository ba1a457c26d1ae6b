"""Several GPUs as replicas of the moment loop over disjoint random vectors.

The stochastic trace (Eq. E-2-7) averages over R random vectors, and vectors
are independent: rank q of a world of size P runs its own R vectors
r = q*R .. q*R + R - 1 (the r0 argument of kpm_moments) on its own GPU, and
the estimates are combined by averaging the moments, one all-reduce of
3 x sectors x K doubles per pass.  Nothing else is exchanged.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def vector_offset(rank: int, R: int) -> int:
    """First random-vector index of a rank running R vectors."""
    return rank * R


def combine_moments(moments: dict, world_size: int, group=None) -> dict:
    """Average mu, mu_M, mu_M2 (torch tensors, equal R on every rank) over all ranks in place."""
    if world_size <= 1:
        return moments
    for key in ("mu", "mu_M", "mu_M2"):
        t = moments.get(key)
        if t is None:
            continue
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        t /= world_size
    return moments
