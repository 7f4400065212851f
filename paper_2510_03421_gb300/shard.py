"""Sharding one permanent across processes (one per GPU) by Gray-code term range.

Every rank sums its own contiguous range of the 2^(n-1) Glynn terms (or 2^n Ryser
subsets) with ``perm_glynn_partial`` / ``perm_ryser_partial``; the unnormalised
double-double partials are exchanged once (an all-gather of two doubles per rank,
summed in rank order so the result does not depend on the collective's reduction
order) and normalised by 2^(n-1) (n-m)!.  This is the path's only exchange step.
"""
from __future__ import annotations

import math
from fractions import Fraction


def term_range(total: int, world: int, rank: int):
    """[begin, end) of rank's share of `total` terms (contiguous, sizes differ by <= 1)."""
    base, rem = divmod(total, world)
    begin = rank * base + min(rank, rem)
    return begin, begin + base + (1 if rank < rem else 0)


def combine(partials):
    """Exact sum of double-double partials [(hi, lo), ...] in the given order, rounded once."""
    s = Fraction(0)
    for hi, lo in partials:
        s += Fraction(hi) + Fraction(lo)
    return s


def normalise_glynn(total: Fraction, m: int, n: int) -> float:
    """per(A) from the unnormalised Glynn sum: divide by 2^(n-1) (n-m)! (Eq. glynn_rectangle)."""
    return float(total / (Fraction(2) ** (n - 1) * math.factorial(n - m)))


def sharded_glynn(A, partial_fn, group=None):
    """per(A) with this rank's share computed by partial_fn(A, g_begin, g_end) -> (hi, lo).

    Uses torch.distributed (any backend) for the exchange; works with one process too."""
    import torch
    import torch.distributed as dist
    m, n = A.shape
    if m > n:
        A = A.T
        m, n = n, m
    if m == 0:
        return 1.0
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    g0, g1 = term_range(1 << (n - 1), world, rank)
    hi, lo = partial_fn(A, g0, g1)
    mine = torch.tensor([hi, lo], dtype=torch.float64)
    if world > 1:
        gathered = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, mine, group=group)
    else:
        gathered = [mine]
    return normalise_glynn(combine([(float(t[0]), float(t[1])) for t in gathered]), m, n)
