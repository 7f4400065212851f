"""Sharding one permanent across processes (one per GPU) by Gray-code term range,
and resuming a long sweep from a checkpoint of completed ranges.

Every rank sums its own contiguous range of the 2^(n-1) Glynn terms (or 2^n Ryser
subsets) with ``perm_glynn_partial`` / ``perm_ryser_partial``; the unnormalised
double-double partials are exchanged once (an all-gather of two doubles per rank,
summed in rank order so the result does not depend on the collective's reduction
order) and normalised by 2^(n-1) (n-m)!.  This is the path's only exchange step.
"""
from __future__ import annotations

import hashlib
import json
import math
import os
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


def _digest(A) -> str:
    import numpy as np
    a = np.ascontiguousarray(A)
    return hashlib.sha256(str((a.dtype.str, a.shape)).encode() + a.tobytes()).hexdigest()


def resumable_glynn(A, partial_fn, state_path, step_terms=1 << 30, stop_after=None):
    """per(A) by consecutive term ranges of ``step_terms``, each computed by
    partial_fn(A, g_begin, g_end) -> (hi, lo) (e.g. perm_glynn_partial); after every range
    the exact running sum and the next term index are written to ``state_path`` (via a
    temporary file and an atomic rename), so an interrupted sweep resumes where it stopped.
    A checkpoint of another matrix is refused.  ``stop_after`` (ranges) ends the call early
    and returns None, as an interruption would."""
    import numpy as np
    A = np.asarray(A)
    if A.shape[0] > A.shape[1]:
        A = A.T
    m, n = A.shape
    if m == 0:
        return 1.0
    total = 1 << (n - 1)
    digest = _digest(A)
    done, acc = 0, Fraction(0)
    if os.path.exists(state_path):
        with open(state_path) as f:
            st = json.load(f)
        if st.get("digest") != digest or st.get("shape") != [m, n]:
            raise ValueError("checkpoint %s belongs to another matrix" % state_path)
        done, acc = int(st["done"]), Fraction(st["sum"])
    ranges = 0
    while done < total:
        if stop_after is not None and ranges >= stop_after:
            return None
        g1 = min(done + step_terms, total)
        hi, lo = partial_fn(A, done, g1)
        acc += Fraction(hi) + Fraction(lo)
        done = g1
        ranges += 1
        tmp = state_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({"digest": digest, "shape": [m, n], "done": done, "sum": str(acc)}, f)
        os.replace(tmp, state_path)
    return normalise_glynn(acc, m, n)
