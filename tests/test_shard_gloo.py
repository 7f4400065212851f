"""Sharding one permanent over two processes (gloo, CPU): each rank sums its own
Glynn term range, the double-double partials are exchanged once, and the result
equals the single-process value.  The per-rank partial sums come from the oracle
here (no GPU); on GPUs they come from perm_glynn_partial."""
import math
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2510_03421_gb300 import inputs, shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, A, q):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        val = shard.sharded_glynn(A, lambda M, a, b: oracle.glynn_partial(M, a, b, dd=True))
        q.put((rank, val))
    finally:
        dist.destroy_process_group()


def test_term_ranges_cover_once():
    for total in (1, 7, 1 << 20, 12345):
        for world in (1, 2, 3, 8):
            rs = [shard.term_range(total, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == total
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1


@pytest.mark.parametrize("shape", [(9, 9), (6, 11)])
def test_two_rank_gloo_matches_single(shape):
    import oracle
    A = inputs.uniform_real(*shape, 4242 + shape[1])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, A, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = oracle.glynn(A)
    assert got[0] == got[1]
    assert abs(got[0] - ref) <= 1e-14 * abs(ref)


def test_single_process_path():
    import oracle
    A = inputs.uniform_real(7, 7, 4250)
    val = shard.sharded_glynn(A, lambda M, a, b: oracle.glynn_partial(M, a, b, dd=True))
    assert abs(val - oracle.glynn(A)) <= 1e-14 * abs(oracle.glynn(A))
    assert math.isclose(shard.normalise_glynn(shard.combine([(8.0, 0.0)]), 2, 3), 2.0)


def test_resume_from_checkpoint(tmp_path):
    # an interrupted range-by-range sweep resumes from its checkpoint and gives the same
    # exact sum; a checkpoint of another matrix is refused
    import oracle
    A = inputs.uniform_real(9, 12, 4300)
    part = lambda M, a, b: oracle.glynn_partial(M, a, b, dd=True)  # noqa: E731
    path = str(tmp_path / "sweep.json")
    assert shard.resumable_glynn(A, part, path, step_terms=100, stop_after=7) is None
    assert shard.resumable_glynn(A, part, path, step_terms=100, stop_after=5) is None
    got = shard.resumable_glynn(A, part, path, step_terms=100)
    ref = oracle.glynn(A)
    assert abs(got - ref) <= 1e-13 * abs(ref)
    fresh = shard.resumable_glynn(A, part, str(tmp_path / "fresh.json"), step_terms=333)
    assert abs(fresh - got) <= 1e-15 * abs(got)  # other cuts: the same terms
    with pytest.raises(ValueError):
        shard.resumable_glynn(inputs.uniform_real(9, 12, 4301), part, path)
