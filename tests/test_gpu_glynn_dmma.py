"""Parity of the FP64 Glynn sweep whose chunk-start column sums come from the
+-1 x A' contraction on the FP64 tensor cores (opts.start = PERM_START_DMMA)."""
import numpy as np
import pytest

import oracle
from gpu_util import U, close, device, run, to_dev
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu

DMMA = dict(start=2)


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 9, 13, 16, 19, 22])
def test_dmma_square(capi, dev, n):
    A = inputs.uniform_real(n, n, 7600 + n)
    close(run(capi, "perm_glynn", A, dev, DMMA), oracle.glynn(A), A)


@pytest.mark.parametrize("m,n", [(2, 7), (6, 11), (10, 17), (3, 20)])
def test_dmma_rectangular(capi, dev, m, n):
    A = inputs.uniform_real(m, n, 7700 + 31 * m + n, 0.0, 1.0)
    close(run(capi, "perm_glynn", A, dev, DMMA), oracle.glynn(A), A)
    close(run(capi, "perm_glynn", np.ascontiguousarray(A.T), dev, DMMA), oracle.glynn(A), A)


@pytest.mark.parametrize("opts", [dict(start=2, chunk_log2=2), dict(start=2, chunk_log2=5, grid=3, block=64),
                                  dict(start=2, grid=1, block=32, chunk_log2=3)])
def test_dmma_chunk_lengths_and_grids(capi, dev, opts):
    A = inputs.uniform_real(14, 14, 7801)
    close(run(capi, "perm_glynn", A, dev, opts), oracle.glynn(A), A)


def test_dmma_ragged_partial_ranges(capi, dev):
    import torch
    A = inputs.uniform_real(10, 12, 7901)
    dA = to_dev(A, dev)
    for a, b in [(0, 2048), (3, 1000), (1500, 1501), (777, 2047)]:
        out = capi.perm_glynn_partial(dA, a, b, opts=dict(start=2, chunk_log2=4))
        torch.cuda.synchronize(dev)
        ref = oracle.glynn_partial(A, a, b)
        scale = oracle.glynn_partial_abs(A, a, b)
        assert abs(capi.dd_value(out) - ref) <= max(1e-13 * abs(ref), 64 * 12 * U * scale), (a, b)


def test_dmma_sampled_n36(capi, dev):
    import torch
    A = inputs.square36_f64()
    a = (1 << 34) + 4099
    out = capi.perm_glynn_partial(to_dev(A, dev), a, a + 4096, opts=dict(start=2, chunk_log2=8))
    torch.cuda.synchronize(dev)
    ref = oracle.glynn_partial(A, a, a + 4096)
    scale = oracle.glynn_partial_abs(A, a, a + 4096)
    assert abs(capi.dd_value(out) - ref) <= (36 + 4 + 2 * 36 * 2 ** 8) * U * scale
