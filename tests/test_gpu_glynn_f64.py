"""Parity of the real FP64 Glynn sweep (perm_glynn / perm_glynn_partial, dtype
PERM_F64, opts.arith = PERM_ARITH_FP64) with the long-double CPU oracle, through the
C ABI.

Tolerance (gpu_util.close): max(1e-12 |ref|, 8 (n+2) u sum|t|), sum|t| the oracle's
sum of |term| over the terms this sweep evaluates (the padded terms of Eq.
glynn_rectangle for a rectangle), normalised like the result.  The FP64 sweep
evaluates the padded sum, which cancels heavily for rectangles with entries of both
signs (m << n); its rectangle tests take uniform[0,1] entries, as the paper's
rectangular workload does, or small shapes, and check that the tolerance stays
below 1e-9 |per|."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import U, close, tol_ratio
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


def to_dev(A, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(A)).to(dev)


FP64 = dict(arith=1)


def glynn(capi, A, dev, opts=None):
    import torch
    out = capi.perm_glynn(to_dev(A, dev), opts=dict(FP64, **(opts or {})))
    torch.cuda.synchronize(dev)
    return capi.value(out, capi.PERM_F64)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 8, 9, 12, 13, 16, 17, 20, 21])
def test_square_random(capi, dev, n):
    A = inputs.uniform_real(n, n, 1000 + n)
    ref = oracle.glynn(A)
    close(glynn(capi, A, dev), ref, A)
    assert tol_ratio(ref, A) <= 1e-9


@pytest.mark.parametrize("m,n,lo", [(1, 4, -1.0), (2, 3, -1.0), (3, 7, -1.0), (5, 9, -1.0), (8, 13, 0.0),
                                    (10, 18, 0.0), (4, 20, 0.0), (12, 21, 0.0), (13, 21, 0.0)])
def test_rectangular_random(capi, dev, m, n, lo):
    A = inputs.uniform_real(m, n, 2000 + 31 * m + n, lo, 1.0)
    ref = oracle.glynn(A)
    close(glynn(capi, A, dev), ref, A)
    assert tol_ratio(ref, A) <= 1e-9


def test_transposed_input(capi, dev):
    A = inputs.uniform_real(11, 6, 3001)
    ref = oracle.glynn(A.T)
    close(glynn(capi, A, dev), ref, A)
    assert tol_ratio(ref, A) <= 1e-9


def test_empty_matrix_is_one(capi, dev):
    assert glynn(capi, np.zeros((0, 5)), dev) == 1.0
    assert glynn(capi, np.zeros((0, 0)), dev) == 1.0


@pytest.mark.parametrize("n", [3, 10, 18])
def test_ones_and_identity_closed_forms(capi, dev, n):
    close(glynn(capi, np.ones((n, n)), dev), float(math.factorial(n)), np.ones((n, n)), rel=1e-14)
    close(glynn(capi, np.eye(n), dev), 1.0, np.eye(n), rel=1e-15)
    m = n // 2 + 1
    ones = np.ones((m, n))
    close(glynn(capi, ones, dev), math.factorial(n) / math.factorial(n - m), ones, rel=1e-13)
    eye = np.zeros((m, n))
    eye[np.arange(m), np.arange(m)] = 1.0
    close(glynn(capi, eye, dev), 1.0, eye)


def test_host_buffers_match_device(capi, dev):
    A = inputs.uniform_real(14, 14, 3101)
    host_out = np.zeros(1)
    capi.perm_glynn(A, out=host_out, opts=FP64)
    assert host_out[0] == glynn(capi, A, dev)


def test_deterministic(capi, dev):
    A = inputs.uniform_real(19, 19, 3201)
    assert glynn(capi, A, dev) == glynn(capi, A, dev)


@pytest.mark.parametrize("opts", [dict(chunk_log2=2), dict(chunk_log2=5, grid=3, block=64), dict(grid=1, block=32),
                                  dict(chunk_log2=30), dict(grid=7, block=96, chunk_log2=1)])
def test_launch_shapes_and_anchor_periods(capi, dev, opts):
    A = inputs.uniform_real(15, 15, 3301)
    ref = oracle.glynn(A)
    close(glynn(capi, A, dev, opts), ref, A)
    assert tol_ratio(ref, A) <= 1e-9


def test_partial_ranges_match_oracle(capi, dev):
    import torch
    A = inputs.uniform_real(9, 13, 3401)
    dA = to_dev(A, dev)
    T = 1 << 12
    g = inputs.rng(3402)
    cuts = sorted(set([0, T, 1, T - 1] + [int(c) for c in g.integers(0, T, 6)]))
    for a, b in zip(cuts, cuts[1:]):
        out = capi.perm_glynn_partial(dA, a, b, opts=dict(FP64, chunk_log2=3))
        torch.cuda.synchronize(dev)
        got = capi.dd_value(out)
        ref = oracle.glynn_partial(A, a, b)
        scale = oracle.glynn_partial_abs(A, a, b)
        assert abs(got - ref) <= max(1e-13 * abs(ref), (13 + 4 + 2 * 13 * 8) * U * scale), (a, b, got, ref)


def test_error_bound_holds(capi, dev):
    import torch
    A = inputs.uniform_real(17, 17, 3501)
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    out = capi.perm_glynn(to_dev(A, dev), opts=dict(FP64, err=err))
    torch.cuda.synchronize(dev)
    got, ref = capi.value(out, capi.PERM_F64), oracle.glynn(A)
    assert abs(got - ref) <= float(err.item())
    assert float(err.item()) < 1e-6 * abs(ref)


def test_config_square16_f64(capi, dev):
    A = inputs.square16_f64()
    ref_g, ref_r = oracle.glynn(A), oracle.ryser(A)
    assert abs(ref_g - ref_r) <= 1e-14 * abs(ref_g)
    got = glynn(capi, A, dev)
    assert abs(got - ref_g) <= 1e-12 * abs(ref_g)


@pytest.mark.parametrize("where", ["start", "middle", "end"])
def test_config_square36_sampled_ranges(capi, dev, where):
    # the full 2^35-term sum is beyond the oracle; compare sampled term ranges
    import torch
    A = inputs.square36_f64()
    T = 1 << 35
    span = 1 << 12
    a = {"start": 0, "middle": T // 2 - span // 2 + 12345, "end": T - span}[where]
    out = capi.perm_glynn_partial(to_dev(A, dev), a, a + span, opts=dict(FP64, chunk_log2=10))
    torch.cuda.synchronize(dev)
    got = capi.dd_value(out)
    ref = oracle.glynn_partial(A, a, a + span)
    scale = oracle.glynn_partial_abs(A, a, a + span)
    # first-order rounding of the sweep: n products, the sum, and the drift of the
    # column sums over at most 2^10 incremental updates between exact rebuilds
    assert abs(got - ref) <= max(1e-12 * abs(ref), (36 + 4 + 2 * 36 * 2 ** 10) * U * scale)
    assert abs(got - ref) <= 1e-11 * scale


def test_default_arithmetic_is_the_integer_pipe_sweep(capi, dev):
    # with no options a real matrix of order >= 10 takes the integer-pipe sweep; it
    # agrees with the FP64 sweep and the oracle
    import torch
    A = inputs.uniform_real(20, 20, 3601)
    out = capi.perm_glynn(to_dev(A, dev))
    torch.cuda.synchronize(dev)
    ref = oracle.glynn(A)
    close(capi.value(out, capi.PERM_F64), ref, A)
    close(glynn(capi, A, dev), ref, A)
    assert tol_ratio(ref, A) <= 1e-9
