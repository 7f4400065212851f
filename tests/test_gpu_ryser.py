"""Parity of the Ryser sweeps (perm_ryser) with the CPU oracle.

Float tolerance: 8 (n + 2) u times Ryser's own sum of |weight x term| (gpu_util.close
with kind="ryser"); integers bit-exact."""
import numpy as np
import pytest

import oracle
from gpu_util import U, U_FIX, close, device, read_golden, run, to_dev
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


@pytest.mark.parametrize("n", [1, 2, 3, 6, 9, 12, 15, 18])
def test_square_real(capi, dev, n):
    A = inputs.uniform_real(n, n, 6000 + n)
    close(run(capi, "perm_ryser", A, dev), oracle.ryser(A), A, kind="ryser")


@pytest.mark.parametrize("m,n", [(1, 5), (2, 7), (4, 9), (6, 13), (10, 16), (3, 18)])
def test_rectangular_real(capi, dev, m, n):
    A = inputs.uniform_real(m, n, 6100 + 31 * m + n, 0.0, 1.0)
    close(run(capi, "perm_ryser", A, dev), oracle.ryser_rect(A), A, kind="ryser")
    close(run(capi, "perm_ryser", np.ascontiguousarray(A.T), dev), oracle.ryser_rect(A), A, kind="ryser")


@pytest.mark.parametrize("opts", [dict(chunk_log2=1), dict(grid=5, block=64, chunk_log2=3)])
def test_launch_shapes(capi, dev, opts):
    A = inputs.uniform_real(11, 14, 6201)
    close(run(capi, "perm_ryser", A, dev, opts), oracle.ryser_rect(A), A, kind="ryser")


def test_config_square16_golden(capi, dev):
    g = read_golden("square16_f64.txt")
    A = inputs.square16_f64(int(g["seed"][0]))
    ref = float(g["ryser"][0]) + float(g["ryser"][1])
    assert abs(run(capi, "perm_ryser", A, dev) - ref) <= 1e-12 * abs(ref)
    assert abs(run(capi, "perm_glynn", A, dev) - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("m,n", [(4, 4), (7, 7), (3, 9), (8, 13), (12, 12)])
def test_complex(capi, dev, m, n):
    A = inputs.complex_gaussian(m, n, 6300 + 31 * m + n)
    close(run(capi, "perm_ryser", A, dev), oracle.glynn(A), A, kind="ryser")


@pytest.mark.parametrize("m,n", [(5, 5), (9, 9), (4, 11), (10, 14), (16, 16)])
def test_integer_exact(capi, dev, m, n):
    B = inputs.bernoulli01(m, n, 6400 + 31 * m + n)
    assert run(capi, "perm_ryser", B, dev) == oracle.subset_dp(B.astype(np.int64))
    Z = inputs.rng(6500 + m).integers(-30, 31, (m, n)).astype(np.int64)
    assert run(capi, "perm_ryser", Z, dev) == oracle.subset_dp(Z)


def test_config_square26_binary_ryser(capi, dev):
    g = read_golden("square26_01.txt")
    A = inputs.square26_01(int(g["seed"][0]))
    assert run(capi, "perm_ryser", A, dev) == int(g["per"][0])


@pytest.mark.parametrize("m,n", [(1, 12), (2, 20), (3, 16), (4, 22), (6, 24), (2, 40)])
def test_rectangular_by_size(capi, dev, m, n):
    # m << n: perm_ryser visits only the subsets of size <= m (colex order per size)
    A = inputs.uniform_real(m, n, 6600 + 31 * m + n)
    ref = oracle.ryser_rect(A)  # the appendix algorithm: combinations of each size
    close(run(capi, "perm_ryser", A, dev), ref, A, kind="ryser")
    close(run(capi, "perm_ryser", A, dev, dict(chunk_log2=3)), ref, A, kind="ryser")
    close(run(capi, "perm_ryser", np.ascontiguousarray(A.T), dev), ref, A, kind="ryser")


# ---------------------------------------------------------------- integer pipes
@pytest.mark.parametrize("m,n", [(1, 1), (4, 4), (9, 9), (13, 13), (17, 17), (5, 12), (10, 16), (12, 20), (3, 5)])
def test_integer_pipes_against_oracle(capi, dev, m, n):
    # exact fixed-point row sums, 64-bit-mantissa products (opts.arith = FIXED; the
    # default from n = 10 unless the by-size enumeration is much shorter)
    A = inputs.uniform_real(m, n, 6700 + 31 * m + n)
    ref = oracle.ryser(A)
    close(run(capi, "perm_ryser", A, dev, dict(arith=2)), ref, A, kind="ryser", c=2, u=U_FIX)
    close(run(capi, "perm_ryser", np.ascontiguousarray(A.T), dev, dict(arith=2)), ref, A, kind="ryser", c=2,
          u=U_FIX)


def test_integer_pipes_error_bound_and_grids(capi, dev):
    import torch
    A = inputs.uniform_real(15, 15, 6801)
    ref = oracle.ryser(A)
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    out = capi.perm_ryser(to_dev(A, dev), opts=dict(arith=2, err=err))
    torch.cuda.synchronize(dev)
    got = capi.value(out, capi.PERM_F64)
    assert 0.0 < float(err.item()) < 1e-9 * abs(ref)
    assert abs(got - ref) <= float(err.item()) + 2 * U * abs(ref)
    for opts in (dict(arith=2, grid=1, block=32, chunk_log2=3), dict(arith=2, grid=11, block=96)):
        close(run(capi, "perm_ryser", A, dev, opts), ref, A, kind="ryser", c=2, u=U_FIX)


@pytest.mark.parametrize("opts", [dict(grid=1, block=32, chunk_log2=3), dict(grid=11, block=96, chunk_log2=10),
                                  dict(grid=3, block=64, chunk_log2=16), dict()])
def test_integer_pipes_rectangle_chunk_orders(capi, dev, opts):
    # 12 x 20: the subsets of size <= 12 are 87% of the 2^20, so the integer-pipe Gray walk
    # over all subsets runs (not the by-size walk); with at least 2^6 chunks it hands them
    # out by the popcount of their high bits (chunk_log2 = 3, 10, planner), with fewer in
    # Gray order (chunk_log2 = 16).  Against the exact value, with and without a bound.
    import torch
    from oracle import exact
    A = inputs.uniform_real(12, 20, 6811)
    ref = float(exact.glynn_rect_grouped(A))
    o = dict(opts, arith=2)
    close(run(capi, "perm_ryser", A, dev, o), ref, A, kind="ryser", c=2, u=U_FIX)
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    out = capi.perm_ryser(to_dev(A, dev), opts=dict(o, err=err))
    torch.cuda.synchronize(dev)
    assert abs(capi.value(out, capi.PERM_F64) - ref) <= float(err.item())


def test_config_rect20x40_ryser_against_exact_golden(capi, dev):
    # the 20 x 40 uniform[0,1] workload by rectangular Ryser: 2^40 Gray-ordered subsets,
    # the 6.19e11 of size <= 20 weighted by C(40-s, 20-s); the stored truth is exact
    # (oracle.exact).  Checked within the stated bound, which must itself be far below |per|
    import torch
    gold = read_golden("rect20x40_f64.txt")
    A = inputs.rect20x40_f64()
    ref = float(gold["exact"][0]) + float(gold["exact"][1])
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    out = capi.perm_ryser(to_dev(A, dev), opts=dict(err=err))
    torch.cuda.synchronize(dev)
    got = capi.value(out, capi.PERM_F64)
    stated = float(err.item())
    print("20x40 Ryser: got %r exact %r |err|/|per| %.3g stated/|per| %.3g" % (
        got, ref, abs(got - ref) / abs(ref), stated / abs(ref)))
    assert 0.0 < stated < 1e-6 * abs(ref)
    assert abs(got - ref) <= stated + 2 * U * abs(ref)
