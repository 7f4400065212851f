"""Parity of the integer-pipe Glynn sweep (opts.arith = PERM_ARITH_FIXED: exact
fixed-point column sums, 64-bit-mantissa products, 192-bit accumulation) with the
CPU oracle.  Same tolerances as the FP64 path; the arithmetic is more accurate."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import U, close, device, read_golden, run, term_bound, to_dev
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu

FIXED = dict(arith=2)


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 11, 14, 17, 20, 23])
def test_fixed_square(capi, dev, n):
    A = inputs.uniform_real(n, n, 7000 + n)
    close(run(capi, "perm_glynn", A, dev, FIXED), oracle.glynn(A), A, rel=1e-13)


@pytest.mark.parametrize("m,n", [(1, 3), (2, 9), (5, 12), (9, 16), (13, 21)])
def test_fixed_rectangular_and_transposed(capi, dev, m, n):
    A = inputs.uniform_real(m, n, 7100 + 31 * m + n, 0.0, 1.0)
    ref = oracle.glynn(A)
    close(run(capi, "perm_glynn", A, dev, FIXED), ref, A, rel=1e-13)
    close(run(capi, "perm_glynn", np.ascontiguousarray(A.T), dev, FIXED), ref, A, rel=1e-13)


def test_fixed_wide_dynamic_range(capi, dev):
    # entries spanning many binades, including exact zeros and a zero column
    g = inputs.rng(7201)
    A = g.uniform(-1, 1, (12, 12)) * np.exp2(g.integers(-30, 30, (12, 12)))
    A[3, 5] = 0.0
    close(run(capi, "perm_glynn", A, dev, FIXED), oracle.glynn(A), A, rel=1e-12)
    A[:, 7] = 0.0
    assert run(capi, "perm_glynn", A, dev, FIXED) == 0.0


@pytest.mark.parametrize("n", [6, 13, 22])
def test_fixed_closed_forms(capi, dev, n):
    # the ones and padded-identity sums cancel heavily: first-order bound as for FP64
    close(run(capi, "perm_glynn", np.ones((n, n)), dev, FIXED), float(math.factorial(n)), np.ones((n, n)), rel=1e-14)
    assert run(capi, "perm_glynn", np.eye(n), dev, FIXED) == 1.0
    m = n // 2
    eye = np.zeros((m, n))
    eye[np.arange(m), np.arange(m)] = 1.0
    close(run(capi, "perm_glynn", eye, dev, FIXED), 1.0, eye)


def test_fixed_error_bound_and_grid_shapes(capi, dev):
    import torch
    A = inputs.uniform_real(18, 18, 7301)
    ref = oracle.glynn(A)
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    out = capi.perm_glynn(to_dev(A, dev), opts=dict(arith=2, err=err))
    torch.cuda.synchronize(dev)
    got = capi.value(out, capi.PERM_F64)
    assert abs(got - ref) <= float(err.item()) + 2 * U * abs(ref)
    for opts in (dict(arith=2, grid=1, block=32), dict(arith=2, grid=9, block=96)):
        close(run(capi, "perm_glynn", A, dev, opts), ref, A, rel=1e-13)


def test_fixed_partial_and_sampled_n36(capi, dev):
    import torch
    A = inputs.square36_f64()
    T = 1 << 35
    for a in (0, T // 3 + 77, T - 4096):
        out = capi.perm_glynn_partial(to_dev(A, dev), a, a + 4096, opts=FIXED)
        torch.cuda.synchronize(dev)
        got = capi.dd_value(out)
        ref = oracle.glynn_partial(A, a, a + 4096)
        scale = oracle.glynn_partial_abs(A, a, a + 4096)
        assert abs(got - ref) <= max(1e-13 * abs(ref), 8 * 38 * 2.0 ** -62 * scale + 1e-18 * scale)


def test_fixed_matches_fp64_path_at_n24(capi, dev):
    A = inputs.uniform_real(24, 24, 7401)
    f = run(capi, "perm_glynn", A, dev, FIXED)
    d = run(capi, "perm_glynn", A, dev, dict(arith=1))
    assert abs(f - d) <= 1e-12 * abs(d)


def test_fixed_nonfinite_input_gives_nan(capi, dev):
    A = inputs.uniform_real(6, 6, 7501)
    A[2, 2] = np.inf
    assert math.isnan(run(capi, "perm_glynn", A, dev, FIXED))


# ---------------------------------------------------------------- mixed arithmetic
MIXED = dict(arith=3)


@pytest.mark.parametrize("n", [10, 13, 16, 19, 21])
def test_mixed_square(capi, dev, n):
    # the last 4 columns of each term multiplied on the FP64 unit (2^-53 per factor)
    A = inputs.uniform_real(n, n, 7600 + n)
    close(run(capi, "perm_glynn", A, dev, MIXED), oracle.glynn(A), A, rel=1e-12)


@pytest.mark.parametrize("n", [26, 30, 34])
def test_mixed_sampled_partials(capi, dev, n):
    # padded orders 28, 32, 36: 4, 6 and 8 columns on the FP64 unit; sampled term
    # ranges (ragged ends, a range crossing a chunk boundary) against the oracle
    import torch
    A = inputs.uniform_real(n, n, 7650 + n)
    T = 1 << (n - 1)
    K = {26: 4, 30: 6, 34: 8}[n]
    for a, b in ((0, 3000), (T // 3 + 5, T // 3 + 5000), (T - 2049, T)):
        out = capi.perm_glynn_partial(to_dev(A, dev), a, b, opts=MIXED)
        torch.cuda.synchronize(dev)
        got = capi.dd_value(out)
        ref = oracle.glynn_partial(A, a, b)
        scale = oracle.glynn_partial_abs(A, a, b)
        assert abs(got - ref) <= max(1e-13 * abs(ref), ((n - K + 5) * 2.0 ** -60 + 2 * K * 2.0 ** -53) * scale)


def test_mixed_is_default_and_error_bound_holds(capi, dev):
    import torch
    A = inputs.uniform_real(22, 22, 7701)
    ref = oracle.glynn(A)
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    out = capi.perm_glynn(to_dev(A, dev), opts=dict(err=err))
    torch.cuda.synchronize(dev)
    got = capi.value(out, capi.PERM_F64)
    assert abs(got - ref) <= float(err.item()) + 2 * U * abs(ref)
    assert got == run(capi, "perm_glynn", A, dev, MIXED)


def test_mixed_sampled_n36_against_oracle_partials(capi, dev):
    import torch
    A = inputs.square36_f64()
    T = 1 << 35
    for a in (4096, T // 2 + 12345, T - 8192):
        out = capi.perm_glynn_partial(to_dev(A, dev), a, a + 4096, opts=MIXED)
        torch.cuda.synchronize(dev)
        got = capi.dd_value(out)
        ref = oracle.glynn_partial(A, a, a + 4096)
        scale = oracle.glynn_partial_abs(A, a, a + 4096)
        # 28 integer columns (< 2^-60 per column) and 8 on the FP64 unit (2 x 2^-53 each)
        assert abs(got - ref) <= max(1e-13 * abs(ref), (33 * 2.0 ** -60 + 16 * 2.0 ** -53) * scale)


# ------------------------------------------------- grouped rectangular walk (m < n)
@pytest.mark.parametrize("m,n", [(1, 2), (1, 12), (2, 11), (3, 30), (5, 13), (9, 20), (12, 17), (4, 64),
                                 (15, 16), (11, 44), (16, 33)])
@pytest.mark.parametrize("arith", [2, 3])
def test_grouped_rectangle_against_oracle(capi, dev, m, n, arith):
    # 2^(m-1) (n-m+1) grouped terms instead of 2^(n-1); the oracle's grouped sum is
    # pinned against its ungrouped Glynn, Ryser and the definition on small shapes
    A = inputs.uniform_real(m, n, 7800 + 67 * m + n)
    ref = oracle.glynn(A) if n <= 20 else oracle.glynn_rect_grouped(A)
    close(run(capi, "perm_glynn", A, dev, dict(arith=arith)), ref, A, rel=1e-12)
    close(run(capi, "perm_glynn", np.ascontiguousarray(A.T), dev, dict(arith=arith)), ref, A, rel=1e-12)


@pytest.mark.parametrize("m,n", [(1, 40), (3, 17), (6, 40), (20, 40)])
def test_grouped_rectangle_all_ones(capi, dev, m, n):
    # all-ones m x n: n! / (n-m)!; the alternating binomial sums cancel completely
    A = np.ones((m, n))
    ref = float(math.factorial(n) // math.factorial(n - m))
    close(run(capi, "perm_glynn", A, dev), ref, A, rel=1e-13)


def test_grouped_rectangle_20x40_against_golden(capi, dev):
    # the 20 x 40 uniform[0,1] workload: 2^19 x 21 grouped terms; value and sum |t| from
    # the oracle (grouped sum in long double).  The sum cancels (sum|t| / |per| ~ 4e7), so
    # the tolerance is the stated bound of each side plus the oracle's long-double bound
    import torch
    gold = read_golden("rect20x40_f64.txt")
    A = inputs.rect20x40_f64()
    assert int(gold["seed"][0]) == inputs.SEED_BASE + 3
    ref = float(gold["glynn"][0]) + float(gold["glynn"][1])
    m, n = A.shape
    norm = 2.0 ** (n - 1) * math.factorial(n - m)
    scale = float(gold["sum_abs"][0]) / norm
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    out = capi.perm_glynn(to_dev(A, dev), opts=dict(err=err))
    torch.cuda.synchronize(dev)
    got = capi.value(out, capi.PERM_F64)
    stated = float(err.item())
    assert 0.0 < stated <= (n + 5) * 2.0 ** -60 * scale * 1.001
    oracle_bound = (n + 4) * 2.0 ** -64 * scale
    assert abs(got - ref) <= stated + oracle_bound + 1e-15 * abs(ref), (got, ref, stated)


def test_grouped_rectangle_is_not_used_for_partials(capi, dev):
    # perm_glynn_partial keeps the ungrouped term index (2^(n-1) Gray-code terms)
    import torch
    A = inputs.uniform_real(5, 12, 7901)
    out = capi.perm_glynn_partial(to_dev(A, dev), 0, 1 << 11, opts=FIXED)
    torch.cuda.synchronize(dev)
    total = capi.dd_value(out) / (2.0 ** 11 * math.factorial(7))
    close(total, oracle.glynn(A), A, rel=1e-13)


def test_resumable_sweep_on_the_gpu(capi, dev, tmp_path):
    # a sweep cut into term ranges through perm_glynn_partial, interrupted and resumed
    # from its checkpoint, against the oracle
    import torch

    from paper_2510_03421_gb300 import shard
    A = inputs.uniform_real(20, 20, 7950)
    dA = torch.from_numpy(A).to(dev)

    def part(M, a, b):
        o = capi.perm_glynn_partial(dA, a, b)
        torch.cuda.synchronize(dev)
        return float(o[0]), float(o[1])

    path = str(tmp_path / "ck.json")
    assert shard.resumable_glynn(A, part, path, step_terms=1 << 16, stop_after=3) is None
    got = shard.resumable_glynn(A, part, path, step_terms=1 << 16)
    close(got, oracle.glynn(A), A, rel=1e-13)
