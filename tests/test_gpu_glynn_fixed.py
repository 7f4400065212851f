"""Parity of the integer-pipe Glynn sweep (opts.arith = PERM_ARITH_FIXED: exact
fixed-point column sums, 64-bit-mantissa products, 192-bit accumulation) with the
long-double CPU oracle.  Tolerances: c (n + 2) u sum|t| with u = 2^-60 for the
integer-pipe arithmetic (gpu_util), on the term set the kernel evaluates; rectangles
take the closed-form padding sum by default (scale "esym")."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import U, U_CFIX, U_FIX, close, device, read_golden, real_default_kind, run, scale, to_dev
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
    close(run(capi, "perm_glynn", A, dev, FIXED), oracle.glynn(A), A, rel=1e-13, c=2, u=U_FIX)


@pytest.mark.parametrize("m,n", [(1, 3), (2, 9), (5, 12), (9, 16), (13, 21)])
def test_fixed_rectangular_and_transposed(capi, dev, m, n):
    A = inputs.uniform_real(m, n, 7100 + 31 * m + n, 0.0, 1.0)
    ref = oracle.glynn(A)
    kind = real_default_kind(A)
    close(run(capi, "perm_glynn", A, dev, FIXED), ref, A, rel=1e-13, c=2, u=U_FIX, kind=kind)
    close(run(capi, "perm_glynn", np.ascontiguousarray(A.T), dev, FIXED), ref, A, rel=1e-13, c=2, u=U_FIX, kind=kind)


def test_fixed_wide_dynamic_range(capi, dev):
    # entries spanning many binades, including exact zeros and a zero column
    g = inputs.rng(7201)
    A = g.uniform(-1, 1, (12, 12)) * np.exp2(g.integers(-30, 30, (12, 12)))
    A[3, 5] = 0.0
    close(run(capi, "perm_glynn", A, dev, FIXED), oracle.glynn(A), A, rel=1e-12, c=2, u=U_FIX)
    A[:, 7] = 0.0
    assert run(capi, "perm_glynn", A, dev, FIXED) == 0.0


@pytest.mark.parametrize("n", [6, 13, 22])
def test_fixed_closed_forms(capi, dev, n):
    # the all-ones sum cancels heavily (bound on its own sum of |term|); the padded
    # identity is exact in the closed-form padding sum (one nonzero product per sign vector)
    close(run(capi, "perm_glynn", np.ones((n, n)), dev, FIXED), float(math.factorial(n)), np.ones((n, n)), rel=1e-14,
          c=2, u=U_FIX)
    assert run(capi, "perm_glynn", np.eye(n), dev, FIXED) == 1.0
    m = n // 2
    eye = np.zeros((m, n))
    eye[np.arange(m), np.arange(m)] = 1.0
    assert run(capi, "perm_glynn", eye, dev, FIXED) == 1.0


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
        close(run(capi, "perm_glynn", A, dev, opts), ref, A, rel=1e-13, c=2, u=U_FIX)


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
    # without a bound the default is the mixed sweep (the bound variant differs in the
    # last bits: it takes exact magnitudes of the column sums)
    assert run(capi, "perm_glynn", A, dev) == run(capi, "perm_glynn", A, dev, MIXED)


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


@pytest.mark.parametrize("n", [37, 41, 47, 58, 64])
def test_lane_pair_sweep_sampled_partials(capi, dev, n):
    # from n = 37 the mixed sweep runs a lane pair per term (each lane half of the
    # columns, 4 of them on the FP64 unit, one more truncated product to join the
    # halves): ragged ranges and one crossing chunk boundaries, on the planned grid, one
    # block, 7 blocks with 8-term chunks (pairs past the range's end), and the one-lane
    # kernel (block = 128), against the oracle
    import torch
    A = inputs.uniform_real(n, n, 7660 + n)
    T = 1 << (n - 1)
    for a, b in ((0, 3000), (T // 3 + 5, T // 3 + 5000), (T - 2049, T)):
        ref = oracle.glynn_partial(A, a, b)
        scale = oracle.glynn_partial_abs(A, a, b)
        tol = max(1e-13 * abs(ref), ((n - 8 + 6) * 2.0 ** -60 + 16 * 2.0 ** -53) * scale)
        for opts in (MIXED, dict(MIXED, grid=1), dict(MIXED, grid=7, chunk_log2=3), dict(MIXED, block=128)):
            out = capi.perm_glynn_partial(to_dev(A, dev), a, b, opts=opts)
            torch.cuda.synchronize(dev)
            got = capi.dd_value(out)
            assert abs(got - ref) <= tol, (n, a, b, opts, abs(got - ref), "tol/|ref|", tol / abs(ref))


# ------------------------------------------------- rectangles (m < n)
_exact_cache = {}


def _exact_rect(m, n):
    from oracle import exact
    if (m, n) not in _exact_cache:
        A = inputs.uniform_real(m, n, 7800 + 67 * m + n)
        _exact_cache[(m, n)] = float(exact.glynn_rect_grouped(A, workers=8 if m > 12 else 1))
    return _exact_cache[(m, n)]


@pytest.mark.parametrize("m,n", [(1, 2), (1, 12), (2, 11), (3, 30), (5, 13), (9, 20), (12, 17), (4, 64),
                                 (15, 16), (11, 44), (16, 33)])
@pytest.mark.parametrize("arith", [2, 3])
def test_rectangle_against_oracle(capi, dev, m, n, arith):
    # uniform[-1,1] rectangles: the padded sum of Eq. glynn_rectangle cancels up to
    # 10^16-fold here, the closed-form padding sum (default for n - m >= 3 or m <= 8)
    # like the square blocks; the truth is the oracle's long-double padded sum
    A = inputs.uniform_real(m, n, 7800 + 67 * m + n)
    # truth: long-double Glynn up to n = 20, else the padded sum in exact integers
    ref = oracle.glynn(A) if n <= 20 else _exact_rect(m, n)
    kind = real_default_kind(A)
    tol = close(run(capi, "perm_glynn", A, dev, dict(arith=arith)), ref, A, rel=1e-12, c=2, u=U_FIX, kind=kind)
    close(run(capi, "perm_glynn", np.ascontiguousarray(A.T), dev, dict(arith=arith)), ref, A, rel=1e-12, c=2,
          u=U_FIX, kind=kind)
    assert tol <= 2e-9 * abs(ref)


@pytest.mark.parametrize("opts", [dict(grid=1, block=32), dict(grid=5, block=64, chunk_log2=2),
                                  dict(grid=3, block=96, chunk_log2=1), dict(grid=152, block=128, chunk_log2=4)])
def test_closed_form_launch_shapes(capi, dev, opts):
    # the closed-form padding sum walks 2^(m-1) sign vectors in aligned chunks, a warp's
    # lanes on consecutive chunks, the column sums of every thread in shared memory: user
    # grid, block and chunk sizes (idle lanes, ragged rounds) give the same sum, and the
    # bound variant's stated error still covers the exact value
    import torch
    from oracle import exact
    A = inputs.uniform_real(11, 17, 7961)
    assert real_default_kind(A) == "esym"
    ref = float(exact.glynn_rect_grouped(A))
    close(run(capi, "perm_glynn", A, dev, opts), ref, A, rel=1e-12, c=2, u=U_FIX, kind="esym")
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    out = capi.perm_glynn(to_dev(A, dev), opts=dict(opts, err=err))
    torch.cuda.synchronize(dev)
    assert abs(capi.value(out, capi.PERM_F64) - ref) <= float(err.item())
    C = inputs.complex_gaussian(9, 14, 7962)  # truth: the oracle's rectangular Ryser
    close(run(capi, "perm_glynn", C, dev, opts), oracle.ryser_rect(C), C, rel=1e-12, c=8, u=U_CFIX, kind="esym")


@pytest.mark.parametrize("m,n", [(3, 17), (6, 40), (1, 40), (20, 40)])
def test_rectangle_all_ones(capi, dev, m, n):
    # all-ones m x n: n! / (n-m)!, every column sum an integer and e_m exact in the
    # closed-form padding sum (products of at most m integers below 2^62 ... kept to 62 bits)
    A = np.ones((m, n))
    ref = float(math.factorial(n) // math.factorial(n - m))
    close(run(capi, "perm_glynn", A, dev), ref, A, rel=1e-13, c=2, u=U_FIX, kind="esym")


@pytest.mark.parametrize("m,n", [(9, 10), (12, 14), (15, 16)])
def test_grouped_padded_walk_near_square(capi, dev, m, n):
    # n - m <= 2 and m > 8: the padded walk with the padding rows grouped by their
    # number of -1 signs (as well conditioned as the closed form here)
    A = inputs.uniform_real(m, n, 7850 + m + n)
    assert real_default_kind(A) == "glynn"
    close(run(capi, "perm_glynn", A, dev), oracle.glynn(A), A, rel=1e-12, c=2, u=U_FIX)


def test_rectangle_20x40_against_exact_golden(capi, dev):
    # the 20 x 40 uniform[0,1] workload: 2^19 sign vectors; the stored truth is the padded
    # sum in exact integers, stored with the oracle's scales.  The stated bound of the
    # closed-form sum is (m + n + 4) 2^-60 sum e_m(|c|) (plus the final rounding); the
    # quantisation of uniform[0,1] doubles is exact here
    import torch
    gold = read_golden("rect20x40_f64.txt")
    A = inputs.rect20x40_f64()
    assert int(gold["seed"][0]) == inputs.SEED_BASE + 3
    ref = float(gold["exact"][0]) + float(gold["exact"][1])
    m, n = A.shape
    S = float(gold["esym_abs"][0])
    assert abs(S - scale(A, "esym")) <= 1e-9 * S
    err = torch.zeros(1, dtype=torch.float64, device=dev)
    out = capi.perm_glynn(to_dev(A, dev), opts=dict(err=err))
    torch.cuda.synchronize(dev)
    got = capi.value(out, capi.PERM_F64)
    stated = float(err.item())
    assert 0.0 < stated <= (m + n + 4) * 2.0 ** -60 * S * 1.001 + 2 * U * abs(ref)
    assert abs(got - ref) <= stated, (got, ref, stated)
    assert stated <= 1e-12 * abs(ref)
    # the FP64 sweep of the padded sum (the paper's own evaluation, 2^39 terms) is not
    # run here: it takes minutes; its ragged term ranges are checked in test_gpu_limits


def test_grouped_rectangle_is_not_used_for_partials(capi, dev):
    # perm_glynn_partial keeps the ungrouped term index (2^(n-1) Gray-code terms)
    import torch
    A = inputs.uniform_real(5, 12, 7901)
    out = capi.perm_glynn_partial(to_dev(A, dev), 0, 1 << 11, opts=FIXED)
    torch.cuda.synchronize(dev)
    total = capi.dd_value(out) / (2.0 ** 11 * math.factorial(7))
    close(total, oracle.glynn(A), A, rel=1e-13, c=2, u=U_FIX)


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
