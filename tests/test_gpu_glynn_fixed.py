"""Parity of the integer-pipe Glynn sweep (opts.arith = PERM_ARITH_FIXED: exact
fixed-point column sums, 64-bit-mantissa products, 192-bit accumulation) with the
CPU oracle.  Same tolerances as the FP64 path; the arithmetic is more accurate."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import U, close, device, run, term_bound, to_dev
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
