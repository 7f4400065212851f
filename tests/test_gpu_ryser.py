"""Parity of the Ryser sweeps (perm_ryser) with the CPU oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import close, device, read_golden, run
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
    close(run(capi, "perm_ryser", A, dev), oracle.ryser(A), A)


@pytest.mark.parametrize("m,n", [(1, 5), (2, 7), (4, 9), (6, 13), (10, 16), (3, 18)])
def test_rectangular_real(capi, dev, m, n):
    A = inputs.uniform_real(m, n, 6100 + 31 * m + n, 0.0, 1.0)
    close(run(capi, "perm_ryser", A, dev), oracle.ryser_rect(A), A)
    close(run(capi, "perm_ryser", np.ascontiguousarray(A.T), dev), oracle.ryser_rect(A), A)


@pytest.mark.parametrize("opts", [dict(chunk_log2=1), dict(grid=5, block=64, chunk_log2=3)])
def test_launch_shapes(capi, dev, opts):
    A = inputs.uniform_real(11, 14, 6201)
    close(run(capi, "perm_ryser", A, dev, opts), oracle.ryser_rect(A), A)


def test_config_square16_golden(capi, dev):
    g = read_golden("square16_f64.txt")
    A = inputs.square16_f64(int(g["seed"][0]))
    ref = float(g["ryser"][0]) + float(g["ryser"][1])
    assert abs(run(capi, "perm_ryser", A, dev) - ref) <= 1e-12 * abs(ref)
    assert abs(run(capi, "perm_glynn", A, dev) - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("m,n", [(4, 4), (7, 7), (3, 9), (8, 13), (12, 12)])
def test_complex(capi, dev, m, n):
    A = inputs.complex_gaussian(m, n, 6300 + 31 * m + n)
    close(run(capi, "perm_ryser", A, dev), oracle.glynn(A), A)


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
    close(run(capi, "perm_ryser", A, dev), ref, A)
    close(run(capi, "perm_ryser", A, dev, dict(chunk_log2=3)), ref, A)
    close(run(capi, "perm_ryser", np.ascontiguousarray(A.T), dev), ref, A)
