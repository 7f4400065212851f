"""Parity of the combinatoric algorithm (perm_combinatoric) with the CPU oracle.

Float tolerance: 8 (n + 2) u per(|A|), the sum of |term| of the definition's terms
(gpu_util.close with kind="definition"); integers bit-exact."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import close, device, read_golden, run, to_dev
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


@pytest.mark.parametrize("m,n", [(1, 1), (1, 6), (2, 2), (3, 3), (4, 6), (5, 5), (6, 9), (8, 8), (9, 9)])
def test_dense_real_vs_definition(capi, dev, m, n):
    A = inputs.uniform_real(m, n, 8000 + 31 * m + n)
    close(run(capi, "perm_combinatoric", A, dev), oracle.definition(A), A, kind="definition")


def test_dense_real_12(capi, dev):
    A = inputs.uniform_real(12, 12, 8101)
    close(run(capi, "perm_combinatoric", A, dev), oracle.glynn(A), A, kind="definition")


@pytest.mark.parametrize("density", [0.15, 0.3])
def test_sparse_real_16(capi, dev, density):
    # the work cap counts dense leaves (16!); a sparse input is pruned, so raise it
    A = inputs.sparse_real(16, 16, density, 8200 + int(100 * density))
    close(run(capi, "perm_combinatoric", A, dev, dict(max_terms=1 << 62)), oracle.glynn(A), A, kind="definition")


@pytest.mark.parametrize("m,n", [(9, 13), (11, 14), (12, 16)])
def test_rectangular_tail_tables(capi, dev, m, n):
    # below the prefix rows the search meets the tables of the last three and four rows
    # with more free columns than rows left (sums over all triples / quadruples of the
    # free columns): uniform[0,1] against the long-double Glynn (no cancellation there),
    # a signed 9 x 13 against the exact value, and 0/1 input bit-exact
    from oracle import exact
    cap = dict(max_terms=1 << 46)
    A = inputs.uniform_real(m, n, 8800 + 31 * m + n, 0.0, 1.0)
    close(run(capi, "perm_combinatoric", A, dev, cap), oracle.glynn(A), A, kind="definition")
    if m == 9:
        S = inputs.uniform_real(m, n, 8850 + n)
        close(run(capi, "perm_combinatoric", S, dev, cap), float(exact.glynn_rect_grouped(S)), S, kind="definition")
    B = inputs.bernoulli01(m, n, 8900 + 31 * m + n, 0.5)
    assert run(capi, "perm_combinatoric", B, dev, cap) == oracle.subset_dp(B.astype(np.int64))


@pytest.mark.parametrize("opts", [dict(block=64, grid=3), dict(block=256, grid=1), dict(block=96, grid=7),
                                  dict(block=32, grid=152)])
def test_launch_shapes(capi, dev, opts):
    # the tables are built by every block and the prefixes spread over a grid-stride
    # loop: user block and grid sizes (real input takes up to 256 threads, the others
    # up to 128) must give the same sum; 12x12 real with the five-row table, 9x11
    # complex (four rows), 10x10 0/1 (int128)
    A = inputs.uniform_real(12, 12, 8961)
    close(run(capi, "perm_combinatoric", A, dev, opts), oracle.glynn(A), A, kind="definition")
    small = dict(opts, block=min(opts["block"], 128))
    C = inputs.complex_gaussian(9, 11, 8962)
    close(run(capi, "perm_combinatoric", C, dev, small), oracle.glynn(C), C, kind="definition")
    B = inputs.bernoulli01(10, 10, 8963, 0.6)
    assert run(capi, "perm_combinatoric", B, dev, small) == oracle.subset_dp(B.astype(np.int64))
    with pytest.raises(capi.PermError):
        capi.perm_combinatoric(to_dev(B, dev), opts=dict(block=256))  # int128 partials: 128 threads at most


def test_transposed_and_complex(capi, dev):
    A = inputs.uniform_real(7, 4, 8301)
    close(run(capi, "perm_combinatoric", A, dev), oracle.definition(A.T), A, kind="definition")
    C = inputs.complex_gaussian(7, 7, 8302)
    close(run(capi, "perm_combinatoric", C, dev), oracle.definition(C), C, kind="definition")


@pytest.mark.parametrize("n", [3, 7, 10])
def test_integers_exact(capi, dev, n):
    B = inputs.bernoulli01(n, n, 8400 + n, 0.6)
    assert run(capi, "perm_combinatoric", B, dev) == oracle.subset_dp(B.astype(np.int64))
    Z = inputs.rng(8500 + n).integers(-20, 21, (n - 1, n)).astype(np.int64)
    assert run(capi, "perm_combinatoric", Z, dev) == oracle.subset_dp(Z)


def test_structure(capi, dev):
    assert run(capi, "perm_combinatoric", np.eye(14), dev) == 1.0
    A = inputs.uniform_real(9, 9, 8601)
    A[4] = 0.0
    assert run(capi, "perm_combinatoric", A, dev) == 0.0
    assert run(capi, "perm_combinatoric", np.ones((6, 10), dtype=np.uint8), dev) == math.factorial(10) // math.factorial(4)


def test_work_cap(capi, dev):
    A = inputs.uniform_real(20, 20, 8701)
    with pytest.raises(capi.PermError) as e:
        capi.perm_combinatoric(A)
    assert e.value.status == capi.PERM_ETOOBIG


def test_config_square16_dense(capi, dev):
    # the 16 x 16 uniform[-1,1] workload by the combinatoric algorithm: 16! injective
    # maps (the default work cap of 2^44 leaves refuses it; the cap is raised for it),
    # against the stored long-double Glynn and Ryser values of the same matrix
    g = read_golden("square16_f64.txt")
    A = inputs.square16_f64(int(g["seed"][0]))
    ref = float(g["glynn"][0]) + float(g["glynn"][1])
    assert abs(ref - (float(g["ryser"][0]) + float(g["ryser"][1]))) <= 1e-14 * abs(ref)
    with pytest.raises(capi.PermError) as e:
        capi.perm_combinatoric(to_dev(A, dev))
    assert e.value.status == capi.PERM_ETOOBIG
    got = run(capi, "perm_combinatoric", A, dev, dict(max_terms=1 << 46))
    close(got, ref, A, kind="definition")
