"""Parity of the complex and exact-integer Glynn sweeps with the CPU oracle.

Complex tolerances: 8 (n + 2) u sum|t| on the term set the call evaluates
(gpu_util.default_kind), u = 2^-53 on the FP64 pipe and 2^-56 on the integer pipes;
truths from the long-double oracle.  Integers are bit-exact."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import U_CFIX, close, default_kind, device, read_golden, run, to_dev, tol_ratio
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


# ------------------------------------------------------------------ complex
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11, 14, 17])
def test_complex_square(capi, dev, n):
    A = inputs.complex_gaussian(n, n, 4000 + n)
    ref = oracle.glynn(A)
    close(run(capi, "perm_glynn", A, dev), ref, A, u=U_CFIX)
    assert tol_ratio(ref, A, u=U_CFIX) <= 1e-9


@pytest.mark.parametrize("m,n", [(2, 5), (4, 9), (7, 12), (10, 15)])
def test_complex_rectangular(capi, dev, m, n):
    A = inputs.complex_gaussian(m, n, 4100 + m * 31 + n)
    ref, kind = oracle.glynn(A), default_kind(A)
    close(run(capi, "perm_glynn", A, dev), ref, A, u=U_CFIX, kind=kind)
    close(run(capi, "perm_glynn", np.ascontiguousarray(A.T), dev), ref, A, u=U_CFIX, kind=kind)
    assert tol_ratio(ref, A, u=U_CFIX, kind=kind) <= 1e-9


def test_complex_real_valued_matches_real_path(capi, dev):
    A = inputs.uniform_real(13, 13, 4201)
    assert abs(run(capi, "perm_glynn", A + 0j, dev) - run(capi, "perm_glynn", A, dev)) <= 1e-13 * abs(oracle.glynn(A))


def test_complex_haar_block(capi, dev):
    A = inputs.haar_unitary_block(12, 4301)
    close(run(capi, "perm_glynn", A, dev), oracle.glynn(A), A, u=U_CFIX)


def test_complex_partial(capi, dev):
    import torch
    A = inputs.complex_gaussian(10, 10, 4401)
    out = capi.perm_glynn_partial(to_dev(A, dev), 37, 400, opts=dict(chunk_log2=4))
    torch.cuda.synchronize(dev)
    o = out.cpu().numpy()
    got = complex(o[0] + o[1], o[2] + o[3])
    ref = oracle.glynn_partial(A, 37, 400)
    assert abs(got - ref) <= 1e-12 * max(abs(ref), 1.0) * 400


# ------------------------------------------------------------------ integers (bit-exact)
@pytest.mark.parametrize("n", [1, 2, 4, 7, 10, 13, 16, 19, 22])
def test_binary_exact(capi, dev, n):
    A = inputs.bernoulli01(n, n, 5000 + n)
    assert run(capi, "perm_glynn", A, dev) == oracle.subset_dp(A.astype(np.int64))


@pytest.mark.parametrize("m,n", [(3, 6), (5, 11), (9, 14), (12, 20)])
def test_binary_rectangular_exact(capi, dev, m, n):
    A = inputs.bernoulli01(m, n, 5100 + m * 31 + n, 0.6)
    assert run(capi, "perm_glynn", A, dev) == oracle.subset_dp(A.astype(np.int64))
    assert run(capi, "perm_glynn", np.ascontiguousarray(A.T), dev) == oracle.subset_dp(A.astype(np.int64))


@pytest.mark.parametrize("n", [5, 12, 20, 26])
def test_all_ones_factorial_exact(capi, dev, n):
    assert run(capi, "perm_glynn", np.ones((n, n), dtype=np.uint8), dev) == math.factorial(n)
    m = n // 2
    assert run(capi, "perm_glynn", np.ones((m, n), dtype=np.uint8), dev) == math.factorial(n) // math.factorial(n - m)


@pytest.mark.parametrize("m,n", [(1, 24), (3, 24), (8, 24), (10, 26), (17, 18)])
def test_grouped_rectangular_exact(capi, dev, m, n):
    # the grouped rectangular walk (2^(m-1) (n-m+1) terms with binomial weights), exact
    # modulo 2^128, against the oracle's rectangular Ryser in exact 128-bit integers.
    # Host buffers: an input whose 2^(n-1) (n-m)! per(A) may leave int128 raises.
    A = inputs.rng(5150 + 7 * m + n).integers(-3, 4, (m, n)).astype(np.int64)
    out = np.zeros(2, dtype=np.int64)
    capi.perm_glynn(A, out=out)
    assert capi.value(out, capi.PERM_I64) == oracle.ryser_rect(A)
    B = inputs.bernoulli01(m, n, 5160 + m + n, 0.5)
    assert run(capi, "perm_glynn", B, dev) == oracle.ryser_rect(B.astype(np.int64))


def test_grouped_rectangular_outside_int128_is_refused(capi, dev):
    # 2^39 (40-6)! exceeds 2^127 by itself: no exact int128 result exists
    A = inputs.rng(5170).integers(-3, 4, (6, 40)).astype(np.int64)
    with pytest.raises(capi.PermError) as e:
        capi.perm_glynn(A, out=np.zeros(2, dtype=np.int64))
    assert e.value.status == capi.PERM_EOVERFLOW


@pytest.mark.parametrize("n", [4, 9, 14])
def test_int64_exact(capi, dev, n):
    A = inputs.rng(5200 + n).integers(-50, 51, (n, n)).astype(np.int64)
    assert run(capi, "perm_glynn", A, dev) == oracle.subset_dp(A)


def test_int64_host_buffers_and_overflow_status(capi, dev):
    A = inputs.rng(5301).integers(-9, 10, (8, 8)).astype(np.int64)
    out = np.zeros(2, dtype=np.int64)
    capi.perm_glynn(A, out=out)
    assert capi.value(out, capi.PERM_I64) == oracle.subset_dp(A)
    big = np.full((20, 20), 1 << 40, dtype=np.int64)
    with pytest.raises(capi.PermError) as e:
        capi.perm_glynn(big, out=np.zeros(2, dtype=np.int64))
    assert e.value.status == capi.PERM_EOVERFLOW


def test_device_overflow_status(capi, dev):
    import ctypes

    import torch
    big = torch.full((20, 20), 1 << 40, dtype=torch.int64, device=dev)
    capi.perm_glynn(big)
    st = ctypes.c_int(-1)
    assert capi.lib().perm_device_status(capi.handle(0), None, ctypes.byref(st)) == 0
    assert st.value == capi.PERM_EOVERFLOW
    A = torch.ones((6, 6), dtype=torch.uint8, device=dev)
    capi.perm_glynn(A)
    assert capi.lib().perm_device_status(capi.handle(0), None, ctypes.byref(st)) == 0
    assert st.value == 0


def test_int_partial_modular(capi, dev):
    import torch
    A = inputs.rng(5401).integers(-3, 4, (9, 12)).astype(np.int64)
    for a, b in [(0, 2048), (5, 777), (1000, 1001)]:
        out = capi.perm_glynn_partial(to_dev(A, dev), a, b)
        torch.cuda.synchronize(dev)
        assert capi.value(out, capi.PERM_I64) == oracle.glynn_partial(A, a, b)


def test_config_square26_binary_golden(capi, dev):
    g = read_golden("square26_01.txt")
    A = inputs.square26_01(int(g["seed"][0]))
    assert run(capi, "perm_glynn", A, dev) == int(g["per"][0])


@pytest.mark.parametrize("m,n", [(3, 3), (6, 6), (10, 10), (13, 13), (16, 16), (7, 12), (11, 18)])
def test_complex_integer_pipes(capi, dev, m, n):
    # opts.arith = PERM_ARITH_FIXED: fixed-point column sums and a complex software float
    A = inputs.complex_gaussian(m, n, 4500 + 31 * m + n)
    ref = oracle.glynn(A)
    close(run(capi, "perm_glynn", A, dev, dict(arith=2)), ref, A, u=U_CFIX, kind=default_kind(A, 2))
    assert tol_ratio(ref, A, u=U_CFIX, kind=default_kind(A, 2)) <= 1e-9
    if m == n:
        # the FP64 sweep evaluates the padded sum, which cancels 10^6-fold and more on
        # these complex rectangles: it is checked on the squares
        close(run(capi, "perm_glynn", A, dev, dict(arith=1)), ref, A)


def test_complex_integer_pipes_haar_and_partial(capi, dev):
    import torch
    A = inputs.haar_unitary_block(14, 4601)
    close(run(capi, "perm_glynn", A, dev, dict(arith=2)), oracle.glynn(A), A, u=U_CFIX)
    B = inputs.complex_gaussian(11, 11, 4602)
    out = capi.perm_glynn_partial(to_dev(B, dev), 100, 900, opts=dict(arith=2))
    torch.cuda.synchronize(dev)
    o = out.cpu().numpy()
    got = complex(o[0] + o[1], o[2] + o[3])
    ref = oracle.glynn_partial(B, 100, 900)
    assert abs(got - ref) <= 1e-12 * 800 * max(1.0, abs(ref))


@pytest.mark.parametrize("m,n", [(1, 30), (3, 30), (6, 40), (9, 22), (20, 21)])
def test_complex_rectangle_closed_form_padding(capi, dev, m, n):
    # complex rectangles on the integer pipes (default for n >= 10): the padding summed
    # in closed form, 2^(m-1) sign vectors, against the oracle's rectangular Ryser
    A = inputs.complex_gaussian(m, n, 4700 + 13 * m + n)
    ref = oracle.ryser_rect(A)
    assert default_kind(A) == "esym"
    close(run(capi, "perm_glynn", A, dev), ref, A, u=U_CFIX, kind="esym")
    close(run(capi, "perm_glynn", np.ascontiguousarray(A.T), dev, dict(arith=2)), ref, A, u=U_CFIX, kind="esym")
    assert tol_ratio(ref, A, u=U_CFIX, kind="esym") <= 1e-9


_ref_cache = {}


@pytest.mark.parametrize("n", [20, 21])
@pytest.mark.parametrize("arith", [0, 2, 3])
def test_complex_fp64_share(capi, dev, n, arith):
    # from n = 20 MIXED multiplies 3n/8 of each product's columns on the FP64 unit; the
    # default and FIXED keep all on the integer pipes
    A = inputs.complex_gaussian(n, n, 4800 + n)
    if n not in _ref_cache:
        _ref_cache[n] = oracle.glynn(A)
    ref = _ref_cache[n]
    close(run(capi, "perm_glynn", A, dev, dict(arith=arith)), ref, A, u=U_CFIX)
    assert tol_ratio(ref, A, u=U_CFIX) <= 1e-9


def test_complex_fp64_share_sampled_n32(capi, dev):
    import torch
    A = inputs.square32_c128()
    T = 1 << 31
    for a, b in ((0, 3000), (T // 2 - 1500, T // 2 + 1500), (T - 2999, T)):
        out = capi.perm_glynn_partial(to_dev(A, dev), a, b, opts=dict(arith=3))
        torch.cuda.synchronize(dev)
        o = out.cpu().numpy()
        got = complex(o[0] + o[1], o[2] + o[3])
        ref = oracle.glynn_partial(A, a, b)
        # 3000 terms of comparable size (no strong cancellation in a random complex
        # partial sum): 2^-50 relative per term is far inside 1e-12 of the sum
        assert abs(got - ref) <= 1e-12 * abs(ref)
