"""Parity of perm_cauchy (Borchardt's theorem, Eq. caucy_permanent, in multi-limb
floating point) with the oracle's exact rational permanents of the same Cauchy
matrices.  The kernel returns the permanent of the exact matrix of the given doubles
rounded to double, so the bar is one unit in the last place of the exact value."""
import os

import numpy as np
import pytest

import oracle
from gpu_util import GOLDEN, device
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu

ULP = 2.0 ** -52


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


def gpu_cauchy(capi, dev, x, y, want_err=False):
    import torch
    dx = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    dy = torch.from_numpy(np.ascontiguousarray(y)).to(dev)
    n = x.shape[-1]
    count = x.size // n
    err = torch.full((count,), -1.0, dtype=torch.float64, device=dev) if want_err else None
    out = capi.perm_cauchy(dx, dy, opts={"err": err} if want_err else None)
    torch.cuda.synchronize(dev)
    return (out.cpu().numpy(), err.cpu().numpy()) if want_err else out.cpu().numpy()


def exact(x, y):
    return oracle.cauchy.permanent_borchardt(x, y)


def within_ulp(got, ex):
    return abs(got - float(ex)) <= ULP * abs(float(ex))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11, 16, 20])
def test_small_orders_exact_value(capi, dev, n):
    x, y = inputs.cauchy_points(n, 1200 + n, count=3)
    got, err = gpu_cauchy(capi, dev, x, y, want_err=True)
    for b in range(3):
        ex = exact(x[b], y[b])
        assert within_ulp(got[b], ex), (b, got[b], float(ex))
        assert abs(got[b] - float(ex)) <= err[b] <= 2.0 ** -50 * abs(got[b])
    if n <= 7:
        C = oracle.cauchy.cauchy_matrix(x[0], y[0])
        assert within_ulp(got[0], oracle.cauchy.permanent_definition(C))


@pytest.mark.parametrize("n", [4, 9, 14])
def test_interleaved_points_entries_of_both_signs(capi, dev, n):
    g = inputs.rng(1300 + n)
    pts = g.permutation(g.uniform(-1.0, 1.0, 2 * n))
    x, y = pts[:n].copy(), pts[n:].copy()
    got = gpu_cauchy(capi, dev, x[None], y[None])
    assert within_ulp(got[0], exact(x, y))


def golden_cases():
    path = os.path.join(GOLDEN, "cauchy_exact.txt")
    cases = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        kv = dict(zip(f[0::2], f[1::2]))
        cases.append({k: (float(v) if k == "per" else int(v)) for k, v in kv.items()})
    return cases


def test_large_orders_against_stored_exact_values(capi, dev):
    # orders whose exact evaluation takes the oracle minutes; values written by
    # tests/golden/make_golden.py from oracle.cauchy alone
    seen = set()
    for case in golden_cases():
        n, seed, count, b = case["n"], case["seed"], case["count"], case["index"]
        key = (n, seed, count)
        if key in seen:
            continue
        seen.add(key)
        x, y = inputs.cauchy_points(n, seed, count=count)
        got, err = gpu_cauchy(capi, dev, x, y, want_err=True)
        for c in golden_cases():
            if (c["n"], c["seed"], c["count"]) == key:
                i = c["index"]
                assert abs(got[i] - c["per"]) <= ULP * abs(c["per"]), (n, i, got[i], c["per"])
                assert err[i] <= 2.0 ** -50 * abs(got[i])
        assert np.all(np.isfinite(got)) and np.all(got > 0)  # x > y: every term is positive


def test_host_and_device_buffers_agree_and_repeat_bit_for_bit(capi, dev):
    x, y = inputs.cauchy_points(18, 1400, count=5)
    a = gpu_cauchy(capi, dev, x, y)
    host = capi.perm_cauchy(x, y)
    b = gpu_cauchy(capi, dev, x, y)
    assert np.array_equal(a, host) and np.array_equal(a, b)
    one = capi.perm_cauchy(x[2], y[2])
    assert one.shape == (1,) and one[0] == a[2]


def test_coinciding_points_give_nan_and_a_status(capi, dev):
    import torch
    stream = torch.cuda.current_stream(dev).cuda_stream
    st = capi.ctypes.c_int(-1)
    assert capi.lib().perm_device_status(capi.handle(0), stream, capi.ctypes.byref(st)) == capi.PERM_OK  # clear
    x, y = inputs.cauchy_points(6, 1500, count=4)
    x[1, 3] = x[1, 0]          # repeated x: det(C) = 0
    y[2, 5] = x[2, 2]          # infinite entry
    x[3, 4] = np.inf
    got = gpu_cauchy(capi, dev, x, y)
    assert np.isfinite(got[0]) and np.all(np.isnan(got[1:]))
    rc = capi.lib().perm_device_status(capi.handle(0), stream, capi.ctypes.byref(st))
    assert rc == capi.PERM_OK and st.value == capi.PERM_EINVAL
    with pytest.raises(capi.PermError) as e:
        capi.perm_cauchy(x, y)  # host output: the status comes back from the call
    assert e.value.status == capi.PERM_EINVAL


def test_argument_errors(capi, dev):
    x, y = inputs.cauchy_points(65, 1600)
    with pytest.raises(capi.PermError) as e:
        capi.perm_cauchy(x, y)
    assert e.value.status == capi.PERM_ETOOBIG
    empty = np.zeros((0, 5))
    assert capi.perm_cauchy(empty, empty).shape == (0,)


def test_order_64_top_of_the_range(capi, dev):
    # at n = 64 every entry is in [2/3, 2]; per lies between 64! (2/3)^64 and 64! 2^64
    import math
    x, y = inputs.cauchy_points(64, 1700, count=2)
    got = gpu_cauchy(capi, dev, x, y)
    lo = math.lgamma(65) + 64 * math.log(2.0 / 3.0)
    hi = math.lgamma(65) + 64 * math.log(2.0)
    for v in got:
        assert lo <= math.log(v) <= hi


# --- perm_auto recognises a Cauchy matrix given as a dense double matrix


def cauchy_matrix_double(x, y):
    return 1.0 / (x[:, None] - y[None, :])


def auto_choice(capi, A):
    import ctypes
    cand = ctypes.c_int(-1)
    A = np.ascontiguousarray(A)
    rc = capi.lib().perm_auto_choice(capi.handle(0), A.ctypes.data, A.shape[0], A.shape[1], A.shape[1],
                                     capi.PERM_F64, None, ctypes.byref(cand), None)
    assert rc == capi.PERM_OK
    return cand.value


def test_perm_auto_takes_borchardt_for_cauchy_matrices(capi, dev):
    import torch
    for case in golden_cases():
        if case["count"] != 1:
            continue
        n = case["n"]
        x, y = inputs.cauchy_points(n, case["seed"])
        A = cauchy_matrix_double(x[0], y[0])
        assert auto_choice(capi, A) == capi.PERM_CAND_CAUCHY, n
        err = torch.zeros(1, dtype=torch.float64, device=dev)
        out = capi.perm_auto(torch.from_numpy(A).to(dev), opts={"err": err})
        torch.cuda.synchronize(dev)
        got, e = float(out.item()), float(err.item())
        # A is the exact matrix of the points rounded entrywise (two roundings: |rel| <= 2u),
        # and every term is positive: per(A) is within n 2u of the stored per(C); the fit
        # adds at most n 2^-48, the result's own rounding 1 ulp
        tol = (n * 2.0 ** -52 + n * 2.0 ** -48 * 1.01 + 2.0 ** -52) * case["per"]
        assert abs(got - case["per"]) <= tol, (n, got, case["per"])
        assert 0 < e <= (n * 2.0 ** -48 * 1.01 + 2.0 ** -50) * got
        host = capi.perm_auto(A)
        assert float(host[0]) == got


def test_perm_auto_keeps_the_general_path_off_cauchy_structure(capi, dev):
    x, y = inputs.cauchy_points(26, 1800)
    A = cauchy_matrix_double(x[0], y[0])
    assert auto_choice(capi, A) == capi.PERM_CAND_CAUCHY
    B = A.copy()
    B[3, 7] *= 1.0 + 1e-9  # no longer 1/(x_i - y_j) within 2^-48
    assert auto_choice(capi, B) != capi.PERM_CAND_CAUCHY
    g = inputs.rng(1801)
    pts = g.permutation(g.uniform(-1.0, 1.0, 52))  # Cauchy, but entries of both signs
    assert auto_choice(capi, cauchy_matrix_double(pts[:26], pts[26:])) != capi.PERM_CAND_CAUCHY
    x, y = inputs.cauchy_points(20, 1802)  # below the order where the ladder pays
    assert auto_choice(capi, cauchy_matrix_double(x[0], y[0])) != capi.PERM_CAND_CAUCHY


def test_invariances_scaling_translation_permutation(capi, dev):
    # c_ij(2^k x, 2^k y) = 2^-k c_ij(x, y): per scales by 2^(-k n) exactly, while det(C)
    # and det(C o C) leave the double range by far (2^(+-k n^2)); a shift of both point
    # sets leaves C unchanged (points on a dyadic grid, so the shift is exact); permuting
    # the points permutes rows or columns
    import math
    g = inputs.rng(1900)
    n = 8
    x = np.round(g.uniform(0.25, 0.75, n) * 2 ** 20) / 2 ** 20
    y = np.round(g.uniform(-0.75, -0.25, n) * 2 ** 20) / 2 ** 20
    base = gpu_cauchy(capi, dev, x[None], y[None])[0]
    assert within_ulp(base, exact(x, y))
    for k in (-100, 60, 110):
        got = gpu_cauchy(capi, dev, np.ldexp(x, k)[None], np.ldexp(y, k)[None])[0]
        assert got == math.ldexp(base, -k * n), k
    shifted = gpu_cauchy(capi, dev, (x + 3.0)[None], (y + 3.0)[None])[0]
    assert shifted == base
    p, q = g.permutation(n), g.permutation(n)
    assert gpu_cauchy(capi, dev, x[p][None], y[q][None])[0] == base


def test_perm_auto_cauchy_strided_and_transposed_operands(capi, dev):
    # the fit reads the operand through its strides: a view with ld > n, and the
    # transpose (a Cauchy matrix with the roles of x and -y exchanged), give the same value
    import torch
    x, y = inputs.cauchy_points(30, 1850)
    A = cauchy_matrix_double(x[0], y[0])
    dense = capi.perm_auto(torch.from_numpy(A).to(dev))
    big = torch.zeros((30, 37), dtype=torch.float64, device=dev)
    big[:, 3:33] = torch.from_numpy(A).to(dev)
    view = capi.perm_auto(big[:, 3:33])
    tr = capi.perm_auto(torch.from_numpy(A.T.copy()).to(dev))
    torch.cuda.synchronize(dev)
    exact_v = float(oracle.cauchy.permanent_borchardt(x[0], y[0]))
    tol = (30 * 2.0 ** -52 + 30 * 2.0 ** -48 * 1.01 + 2.0 ** -52) * exact_v
    for v in (dense, view, tr):
        assert abs(float(v.item()) - exact_v) <= tol
    assert float(view.item()) == float(dense.item())


def test_vanishing_permanent_of_order_two(capi, dev):
    # x = (0, 1), y = (3/2, 3/4): C = [[-2/3, -4/3], [-2, 4]], per(C) = -8/3 + 8/3 = 0 and
    # det(C o C) = 0; the two entries of the first row differ by a power of two, so the
    # elimination cancels exactly and the call returns zero with a zero error estimate
    x = np.array([[0.0, 1.0]])
    y = np.array([[1.5, 0.75]])
    C = oracle.cauchy.cauchy_matrix(x[0], y[0])
    assert oracle.cauchy.permanent_definition(C) == 0
    got, err = gpu_cauchy(capi, dev, x, y, want_err=True)
    assert got[0] == 0.0 and err[0] == 0.0


# --- SBP coefficients of a Cauchy coefficient matrix (perm_cauchy_sbp)


def test_cauchy_sbp_matches_gathered_points_and_exact_values(capi, dev):
    import torch
    g = inputs.rng(2200)
    n, N, count = 6, 14, 500
    x = g.uniform(0.25, 0.75, n)        # rapidities
    y = g.uniform(-0.75, -0.25, N)      # single-particle energies
    cols = np.argsort(g.random((count, N)), axis=1)[:, :n]
    occ = np.bitwise_or.reduce(np.left_shift(np.uint64(1), cols.astype(np.uint64)), axis=1)
    out = capi.perm_cauchy_sbp(torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev),
                               torch.from_numpy(occ.view(np.int64)).to(dev))
    torch.cuda.synchronize(dev)
    got = out.cpu().numpy()
    ys = np.stack([y[[j for j in range(N) if (int(o) >> j) & 1]] for o in occ])
    xs = np.tile(x, (count, 1))
    ref = gpu_cauchy(capi, dev, xs, ys)
    assert np.array_equal(got, ref)  # the same points through perm_cauchy: bit-identical
    for k in range(0, count, 50):  # and exact: the oracle's C P (Eq. SBGpermanent) in rationals
        assert within_ulp(got[k], exact(x, ys[k]))
    host = capi.perm_cauchy_sbp(x, y, occ)
    assert np.array_equal(host, got)


def test_cauchy_sbp_bad_bitstrings_and_limits(capi, dev):
    import torch
    stream = torch.cuda.current_stream(dev).cuda_stream
    st = capi.ctypes.c_int(-1)
    assert capi.lib().perm_device_status(capi.handle(0), stream, capi.ctypes.byref(st)) == capi.PERM_OK
    x = np.array([0.3, 0.6])
    y = np.array([-0.3, -0.5, -0.7])
    occ = np.array([0b011, 0b111, 0b1001, 0b110], dtype=np.uint64)  # 2nd: three states, 3rd: state 3 >= N
    out = capi.perm_cauchy_sbp(torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev),
                               torch.from_numpy(occ.view(np.int64)).to(dev))
    torch.cuda.synchronize(dev)
    got = out.cpu().numpy()
    assert np.isfinite(got[0]) and np.isnan(got[1]) and np.isnan(got[2]) and np.isfinite(got[3])
    assert within_ulp(got[3], exact(x, y[[1, 2]]))
    assert capi.lib().perm_device_status(capi.handle(0), stream, capi.ctypes.byref(st)) == capi.PERM_OK
    assert st.value == capi.PERM_EINVAL
    with pytest.raises(capi.PermError) as e:
        capi.perm_cauchy_sbp(x, np.zeros(65), np.array([3], dtype=np.uint64))
    assert e.value.status == capi.PERM_ETOOBIG


def test_side_stream_result_read_after_that_stream(capi, dev):
    # a call on a side stream writes its result on that stream; after that stream is
    # synchronised the value read equals the exact Borchardt value of the same points
    import torch
    side = torch.cuda.Stream(device=dev)
    for n in (8, 12, 16):
        x, y = inputs.cauchy_points(n, inputs.SEED_BASE + 20 + n, draws=100)
        dx, dy = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
        torch.cuda.synchronize(dev)
        out = capi.perm_cauchy(dx, dy, stream=side)
        side.synchronize()
        got = float(out[0].item())
        exact = float(oracle.cauchy.permanent_borchardt(x[0], y[0]))
        assert got > 0.0
        assert abs(got - exact) <= 2.0 ** -52 * abs(exact), (n, got, exact)
