"""Parity of perm_sbp (SBP coefficients c_m = per(C P), Eq. SBGpermanent) with the
long-double CPU oracle, which forms C P by a matrix product with the selection
matrix.  Each coefficient is a square Glynn sum: tolerance 8 (n + 2) u sum|t| of that
n x n matrix (u = 2^-56 for the complex integer-pipe items)."""
import itertools

import numpy as np
import pytest

import oracle
from gpu_util import U_CFIX, close, device, scale
from paper_2510_03421_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return device()


@pytest.fixture(scope="module")
def capi():
    from paper_2510_03421_gb300 import capi
    return capi


def bits(cols):
    return sum(1 << j for j in cols)


def sample_occ(g, n, N, count):
    return np.array([bits(sorted(g.choice(N, n, replace=False))) for _ in range(count)], dtype=np.uint64)


def coef(capi, out, code, k):
    return capi.value(out, code, k)


def test_real_all_bitstrings_lane_items(capi, dev):
    import torch
    g = inputs.rng(9900)
    n, N = 6, 14
    C = g.uniform(-1, 1, (n, N))
    occ = np.array([bits(S) for S in itertools.combinations(range(N), n)], dtype=np.uint64)
    out = capi.perm_sbp(torch.from_numpy(C).to(dev), torch.from_numpy(occ.view(np.int64)).to(dev))
    torch.cuda.synchronize(dev)
    got = out.cpu().numpy()
    total_scale = 0.0
    for k in range(len(occ)):
        M = C[:, [j for j in range(N) if (int(occ[k]) >> j) & 1]]
        total_scale += scale(M)
        if k % 7 == 0:
            close(got[k], oracle.sbp_coefficient(C, int(occ[k])), M)
    # every injective map rows -> states has one image: the coefficients sum to the
    # rectangular permanent of C (each coefficient's error bounded by its own scale)
    close(float(np.sum(got)), oracle.glynn_rect_grouped(C), C, rel=1e-11, s=total_scale * (1 + len(occ) / 1e13))


@pytest.mark.parametrize("n,N", [(10, 20), (16, 40)])
def test_complex_sampled_lane_items(capi, dev, n, N):
    import torch
    g = inputs.rng(9910 + n)
    C = (g.standard_normal((n, N)) + 1j * g.standard_normal((n, N))) / np.sqrt(2 * n)
    occ = sample_occ(g, n, N, 200)
    out = capi.perm_sbp(torch.from_numpy(C).to(dev), torch.from_numpy(occ.view(np.int64)).to(dev))
    torch.cuda.synchronize(dev)
    for k in range(0, len(occ), 10 if n > 12 else 1):
        M = C[:, [j for j in range(N) if (int(occ[k]) >> j) & 1]]
        close(coef(capi, out, capi.PERM_C128, k), oracle.sbp_coefficient(C, int(occ[k])), M, u=U_CFIX)


@pytest.mark.parametrize("n,N,kind", [(18, 24, "real"), (20, 26, "complex"), (21, 30, "real")])
def test_warp_items(capi, dev, n, N, kind):
    import torch
    g = inputs.rng(9920 + n)
    if kind == "real":
        C = g.uniform(-1, 1, (n, N))
        code = capi.PERM_F64
    else:
        C = (g.standard_normal((n, N)) + 1j * g.standard_normal((n, N))) / np.sqrt(2 * n)
        code = capi.PERM_C128
    occ = sample_occ(g, n, N, 40)
    out = capi.perm_sbp(torch.from_numpy(C).to(dev), torch.from_numpy(occ.view(np.int64)).to(dev))
    torch.cuda.synchronize(dev)
    for k in range(0, len(occ), 20):
        M = C[:, [j for j in range(N) if (int(occ[k]) >> j) & 1]]
        close(coef(capi, out, code, k), oracle.sbp_coefficient(C, int(occ[k])), M,
              u=U_CFIX if kind == "complex" else 2.0 ** -53)


def test_host_buffers_bad_bitstrings_and_errors(capi, dev):
    g = inputs.rng(9930)
    n, N = 5, 11
    C = g.uniform(-1, 1, (n, N))
    occ = np.array([bits([0, 2, 4, 6, 8]), bits([0, 1, 2]), bits([1, 3, 5, 7, 9, 10]),
                    bits([0, 1, 2, 3, 11]), bits([6, 7, 8, 9, 10])], dtype=np.uint64)
    out = capi.perm_sbp(C, occ)  # numpy in, numpy out
    assert isinstance(out, np.ndarray)
    close(out[0], oracle.sbp_coefficient(C, int(occ[0])), C[:, [0, 2, 4, 6, 8]])
    close(out[4], oracle.sbp_coefficient(C, int(occ[4])), C[:, [6, 7, 8, 9, 10]])
    assert np.isnan(out[1]) and np.isnan(out[2]) and np.isnan(out[3])  # 3, 6 states; a state >= N
    with pytest.raises(capi.PermError) as e:
        capi.perm_sbp(np.ones((33, 40)), occ)
    assert e.value.status == capi.PERM_ETOOBIG
    with pytest.raises(capi.PermError) as e:
        capi.perm_sbp(np.ones((3, 5), dtype=np.uint8), occ)
    assert e.value.status == capi.PERM_EUNSUPPORTED


@pytest.mark.parametrize("arith", [1, 2, 3])
def test_real_arithmetics_and_nonfinite_columns(capi, dev, arith):
    # real input: integer pipes by default (FIXED, MIXED), FP64 sweep with arith = FP64;
    # a non-finite entry spoils exactly the coefficients whose bitstrings occupy its column
    import torch
    g = inputs.rng(9940 + arith)
    for n, N in ((9, 15), (14, 20), (18, 22)):
        C = g.uniform(-1, 1, (n, N))
        C[2, 5] = np.nan
        occ = sample_occ(g, n, N, 64)
        out = capi.perm_sbp(torch.from_numpy(C).to(dev), torch.from_numpy(occ.view(np.int64)).to(dev),
                            opts=dict(arith=arith))
        torch.cuda.synchronize(dev)
        got = out.cpu().numpy()
        for k in range(0, len(occ), 5 if n < 18 else 16):
            cols = [j for j in range(N) if (int(occ[k]) >> j) & 1]
            if 5 in cols:
                assert np.isnan(got[k])
            else:  # (the oracle's product C P would carry NaN * 0 = NaN from column 5)
                clean = np.nan_to_num(C)
                close(got[k], oracle.sbp_coefficient(clean, int(occ[k])), C[:, cols])


def test_bench_workload_full_size_sampled(capi, dev):
    # the bench's SBP workload at its full size (one 12 x 24 real matrix, 1,000,000
    # bitstrings with 12 of 24 states occupied, built as in bench.py), 64 sampled
    # coefficients against the oracle one by one
    import torch
    n, N, count = 12, 24, 1000000
    g = inputs.rng(inputs.SEED_BASE + 7)
    C = g.uniform(-1.0, 1.0, (n, N))
    cols = np.argsort(g.random((count, N)), axis=1)[:, :n]
    occ = np.bitwise_or.reduce(np.left_shift(np.uint64(1), cols.astype(np.uint64)), axis=1)
    out = capi.perm_sbp(torch.from_numpy(C).to(dev), torch.from_numpy(occ.view(np.int64)).to(dev))
    torch.cuda.synchronize(dev)
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    for k in np.linspace(0, count - 1, 64).astype(int):
        M = C[:, [j for j in range(N) if (int(occ[k]) >> j) & 1]]
        close(got[k], oracle.sbp_coefficient(C, int(occ[k])), M)
