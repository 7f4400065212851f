// Coefficients of a symmetric product of bosons (Eq. SBP): for each occupation
// bitstring m with n occupied states, c_m = per(C P) (Eq. SBGpermanent), where P
// selects the occupied columns of the n x N coefficient matrix C in increasing
// order.  C P is never formed: C is staged once per block in shared memory and each
// walk reads its selected columns through a per-item column list.
//   * n <= 16: one bitstring per lane, the lane walks all 2^(n-1) Glynn terms;
//   * n > 16: one bitstring per warp, the lanes take contiguous slices of the terms
//     and their double-double partials are reduced by shuffles.
// Real input, by default: the integer-pipe arithmetic of glynn_fx.cu.  Column j of C
// gets its own fixed-point scale 2^e_j (sum_i |c_ij| 2^e_j <= 2^61) once per call, so a
// bitstring's scale is the sum of its columns' e_j; column sums are exact int64, the
// product a 64-bit-mantissa software float (a few columns on the FP64 unit), the terms
// summed in 192-bit fixed point.  Complex input (and real input with PERM_ARITH_FP64):
// FP64 arithmetic with Kahan-compensated sums, column sums rebuilt exactly at each
// slice start and every 2^chunk_log2 terms (the arithmetic of the batched FP64 class
// kernels).  A bitstring without exactly n occupied states below bit N gets NaN.
#include "device_common.cuh"
#include "fixed_common.cuh"
#include "internal.h"

namespace perm {
namespace {

__device__ __forceinline__ void kahan(double& acc, double& comp, double x) {
  const double y = __dsub_rn(x, comp);
  const double s = __dadd_rn(acc, y);
  comp = __dsub_rn(__dsub_rn(s, acc), y);
  acc = s;
}

// Unnormalised Glynn sum of terms [g, g + len) of the n x n matrix sC[:, col[0..n)].
// sC: n rows of N elements (W doubles each).
template <int NP, int W>
__device__ __forceinline__ void sbp_slice(const double* __restrict__ sC, int N, int n, const int (&col)[NP],
                                          uint64_t g, uint64_t len, int chunk_log2, dd& out_re, dd& out_im) {
  double Sr[NP], Si[NP];
  double accr = 0.0, cr = 0.0, acci = 0.0, ci = 0.0;
  const uint64_t mask = (1ull << chunk_log2) - 1;
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0 || (g & mask) == 0) {
      const uint64_t gray = g ^ (g >> 1);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        Sr[j] = (j < n) ? 0.0 : 1.0;
        Si[j] = 0.0;
      }
      for (int i = 0; i < n; ++i) {
        const double sg = ((gray >> (n - 1 - i)) & 1u) ? -1.0 : 1.0;
        const double* row = sC + (size_t)W * i * N;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          if (j < n) {
            Sr[j] = __fma_rn(sg, row[W * col[j]], Sr[j]);
            if (W == 2) Si[j] = __fma_rn(sg, row[W * col[j] + 1], Si[j]);
          }
        }
      }
    } else {
      const int b = ctz64(g);
      const double sg = ((g >> (b + 1)) & 1u) ? 2.0 : -2.0;
      const double* row = sC + (size_t)W * (n - 1 - b) * N;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        if (j < n) {
          Sr[j] = __fma_rn(sg, row[W * col[j]], Sr[j]);
          if (W == 2) Si[j] = __fma_rn(sg, row[W * col[j] + 1], Si[j]);
        }
      }
    }
    double pr = Sr[0], pi = Si[0];
#pragma unroll
    for (int j = 1; j < NP; ++j) {
      if (W == 2) {
        const double nr = __fma_rn(pr, Sr[j], -__dmul_rn(pi, Si[j]));
        const double ni = __fma_rn(pr, Si[j], __dmul_rn(pi, Sr[j]));
        pr = nr;
        pi = ni;
      } else {
        pr = __dmul_rn(pr, Sr[j]);
      }
    }
    if (g & 1u) {
      pr = -pr;
      pi = -pi;
    }
    kahan(accr, cr, pr);
    if (W == 2) kahan(acci, ci, pi);
  }
  out_re = two_sum(accr, -cr);
  out_im = two_sum(acci, -ci);
}

// Column list of bitstring m; false unless exactly n bits are set, all below bit N.
// Every entry of col is a valid column index (0 for a rejected bitstring).
template <int NP>
__device__ __forceinline__ bool columns_of(uint64_t m, int n, int N, int (&col)[NP]) {
#pragma unroll
  for (int j = 0; j < NP; ++j) col[j] = 0;
  const uint64_t below = (N >= 64) ? ~0ull : ((1ull << N) - 1);
  if ((m & ~below) != 0 || __popcll(m) != n) return false;
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    if (j < n) {
      col[j] = __ffsll((long long)m) - 1;
      m &= m - 1;
    }
  }
  return true;
}

template <int W>
__device__ __forceinline__ void write_coef(double* out, int64_t k, dd vr, dd vi, int n, bool ok) {
  if (!ok) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    out[W * k] = nan;
    if (W == 2) out[W * k + 1] = nan;
    return;
  }
  vr = dd_ldexp(vr, -(n - 1));
  out[W * k] = __dadd_rn(vr.hi, vr.lo);
  if (W == 2) {
    vi = dd_ldexp(vi, -(n - 1));
    out[W * k + 1] = __dadd_rn(vi.hi, vi.lo);
  }
}

struct SbpArgs {
  const double* C;  // n x N, leading dimension ld (elements; complex: (re, im) pairs)
  int64_t ld;
  int n, N;
  const uint64_t* occ;
  int64_t count;
  double* out;
  int chunk_log2;
};

template <int NP, int W, bool LANE>
__global__ void __launch_bounds__(128) sbp_kernel(SbpArgs a) {
  extern __shared__ double sC[];  // n x N elements
  const int n = a.n, N = a.N;
  for (int idx = threadIdx.x; idx < n * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    sC[W * idx] = a.C[W * (i * a.ld + j)];
    if (W == 2) sC[W * idx + 1] = a.C[W * (i * a.ld + j) + 1];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint64_t terms = 1ull << (n - 1);
  if (LANE) {
    for (int64_t base = 32 * warp; base < a.count; base += 32 * warps) {
      const int64_t k = base + lane;
      if (k >= a.count) continue;
      int col[NP];
      const bool ok = columns_of<NP>(a.occ[k], n, N, col);
      dd vr{0.0, 0.0}, vi{0.0, 0.0};
      if (ok) sbp_slice<NP, W>(sC, N, n, col, 0, terms, a.chunk_log2, vr, vi);
      write_coef<W>(a.out, k, vr, vi, n, ok);
    }
  } else {
    for (int64_t k = warp; k < a.count; k += warps) {
      int col[NP];
      const bool ok = columns_of<NP>(a.occ[k], n, N, col);
      dd vr{0.0, 0.0}, vi{0.0, 0.0};
      if (ok) {
        uint64_t g, len;
        split_range(0, terms, 32, (uint64_t)lane, &g, &len);
        sbp_slice<NP, W>(sC, N, n, col, g, len, a.chunk_log2, vr, vi);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        vr = dd_add(vr, shfl_down_dd(vr, o));
        vi = dd_add(vi, shfl_down_dd(vi, o));
      }
      if (lane == 0) write_coef<W>(a.out, k, vr, vi, n, ok);
    }
  }
}

// ---------------------------------------------------------------- integer pipes (real)
// Scales and the quantised +2q table of C (n rows of N int64), one thread per column;
// a column with a non-finite entry gets the exponent kFxBad (its bitstrings give NaN).
__global__ void sbp_fx_prep_kernel(SbpArgs a, long long* table, int* e) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.N) return;
  double colabs = 0.0;
  int nonfinite = 0;
  for (int i = 0; i < a.n; ++i) {
    const double v = a.C[i * a.ld + j];
    if (!isfinite(v)) nonfinite = 1;
    colabs += fabs(v);
  }
  int x = 0;
  if (colabs > 0.0) frexp(colabs, &x);
  const int ej = 61 - x;
  for (int i = 0; i < a.n; ++i) table[i * a.N + j] = nonfinite ? 0 : 2 * llrint(ldexp(a.C[i * a.ld + j], ej));
  e[j] = nonfinite ? kFxBad : ej;
}

// Unnormalised Glynn terms [g, g + len) of sC[:, col[0..n)] into a 192-bit accumulator
// (columns j >= n are the constant 2^31, counted in es).
template <int NP, int K>
__device__ __forceinline__ void sbp_fx_slice(const long long* __restrict__ sq, int N, int n, const int (&col)[NP],
                                             int es, uint64_t g, uint64_t len, u64 (&acc)[3], int& e_lo) {
  long long S[NP];
  bool anchored = false;
  e_lo = 0;
  acc[0] = acc[1] = acc[2] = 0;
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0) {
      const uint64_t gray = g ^ (g >> 1);
#pragma unroll
      for (int j = 0; j < NP; ++j) S[j] = 0;
      for (int i = 0; i < n; ++i) {
        const bool minus = (gray >> (n - 1 - i)) & 1u;
        const long long* row = sq + i * N;
#pragma unroll
        for (int j = 0; j < NP; ++j)
          if (j < n) S[j] += minus ? -row[col[j]] : row[col[j]];
      }
#pragma unroll
      for (int j = 0; j < NP; ++j) S[j] = (j < n) ? (S[j] >> 1) : (1ll << 31);
    } else {
      const int b = ctz64(g);
      const bool plus = (g >> (b + 1)) & 1u;
      const long long* row = sq + (n - 1 - b) * N;
#pragma unroll
      for (int j = 0; j < NP; ++j)
        if (j < n) S[j] += plus ? row[col[j]] : -row[col[j]];
    }
    u64 P;
    int E;
    unsigned neg;
    soft_product<NP, K>(S, P, E, neg);
    if (P != 0) {
      if (!anchored) {
        e_lo = E - es - kAnchorBit;
        anchored = true;
      }
      int p = E - 63 - es - e_lo;
      if (p > kMaxLsb) {
        shr192(acc[0], acc[1], acc[2], p - kMaxLsb);
        e_lo += p - kMaxLsb;
        p = kMaxLsb;
      }
      acc_add(acc[0], acc[1], acc[2], P, p, neg ^ (unsigned)(g & 1u));
    }
  }
}

template <int NP, int K, bool LANE>
__global__ void __launch_bounds__(128) sbp_fx_kernel(SbpArgs a, const long long* __restrict__ table,
                                                     const int* __restrict__ escale) {
  extern __shared__ long long sq[];  // n x N quantised +2q
  __shared__ int se[64];
  const int n = a.n, N = a.N;
  for (int idx = threadIdx.x; idx < n * N; idx += blockDim.x) sq[idx] = table[idx];
  for (int j = threadIdx.x; j < N; j += blockDim.x) se[j] = escale[j];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint64_t terms = 1ull << (n - 1);
  for (int64_t base = LANE ? 32 * warp : warp; base < a.count; base += LANE ? 32 * warps : warps) {
    const int64_t k = LANE ? base + lane : base;
    if (k >= a.count) continue;
    int col[NP];
    bool ok = columns_of<NP>(a.occ[k], n, N, col);
    int es = 31 * (NP - n);
    if (ok) {
#pragma unroll
      for (int j = 0; j < NP; ++j)
        if (j < n) {
          if (se[col[j]] == kFxBad) ok = false;
          es += se[col[j]];
        }
    }
    uint64_t g = 0, len = terms;
    if (!LANE) split_range(0, terms, 32, (uint64_t)lane, &g, &len);
    dd v{0.0, 0.0};
    if (ok) {
      u64 acc[3];
      int e_lo = 0;
      sbp_fx_slice<NP, K>(sq, N, n, col, es, g, len, acc, e_lo);
      v = to_dd(acc[0], acc[1], acc[2], e_lo);
    }
    if (!LANE) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = dd_add(v, shfl_down_dd(v, o));
      if (lane != 0) continue;
    }
    write_coef<1>(a.out, k, v, dd{0.0, 0.0}, n, ok);
  }
}

// FP64 columns per product, by padded order (as the square real sweep)
constexpr int sbp_fp64_columns(int np) { return np >= 32 ? 6 : np >= 16 ? 4 : 0; }

void* pick_fx(int n) {
  switch ((n + 3) & ~3) {
    case 4: return (void*)sbp_fx_kernel<4, 0, true>;
    case 8: return (void*)sbp_fx_kernel<8, 0, true>;
    case 12: return (void*)sbp_fx_kernel<12, 0, true>;
    case 16: return (void*)sbp_fx_kernel<16, sbp_fp64_columns(16), true>;
    case 20: return (void*)sbp_fx_kernel<20, sbp_fp64_columns(20), false>;
    case 24: return (void*)sbp_fx_kernel<24, sbp_fp64_columns(24), false>;
    case 28: return (void*)sbp_fx_kernel<28, sbp_fp64_columns(28), false>;
    case 32: return (void*)sbp_fx_kernel<32, sbp_fp64_columns(32), false>;
    default: return nullptr;
  }
}

template <int W>
void* pick_w(int n) {
  switch ((n + 3) & ~3) {
    case 4: return (void*)sbp_kernel<4, W, true>;
    case 8: return (void*)sbp_kernel<8, W, true>;
    case 12: return (void*)sbp_kernel<12, W, true>;
    case 16: return (void*)sbp_kernel<16, W, true>;
    case 20: return (void*)sbp_kernel<20, W, false>;
    case 24: return (void*)sbp_kernel<24, W, false>;
    case 28: return (void*)sbp_kernel<28, W, false>;
    case 32: return (void*)sbp_kernel<32, W, false>;
    default: return nullptr;
  }
}

}  // namespace

int sbp_run(perm_handle_s* h, const double* dC, int64_t ld, int n, int N, int dtype, const uint64_t* docc,
            int64_t count, double* dout, cudaStream_t stream, int chunk_log2, int sms, bool fp64, void* scratch) {
  (void)h;
  const int W = dtype == 1 ? 2 : 1;
  const bool integer = W == 1 && !fp64;
  void* k = integer ? pick_fx(n) : (W == 2 ? pick_w<2>(n) : pick_w<1>(n));
  if (!k) return 1;
  const size_t smem = integer ? (size_t)n * N * sizeof(long long) : (size_t)W * n * N * sizeof(double);
  if (smem > 32 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                              cudaSuccess)
    return 2;
  int bps = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, 128, smem) != cudaSuccess || bps < 1) bps = 1;
  const bool lane = n <= 16;
  const int64_t items = lane ? (count + 31) / 32 : count;
  int64_t grid = (items + 3) / 4;  // 4 warps per block
  if (grid > (int64_t)sms * bps) grid = (int64_t)sms * bps;
  if (grid < 1) grid = 1;
  SbpArgs a;
  a.C = dC;
  a.ld = ld;
  a.n = n;
  a.N = N;
  a.occ = docc;
  a.count = count;
  a.out = dout;
  a.chunk_log2 = chunk_log2;
  if (integer) {
    // scratch: the n x N table and the N column exponents
    long long* table = static_cast<long long*>(scratch);
    int* e = reinterpret_cast<int*>(table + 64 * 64);
    sbp_fx_prep_kernel<<<1, 64, 0, stream>>>(a, table, e);
    if (cudaGetLastError() != cudaSuccess) return 2;
    const long long* tp = table;
    const int* ep = e;
    void* params[] = {&a, &tp, &ep};
    return cudaLaunchKernel(k, dim3((unsigned)grid), dim3(128), params, smem, stream) == cudaSuccess ? 0 : 2;
  }
  void* params[] = {&a};
  return cudaLaunchKernel(k, dim3((unsigned)grid), dim3(128), params, smem, stream) == cudaSuccess ? 0 : 2;
}

}  // namespace perm
