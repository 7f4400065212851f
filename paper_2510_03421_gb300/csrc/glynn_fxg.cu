// Rectangular Glynn for real input on the integer pipes, with the padding rows of
// ones grouped (same fixed-point arithmetic as glynn_fx.cu: quantised column sums,
// 64-bit-mantissa software-float products, 192-bit accumulation; the preparation
// kernel and its table are shared with the square sweep).
#include "device_common.cuh"
#include "fixed_common.cuh"
#include "internal.h"

namespace perm {
namespace {

// Rectangular Glynn (Eq. glynn_rectangle) with the n - m padding rows of ones grouped:
// a padding sign vector enters a term only through its number t of -1 signs (column
// sums shifted by n - m - 2t, sign (-1)^t), and C(n - m, t) of them share each t.  The
// walk runs over the 2^(m-1) sign vectors of the real rows (Gray code, bit b <-> row
// m-1-b, term sign (-1)^g); at each it takes the n - m + 1 values of t, up for even g
// and down for odd g, so consecutive steps differ by one padding-row update
// (+-2 u_j, u_j the quantised 1 of column j) or one real-row flip.  A term's product is
// multiplied by C(n - m, t) (exact 64-bit mantissa, truncation < 2^-63) before the
// 192-bit accumulation.  2^(m-1) (n - m + 1) products replace 2^(n-1).
template <int N>
__global__ void __launch_bounds__(192, (N <= 36) ? 2 : 1) glynn_fxg_kernel(SweepArgs a, const FxTable* __restrict__ tab) {
  const bool ABS = a.want_abs != 0;
  // with an error bound and inexact quantisation: a column sum's rounding is at most
  // m/2 units (the padding rows are exact)
  const bool use_eta = ABS && tab->inexact != 0;
  const long long eta = (a.m + 1) / 2;
  extern __shared__ __align__(16) long long smem_fx[];
  __shared__ dd scratch[3 * 32];
  __shared__ u64 s_wm[64];  // C(n - m, t) = s_wm[t] 2^(s_we[t] - 64), s_wm normalised
  __shared__ int s_we[64];
  const int n = a.n, m = a.m, k = n - m;
  const int R = m + 1;  // the real rows and one padding row (row m of the table)
  long long* sP = smem_fx;          // +2 q_ij
  long long* sM = smem_fx + R * N;  // -2 q_ij
  for (int idx = threadIdx.x; idx < R * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    const long long v = (j < n) ? tab->d[i * 64 + j] : 0;
    sP[idx] = v;
    sM[idx] = -v;
  }
  for (int t = threadIdx.x; t <= k; t += blockDim.x) {
    const u64 c = binom_u64(k, t);
    const int lz = __clzll((long long)c);
    s_wm[t] = c << lz;
    s_we[t] = 64 - lz;
  }
  const int e_sum = tab->e_sum + 31 * (N - n);
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const uint64_t L = 1ull << a.chunk_log2;
  const uint64_t c_first = a.g_begin >> a.chunk_log2;
  const uint64_t c_end = (a.g_end + L - 1) >> a.chunk_log2;
  const uint64_t rounds = (c_end - c_first + 31) / 32;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long* padP = sP + m * N;  // +2 u_j: the padding sum rises by 2 (t down)
  const long long* padM = sM + m * N;  // -2 u_j: t up

  int e_lo = 0;
  bool anchored = false;
  u64 a0 = 0, a1 = 0, a2 = 0;
  u64 b0 = 0, b1 = 0, b2 = 0;
  u64 c0 = 0, c1 = 0, c2 = 0;
  auto add_term = [&](u64& x0, u64& x1, u64& x2, u64 P, int E, unsigned neg) {
    if (!anchored) {
      e_lo = E - e_sum - kAnchorBit;
      anchored = true;
    }
    int p = E - 63 - e_sum - e_lo;
    if (p > kMaxLsb) {
      shr192(a0, a1, a2, p - kMaxLsb);
      if (ABS) {
        shr192(b0, b1, b2, p - kMaxLsb);
        shr192(c0, c1, c2, p - kMaxLsb);
      }
      e_lo += p - kMaxLsb;
      p = kMaxLsb;
    }
    if (p >= 0) {
      acc_add_nb(x0, x1, x2, P, p, neg);  // no divergence on the sign or the position
    } else {
      acc_add(x0, x1, x2, P, p, neg);
    }
  };
  auto weigh = [&](u64& P, int& E, int t) {
    const u64 h2 = __umul64hi(P, s_wm[t]);
    const int top = (int)(h2 >> 63);
    P = top ? h2 : (h2 << 1);
    E += s_we[t] - 1 + top;
  };
  long long S[N];
  for (uint64_t r = warp; r < rounds; r += warps) {
    const uint64_t chunk = c_first + 32 * r + lane;
    uint64_t ga = chunk << a.chunk_log2, gb = ga + L;
    if (ga < a.g_begin) ga = a.g_begin;
    if (gb > a.g_end) gb = a.g_end;
    if (chunk >= c_end) ga = gb = a.g_end;
    for (uint64_t g = ga; g < gb; ++g) {
      const bool up = (g & 1u) == 0;
      if (g == ga) {
        const uint64_t gray = g ^ (g >> 1);
#pragma unroll
        for (int j = 0; j < N; ++j) S[j] = 0;
        for (int i = 0; i < m; ++i) {
          const long long* row = (((gray >> (m - 1 - i)) & 1u) ? sM : sP) + i * N;
#pragma unroll
          for (int j = 0; j < N; ++j) S[j] += row[j];
        }
        // padding sum n - m - 2t at t = 0 (going up) or t = n - m (going down)
        const long long* pad = up ? padP : padM;
#pragma unroll
        for (int j = 0; j < N; ++j) S[j] += (long long)k * pad[j];
#pragma unroll
        for (int j = 0; j < N; ++j) S[j] = (j < n) ? (S[j] >> 1) : (1ll << 31);
      } else {
        const int b = ctz64(g);
        const long long* row = (((g >> (b + 1)) & 1u) ? sP : sM) + (m - 1 - b) * N;
#pragma unroll
        for (int j = 0; j < N; ++j) S[j] += row[j];
      }
      for (int s = 0; s <= k; ++s) {
        if (s > 0) {
          const long long* pad = up ? padM : padP;
#pragma unroll
          for (int j = 0; j < N; ++j) S[j] += pad[j];
        }
        const int t = up ? s : k - s;
        u64 P;
        int E;
        unsigned neg;
        if (ABS) {
          soft_product<N, 0, true>(S, P, E, neg);  // exact magnitudes in the bound variant
        } else {
          soft_product<N, 0>(S, P, E, neg);
        }
        if (P != 0) {
          weigh(P, E, t);
          add_term(a0, a1, a2, P, E, neg ^ (unsigned)(g & 1u) ^ (unsigned)(t & 1));
          if (ABS) add_term(b0, b1, b2, P, E, 0u);
        }
        if (use_eta) {
          u64 Pe;
          int Ee;
          soft_product_eta<N, 0>(S, n, eta, Pe, Ee);
          if (Pe != 0) {
            weigh(Pe, Ee, t);
            add_term(c0, c1, c2, Pe, Ee, 0u);
          }
        }
      }
    }
  }

  dd v[3] = {to_dd(a0, a1, a2, e_lo), ABS ? to_dd(b0, b1, b2, e_lo) : dd{0.0, 0.0},
             use_eta ? to_dd(c0, c1, c2, e_lo) : dd{0.0, 0.0}};
  block_sum_dd<3>(v, scratch);
  if (threadIdx.x == 0) {
    // records {sum, sum |term|, eta-widened sum}: kCplxRecord doubles with a bound
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * (ABS ? kCplxRecord : kRealRecord);
    const bool bad = tab->bad != 0;
    rec[0] = bad ? __longlong_as_double(0x7ff8000000000000ll) : v[0].hi;
    rec[1] = bad ? 0.0 : v[0].lo;
    rec[2] = v[1].hi;
    rec[3] = v[1].lo;
    if (ABS) {
      rec[4] = v[2].hi;
      rec[5] = v[2].lo;
    }
  }
}

template <int N>
void* kernel_for() {
  return (void*)glynn_fxg_kernel<N>;
}

void* pick(int n) {
  switch ((n + 3) & ~3) {
    case 4: return kernel_for<4>();
    case 8: return kernel_for<8>();
    case 12: return kernel_for<12>();
    case 16: return kernel_for<16>();
    case 20: return kernel_for<20>();
    case 24: return kernel_for<24>();
    case 28: return kernel_for<28>();
    case 32: return kernel_for<32>();
    case 36: return kernel_for<36>();
    case 40: return kernel_for<40>();
    case 44: return kernel_for<44>();
    case 48: return kernel_for<48>();
    case 52: return kernel_for<52>();
    case 56: return kernel_for<56>();
    case 60: return kernel_for<60>();
    case 64: return kernel_for<64>();
    default: return nullptr;
  }
}

// the m real rows and one padding row of the +-2q tables
size_t smem_bytes(int m, int n) { return 2u * (size_t)(m + 1) * (size_t)((n + 3) & ~3) * sizeof(long long); }

}  // namespace

int glynn_fxg_blocks_per_sm(int m, int n, int block) {
  void* k = pick(n);
  if (!k) return 0;
  const size_t smem = smem_bytes(m, n);
  if (smem > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_glynn_fxg(const SweepArgs& a, FxTable* tab, const LaunchCfg& c, bool want_abs) {
  if (a.m >= a.n || a.m < 1) return cudaErrorInvalidValue;
  void* k = pick(a.n);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = launch_fx_prep(a, tab, c.stream);
  if (e != cudaSuccess) return e;
  const size_t smem = smem_bytes(a.m, a.n);
  if (smem > 32 * 1024) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  SweepArgs args = a;
  args.want_abs = want_abs ? 1 : 0;
  const FxTable* tp = tab;
  void* params[] = {&args, &tp};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), params, smem, c.stream);
}

}  // namespace perm
