// Glynn's formula (Eq. glynn, Eq. glynn_rectangle) for real input on the integer
// pipes ("fixed" arithmetic).
//
// GB300 issues FP64 at 1/74 of its FP32/INT32 rate, so this variant keeps the FP64
// unit out of the sweep:
//   * column j is held in fixed point with its own scale 2^e_j, chosen so that
//     sum_i |a'_ij| 2^e_j <= 2^61; a'_ij is rounded once to q_ij = rint(a'_ij 2^e_j)
//     (relative perturbation <= 2^-62 of the column's absolute sum, far below the
//     rounding of the input to double).  The +-2 q updates of the Gray-code walk are
//     exact int64 additions, so the column sums never drift and need no re-anchoring;
//   * the product over columns is a software float with a 64-bit mantissa: each
//     factor is normalised with clz and multiplied with the high half of a 64x64-bit
//     product (truncation error < 2^-62 per factor, below FP64's 2^-53);
//   * the signed terms are added into a 192-bit fixed-point accumulator per thread.
//     Its window is anchored on the thread's first nonzero term (whose leading bit
//     lands on bit 120, leaving 120 bits below it and 70 above); a later term whose
//     leading bit would pass bit 150 first shifts the window up.  Each thread's total
//     is converted to double-double once and reduced as in the FP64 path.
// The preparation kernel derives the scales and the quantised tables on the device.
#include "device_common.cuh"
#include "internal.h"

namespace perm {
namespace {

typedef unsigned long long u64;

constexpr int kAnchorBit = 120;  // leading bit of a thread's first term
constexpr int kMaxLsb = 87;      // a term's lsb may sit at most here (leading bit <= 150)

// One block, one thread per column: scales, quantised +-2q tables and exponents.
__global__ void fx_prep_kernel(SweepArgs a, FxTable* tab) {
  const int n = a.n, m = a.m;
  const double* A = static_cast<const double*>(a.A);
  __shared__ int xs[64];
  __shared__ int es[64];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < n) {
    double colabs = (double)(n - m);
    for (int i = 0; i < m; ++i) {
      const double v = A[i * a.rs + j * a.cs];
      if (!isfinite(v)) bad = 1;
      colabs += fabs(v);
    }
    int x = 0;
    if (colabs > 0.0) {
      frexp(colabs, &x);  // colabs < 2^x
      // rounding of colabs itself: keep one bit of headroom
    }
    const int e = 61 - x;
    xs[j] = x;
    es[j] = e;
    for (int i = 0; i < n; ++i) {
      long long q = 0;
      if (i < m) q = llrint(ldexp(A[i * a.rs + j * a.cs], e));
      else q = (long long)llrint(ldexp(1.0, e));
      tab->d[i * 64 + j] = 2 * q;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int xsum = 0, esum = 0;
    for (int k = 0; k < n; ++k) {
      xsum += xs[k];
      esum += es[k];
    }
    tab->e_max = xsum;
    tab->e_sum = esum;
    tab->bad = bad;
  }
}

// value = sign * P * 2^(E - 63) * 2^(-e_sum), P in [2^63, 2^64); P == 0 iff some
// factor is zero.  Columns are taken in pairs: the product of two column sums
// (each below 2^62 in magnitude) is formed exactly in 128 bits, its leading 64 bits
// are multiplied into P with the high half of a 64x64-bit product (truncation error
// < 2^-62 per pair), and P is renormalised by at most one bit.  The value is
// P 2^(E-63): multiplying by a pair product mc 2^(64-lz) gives h2 2^(E + 1 - lz + 63),
// hence E += 127 - lz + top after the one-bit renormalisation.
template <int N>
__device__ __forceinline__ void soft_product(const long long (&S)[N], u64& P, int& E, unsigned& neg) {
  static_assert(N % 2 == 0, "columns are padded to an even count");
  P = 1ull << 63;  // the value 1
  E = 0;
  neg = 0;
#pragma unroll
  for (int j = 0; j < N; j += 2) {
    const long long qa = S[j], qb = S[j + 1];
    const u64 sa = (u64)(qa >> 63), sb = (u64)(qb >> 63);
    neg ^= (unsigned)(sa ^ sb);
    // magnitudes by one's complement: |q| or |q| - 1, an error of one unit in a value
    // of up to 2^61 (relative 2^-58 or less for all but vanishing column sums)
    const u64 aa = (u64)qa ^ sa, ab = (u64)qb ^ sb;
    const u64 hi = __umul64hi(aa, ab), lo = aa * ab;
    // hi < 2^60 (both factors are below 2^62), so lz >= 4; a pair product below 2^64
    // (vanishing column sums) keeps the bits of lo that fit, the value stays exact
    const int lz = __clzll((long long)(hi | 1ull));
    const u64 mc = (hi << lz) | (lo >> (64 - lz));  // pair product ~ mc * 2^(64 - lz)
    const u64 h2 = __umul64hi(P, mc);                // P mc = h2 * 2^64 + (dropped)
    const int top = (int)(h2 >> 63);
    P = top ? h2 : (h2 << 1);
    E += 127 - lz + top;
  }
  neg &= 1u;
}

// acc += (-1)^neg * P * 2^p (p = position of P's lsb in the accumulator, p <= 127)
__device__ __forceinline__ void acc_add(u64& a0, u64& a1, u64& a2, u64 P, int p, unsigned neg) {
  u64 t0, t1, t2;
  if (p >= 64) {
    const int q = p - 64;
    t0 = 0;
    t1 = P << q;
    t2 = q ? (P >> (64 - q)) : 0;
  } else if (p >= 0) {
    t0 = P << p;
    t1 = p ? (P >> (64 - p)) : 0;
    t2 = 0;
  } else if (p > -64) {
    t0 = P >> (-p);
    t1 = 0;
    t2 = 0;
  } else {
    t0 = t1 = t2 = 0;
  }
  if (neg) {
    asm("sub.cc.u64 %0, %0, %3;\n\tsubc.cc.u64 %1, %1, %4;\n\tsubc.u64 %2, %2, %5;"
        : "+l"(a0), "+l"(a1), "+l"(a2)
        : "l"(t0), "l"(t1), "l"(t2));
  } else {
    asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
        : "+l"(a0), "+l"(a1), "+l"(a2)
        : "l"(t0), "l"(t1), "l"(t2));
  }
}

// Arithmetic right shift of the signed 192-bit integer a2:a1:a0 by s >= 1 bits.
__device__ __forceinline__ void shr192(u64& a0, u64& a1, u64& a2, int s) {
  const u64 sgn = (u64)((long long)a2 >> 63);
  while (s >= 64) {
    a0 = a1;
    a1 = a2;
    a2 = sgn;
    s -= 64;
  }
  if (s > 0) {
    a0 = (a0 >> s) | (a1 << (64 - s));
    a1 = (a1 >> s) | (a2 << (64 - s));
    a2 = (u64)((long long)a2 >> s);
  }
}

// Signed 192-bit integer times 2^e_lo as a double-double (four exact 48-bit pieces).
__device__ __forceinline__ dd acc_to_dd(u64 a0, u64 a1, u64 a2, int e_lo) {
  const bool negative = (long long)a2 < 0;
  if (negative) {
    asm("sub.cc.u64 %0, 0, %0;\n\tsubc.cc.u64 %1, 0, %1;\n\tsubc.u64 %2, 0, %2;" : "+l"(a0), "+l"(a1), "+l"(a2));
  }
  const u64 mask = (1ull << 48) - 1;
  const double p0 = (double)(a0 & mask);
  const double p1 = (double)(((a0 >> 48) | (a1 << 16)) & mask);
  const double p2 = (double)(((a1 >> 32) | (a2 << 32)) & mask);
  const double p3 = (double)(a2 >> 16);
  dd r = dd{scalbn(p3, e_lo + 144), 0.0};
  r = dd_add(r, dd{scalbn(p2, e_lo + 96), 0.0});
  r = dd_add(r, dd{scalbn(p1, e_lo + 48), 0.0});
  r = dd_add(r, dd{scalbn(p0, e_lo), 0.0});
  if (negative) {
    r.hi = -r.hi;
    r.lo = -r.lo;
  }
  return r;
}

template <int N>
__global__ void __launch_bounds__(192, (N <= 36) ? 2 : 1) glynn_fx_kernel(SweepArgs a, const FxTable* __restrict__ tab) {
  const bool ABS = a.want_abs != 0;
  extern __shared__ long long smem_fx[];
  __shared__ dd scratch[2 * 32];
  const int n = a.n;
  long long* sP = smem_fx;          // +2 q_ij
  long long* sM = smem_fx + n * N;  // -2 q_ij
  for (int idx = threadIdx.x; idx < n * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    const long long v = (j < n) ? tab->d[i * 64 + j] : 0;
    sP[idx] = v;
    sM[idx] = -v;
  }
  const int e_sum = tab->e_sum + 31 * (N - n);  // padded columns are 2^31 = 1 * 2^31
  __syncthreads();

  // Work: chunks of L = 2^chunk_log2 terms aligned to multiples of L; a warp takes 32
  // consecutive chunks at a time, one per lane, so all lanes flip the same row at the
  // same step (the table row is read as a broadcast).  Edge chunks are clipped to
  // [g_begin, g_end).
  const int lane = threadIdx.x & 31;
  const uint64_t L = 1ull << a.chunk_log2;
  const uint64_t c_first = a.g_begin >> a.chunk_log2;
  const uint64_t c_end = (a.g_end + L - 1) >> a.chunk_log2;
  const uint64_t rounds = (c_end - c_first + 31) / 32;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);

  // value of a term with mantissa P, exponent E: P * 2^(E - 63 - e_sum); its lsb sits
  // at accumulator bit p = E - 63 - e_sum - e_lo
  int e_lo = 0;
  bool anchored = false;
  u64 a0 = 0, a1 = 0, a2 = 0;
  u64 b0 = 0, b1 = 0, b2 = 0;  // sum of |term| (ABS only)
  long long S[N];
  for (uint64_t r = warp; r < rounds; r += warps) {
    const uint64_t chunk = c_first + 32 * r + lane;
    uint64_t ga = chunk << a.chunk_log2, gb = ga + L;
    if (ga < a.g_begin) ga = a.g_begin;
    if (gb > a.g_end) gb = a.g_end;
    if (chunk >= c_end) ga = gb = a.g_end;  // idle lane
    for (uint64_t g = ga; g < gb; ++g) {
      if (g == ga) {
        const uint64_t gray = g ^ (g >> 1);
#pragma unroll
        for (int j = 0; j < N; ++j) S[j] = 0;
        for (int i = 0; i < n; ++i) {
          const long long* row = (((gray >> (n - 1 - i)) & 1u) ? sM : sP) + i * N;
#pragma unroll
          for (int j = 0; j < N; ++j) S[j] += row[j];
        }
        // padded columns hold the constant 2^31 (their scale is counted in e_sum below),
        // large enough that a pair of them forms a normalisable 64-bit product
#pragma unroll
        for (int j = 0; j < N; ++j) S[j] = (j < n) ? (S[j] >> 1) : (1ll << 31);
      } else {
        const int b = ctz64(g);
        const long long* row = (((g >> (b + 1)) & 1u) ? sP : sM) + (n - 1 - b) * N;
#pragma unroll
        for (int j = 0; j < N; ++j) S[j] += row[j];
      }
      u64 P;
      int E;
      unsigned neg;
      soft_product(S, P, E, neg);
      if (P != 0) {
        if (!anchored) {
          e_lo = E - e_sum - kAnchorBit;
          anchored = true;
        }
        int p = E - 63 - e_sum - e_lo;
        if (p > kMaxLsb) {  // rare: move the window up
          shr192(a0, a1, a2, p - kMaxLsb);
          if (ABS) shr192(b0, b1, b2, p - kMaxLsb);
          e_lo += p - kMaxLsb;
          p = kMaxLsb;
        }
        acc_add(a0, a1, a2, P, p, neg ^ (unsigned)(g & 1u));
        if (ABS) acc_add(b0, b1, b2, P, p, 0u);
      }
    }
  }

  dd v[2] = {acc_to_dd(a0, a1, a2, e_lo), ABS ? acc_to_dd(b0, b1, b2, e_lo) : dd{0.0, 0.0}};
  block_sum_dd<2>(v, scratch);
  if (threadIdx.x == 0) {
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * kRealRecord;
    const bool bad = tab->bad != 0;  // a non-finite entry: no fixed-point image exists
    rec[0] = bad ? __longlong_as_double(0x7ff8000000000000ll) : v[0].hi;
    rec[1] = bad ? 0.0 : v[0].lo;
    rec[2] = v[1].hi;
    rec[3] = v[1].lo;
  }
}

template <int N>
void* kernel_for(bool) {
  return (void*)glynn_fx_kernel<N>;
}

void* pick(int n, bool abs) {
  switch ((n + 3) & ~3) {
    case 4: return kernel_for<4>(abs);
    case 8: return kernel_for<8>(abs);
    case 12: return kernel_for<12>(abs);
    case 16: return kernel_for<16>(abs);
    case 20: return kernel_for<20>(abs);
    case 24: return kernel_for<24>(abs);
    case 28: return kernel_for<28>(abs);
    case 32: return kernel_for<32>(abs);
    case 36: return kernel_for<36>(abs);
    case 40: return kernel_for<40>(abs);
    case 44: return kernel_for<44>(abs);
    case 48: return kernel_for<48>(abs);
    case 52: return kernel_for<52>(abs);
    case 56: return kernel_for<56>(abs);
    case 60: return kernel_for<60>(abs);
    case 64: return kernel_for<64>(abs);
    default: return nullptr;
  }
}

size_t smem_bytes(int n) { return 2u * (size_t)n * (size_t)((n + 3) & ~3) * sizeof(long long); }

}  // namespace

int glynn_fx_blocks_per_sm(int n, int block, bool want_abs) {
  void* k = pick(n, want_abs);
  if (!k) return 0;
  size_t smem = smem_bytes(n);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_glynn_fx(const SweepArgs& a, FxTable* tab, const LaunchCfg& c, bool want_abs) {
  void* k = pick(a.n, want_abs);
  if (!k) return cudaErrorInvalidValue;
  fx_prep_kernel<<<1, 64, 0, c.stream>>>(a, tab);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  size_t smem = smem_bytes(a.n);
  if (smem > 48 * 1024) {
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
