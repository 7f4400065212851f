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
//   * the product over columns is a software float with a 64-bit mantissa: column
//     sums are multiplied in pairs (exact 128-bit product, normalised with clz) into
//     the running mantissa with the high half of a 64x64-bit product; the running
//     mantissa is renormalised every fourth pair, so it keeps at least 60 bits
//     (truncation error < 2^-59 per pair, against FP64's 2^-53 per multiplication);
//   * "mixed" variants (template K > 0) take the product of the last K columns on
//     the otherwise idle FP64 unit (int64 -> double conversions and K - 1 DMUL,
//     2^-53 each) and fold it into the mantissa once: the FP64 pipe and the integer
//     pipes run side by side;
//   * the signed terms are added into a 192-bit fixed-point accumulator per thread;
//   * the error-bound variant (ABS) takes exact magnitudes of the column sums, adds up
//     sum |term|, and, when some entry was rounded to fixed point, also
//     prod_j (|S_j| + eta) (eta = m/2 units, the most a column sum can be off): the
//     rounding of A moves a term by at most that product minus |term|.
//     Its window is anchored on the thread's first nonzero term (whose leading bit
//     lands on bit 120, leaving 120 bits below it and 70 above); a later term whose
//     leading bit would pass bit 150 first shifts the window up.  Each thread's total
//     is converted to double-double once and reduced as in the FP64 path.
// The preparation kernel derives the scales and the quantised tables on the device.
#include "device_common.cuh"
#include "fixed_common.cuh"
#include "internal.h"

namespace perm {
namespace {

// One block, one thread per column: scales, quantised +-2q tables and exponents.
__global__ void fx_prep_kernel(SweepArgs a, FxTable* tab) {
  const int n = a.n, m = a.m;
  const double* A = static_cast<const double*>(a.A);
  __shared__ int xs[64];
  __shared__ int es[64];
  __shared__ int bad, inexact;
  if (threadIdx.x == 0) {
    bad = 0;
    inexact = 0;
  }
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
      if (i < m) {
        const double sv = ldexp(A[i * a.rs + j * a.cs], e);
        if (isfinite(sv) && rint(sv) != sv) inexact = 1;
        q = llrint(sv);
      } else {
        q = (long long)llrint(ldexp(1.0, e));
      }
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
    tab->inexact = inexact;
  }
}

template <int N, int K, bool ABS>
__global__ void __launch_bounds__((N <= 36) ? 192 : 128, 2) glynn_fx_kernel(SweepArgs a, const FxTable* __restrict__ tab) {
  extern __shared__ __align__(16) long long smem_fx[];
  __shared__ dd scratch[3 * 32];
  const int n = a.n;
  long long* sP = smem_fx;          // +2 q_ij
  long long* sM = smem_fx + n * N;  // -2 q_ij
  // error-bound variant with inexact quantisation: each column sum may be off by eta
  // units (m real rows rounded by half a unit each)
  const bool use_eta = ABS && tab->inexact != 0;
  const long long eta = (a.m + 1) / 2;
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
  u64 c0 = 0, c1 = 0, c2 = 0;  // sum of prod (|S| + eta) (ABS with inexact quantisation)
  // add P 2^(E - 63 - e_sum) (sign neg) into (x0, x1, x2), moving the window up if needed
  auto add_term = [&](u64& x0, u64& x1, u64& x2, u64 P, int E, unsigned neg) {
    if (!anchored) {
      e_lo = E - e_sum - kAnchorBit;
      anchored = true;
    }
    int p = E - 63 - e_sum - e_lo;
    if (p > kMaxLsb) {  // rare: move the window up
      shr192(a0, a1, a2, p - kMaxLsb);
      if (ABS) {
        shr192(b0, b1, b2, p - kMaxLsb);
        shr192(c0, c1, c2, p - kMaxLsb);
      }
      e_lo += p - kMaxLsb;
      p = kMaxLsb;
    }
    if (p >= 0) {
      acc_add_nb(x0, x1, x2, P, p, neg);
    } else {  // a term far below the window (rare): its low bits fall off
      acc_add(x0, x1, x2, P, p, neg);
    }
  };
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
        // rows start on 32-byte boundaries (N is a multiple of 4): 16-byte broadcast loads
        const longlong2* row2 = reinterpret_cast<const longlong2*>(row);
#pragma unroll
        for (int j = 0; j < N / 2; ++j) {
          const longlong2 v = row2[j];
          S[2 * j] += v.x;
          S[2 * j + 1] += v.y;
        }
      }
      u64 P;
      int E;
      unsigned neg;
      soft_product<N, K, ABS>(S, P, E, neg);  // exact magnitudes in the bound variant
      if (P != 0) {
        add_term(a0, a1, a2, P, E, neg ^ (unsigned)(g & 1u));
        if (ABS) add_term(b0, b1, b2, P, E, 0u);
      }
      if (use_eta) {
        u64 Pe;
        int Ee;
        soft_product_eta<N, K>(S, n, eta, Pe, Ee);
        if (Pe != 0) add_term(c0, c1, c2, Pe, Ee, 0u);
      }
    }
  }

  // records {sum, sum |term|, sum prod (|S| + eta)} (the last two with ABS only)
  dd v[3] = {to_dd(a0, a1, a2, e_lo), ABS ? to_dd(b0, b1, b2, e_lo) : dd{0.0, 0.0},
             use_eta ? to_dd(c0, c1, c2, e_lo) : dd{0.0, 0.0}};
  block_sum_dd<3>(v, scratch);
  if (threadIdx.x == 0) {
    const bool bad = tab->bad != 0;  // a non-finite entry: no fixed-point image exists
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * (ABS ? kCplxRecord : kRealRecord);
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

// The same sweep with a lane pair per term: lane 2p + h holds the column sums of
// columns [h N/2, (h + 1) N/2) only, forms their product (the last K2 of them on the
// FP64 unit), and the two half products are multiplied after one exchange between the
// lanes (one more 64x64-bit high product, truncating by < 2^-62).  Half the column
// sums per lane halves the registers, so twice as many warps are resident to hide
// the latency of the product chains.  Both lanes of a pair hold the same term and
// each adds half of it (one exponent less: exact in the 192-bit window).  The loop
// runs the same number of steps on every lane (lanes past their range's end compute
// but do not add), so the exchange always sees the whole warp.  No error-bound
// variant: calls that ask for a bound take glynn_fx_kernel.
template <int N, int K2, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) glynn_fxp_kernel(SweepArgs a, const FxTable* __restrict__ tab) {
  constexpr int H = N / 2;
  static_assert(N % 4 == 0 && (H - K2) % 2 == 0, "halves of whole 16-byte rows, integer columns in pairs");
  extern __shared__ __align__(16) long long smem_fx[];
  __shared__ dd scratch[32];
  const int n = a.n;
  long long* sP = smem_fx;          // +2 q_ij
  long long* sM = smem_fx + n * N;  // -2 q_ij
  for (int idx = threadIdx.x; idx < n * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    const long long v = (j < n) ? tab->d[i * 64 + j] : 0;
    sP[idx] = v;
    sM[idx] = -v;
  }
  const int e_sum = tab->e_sum + 31 * (N - n);
  __syncthreads();

  const int lane = threadIdx.x & 31, half = lane & 1, pair = lane >> 1;
  const int j0 = half * H;  // first column of this lane
  const uint64_t L = 1ull << a.chunk_log2;
  const uint64_t c_first = a.g_begin >> a.chunk_log2;
  const uint64_t c_end = (a.g_end + L - 1) >> a.chunk_log2;
  const uint64_t rounds = (c_end - c_first + 15) / 16;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);

  int e_lo = 0;
  bool anchored = false;
  u64 a0 = 0, a1 = 0, a2 = 0;
  long long S[H];
#pragma unroll
  for (int j = 0; j < H; ++j) S[j] = 0;
  for (uint64_t r = warp; r < rounds; r += warps) {  // uniform over the warp
    const uint64_t chunk = c_first + 16 * r + pair;
    uint64_t ga = chunk << a.chunk_log2, gb = ga + L;
    if (ga < a.g_begin) ga = a.g_begin;
    if (gb > a.g_end) gb = a.g_end;
    if (chunk >= c_end) ga = gb = a.g_end;  // idle pair
    for (uint64_t t = 0; t < L; ++t) {
      const uint64_t g = ga + t;
      const bool active = g < gb;  // the same on both lanes of a pair
      if (active) {
        if (t == 0) {
          const uint64_t gray = g ^ (g >> 1);
#pragma unroll
          for (int j = 0; j < H; ++j) S[j] = 0;
          for (int i = 0; i < n; ++i) {
            const long long* row = (((gray >> (n - 1 - i)) & 1u) ? sM : sP) + i * N + j0;
#pragma unroll
            for (int j = 0; j < H; ++j) S[j] += row[j];
          }
#pragma unroll
          for (int j = 0; j < H; ++j) S[j] = (j0 + j < n) ? (S[j] >> 1) : (1ll << 31);
        } else {
          const int b = ctz64(g);
          const long long* row = (((g >> (b + 1)) & 1u) ? sP : sM) + (n - 1 - b) * N + j0;
          // H is even, so a half row starts on a 16-byte boundary
          const longlong2* row2 = reinterpret_cast<const longlong2*>(row);
#pragma unroll
          for (int j = 0; j < H / 2; ++j) {
            const longlong2 v = row2[j];
            S[2 * j] += v.x;
            S[2 * j + 1] += v.y;
          }
        }
      }
      u64 P;
      int E;
      unsigned neg;
      soft_product<H, K2, false>(S, P, E, neg);
      // the partner's half product; each P is 0 or in [2^63, 2^64), value P 2^(E - 63)
      const u64 Po = __shfl_xor_sync(0xffffffffu, P, 1);
      const int Eo = __shfl_xor_sync(0xffffffffu, (int)(((unsigned)E << 1) | neg), 1);
      const u64 h2 = __umul64hi(P, Po);  // P Po 2^(E + Eo - 126) ~ h2 2^(E + Eo - 62)
      const int top = (int)(h2 >> 63);
      P = top ? h2 : (h2 << 1);
      E = E + (Eo >> 1) + top;
      neg ^= (unsigned)Eo & 1u;
      if (active && P != 0) {
        // half of the term: P 2^(E - 1 - 63 - e_sum)
        const int Eh = E - 1;
        if (!anchored) {
          e_lo = Eh - e_sum - kAnchorBit;
          anchored = true;
        }
        int p = Eh - 63 - e_sum - e_lo;
        if (p > kMaxLsb) {
          shr192(a0, a1, a2, p - kMaxLsb);
          e_lo += p - kMaxLsb;
          p = kMaxLsb;
        }
        if (p >= 0)
          acc_add_nb(a0, a1, a2, P, p, neg ^ (unsigned)(g & 1u));
        else
          acc_add(a0, a1, a2, P, p, neg ^ (unsigned)(g & 1u));
      }
    }
  }
  dd v[1] = {to_dd(a0, a1, a2, e_lo)};
  block_sum_dd<1>(v, scratch);
  if (threadIdx.x == 0) {
    const bool bad = tab->bad != 0;
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * kRealRecord;
    rec[0] = bad ? __longlong_as_double(0x7ff8000000000000ll) : v[0].hi;
    rec[1] = bad ? 0.0 : v[0].lo;
    rec[2] = 0.0;
    rec[3] = 0.0;
  }
}

// Columns multiplied on the FP64 unit by the mixed variant, per padded order: enough
// to move a share of the work off the integer pipes, few enough that the FP64 unit
// (2K - 1 operations per term at 1/74 of the integer rate) is not the bottleneck.
// Measured on GB300 (terms/s, K = 0 -> best K): N = 28: 2.73e10 -> 2.95e10 (K = 4);
// N = 32: 2.54e10 -> 2.82e10 (K = 6); N = 36: 2.31e10 -> 2.60e10 (K = 8).  From N = 40
// one block of 6 warps per SM is resident and the FP64 latency is no longer hidden.
constexpr int mixed_columns(int N) { return N >= 40 ? 0 : N >= 36 ? 8 : N >= 32 ? 6 : N >= 16 ? 4 : 0; }

template <int N>
void* kernel_for(bool mixed, bool abs) {
  constexpr int K = mixed_columns(N);
  if (mixed && K > 0) return abs ? (void*)glynn_fx_kernel<N, K, true> : (void*)glynn_fx_kernel<N, K, false>;
  return abs ? (void*)glynn_fx_kernel<N, 0, true> : (void*)glynn_fx_kernel<N, 0, false>;
}

void* pick(int n, bool mixed, bool abs) {
  switch ((n + 3) & ~3) {
    case 4: return kernel_for<4>(mixed, abs);
    case 8: return kernel_for<8>(mixed, abs);
    case 12: return kernel_for<12>(mixed, abs);
    case 16: return kernel_for<16>(mixed, abs);
    case 20: return kernel_for<20>(mixed, abs);
    case 24: return kernel_for<24>(mixed, abs);
    case 28: return kernel_for<28>(mixed, abs);
    case 32: return kernel_for<32>(mixed, abs);
    case 36: return kernel_for<36>(mixed, abs);
    case 40: return kernel_for<40>(mixed, abs);
    case 44: return kernel_for<44>(mixed, abs);
    case 48: return kernel_for<48>(mixed, abs);
    case 52: return kernel_for<52>(mixed, abs);
    case 56: return kernel_for<56>(mixed, abs);
    case 60: return kernel_for<60>(mixed, abs);
    case 64: return kernel_for<64>(mixed, abs);
    default: return nullptr;
  }
}

size_t smem_bytes(int n) { return 2u * (size_t)n * (size_t)((n + 3) & ~3) * sizeof(long long); }

// Lane-pair kernel, from N = 40 (where the one-lane kernel holds 8 warps per SM):
// 4 FP64 columns per half, 256 threads, two blocks per SM (16 warps, <= 128
// registers; N = 52 would spill and stays on the one-lane kernel).  Measured on
// GB300 against the one-lane kernel (terms/s): n = 40: 1.95e10 -> 2.11e10,
// 44: 1.80e10 -> 1.92e10, 48: 1.77e10 -> 1.78e10, 56: 1.45e10 -> 1.52e10,
// 64: 1.24e10 -> 1.29e10.  Below N = 40 it is slower (n = 28 / 32 / 36: -15%, -11%,
// -13%): the pipes, not latency, bound the one-lane kernel there, and the pair adds
// the exchange and a second accumulation per term.
constexpr int kPairFp64Columns = 4;
constexpr int kPairBlock = 256;
constexpr int kPairMinBlocks = 2;

template <int N>
void* pair_kernel() {
  return (void*)glynn_fxp_kernel<N, kPairFp64Columns, kPairBlock, kPairMinBlocks>;
}

void* pick_pair(int n) {
  switch ((n + 3) & ~3) {
    case 40: return pair_kernel<40>();
    case 44: return pair_kernel<44>();
    case 48: return pair_kernel<48>();
    case 56: return pair_kernel<56>();
    case 60: return pair_kernel<60>();
    case 64: return pair_kernel<64>();
    default: return nullptr;
  }
}

}  // namespace

bool glynn_fx_pair_available(int n) { return pick_pair(n) != nullptr; }
int glynn_fx_pair_block() { return kPairBlock; }
int glynn_fx_pair_mixed_columns(int) { return 2 * kPairFp64Columns; }

// Threads per block: 192 (two blocks, 12 warps per SM, <= 168 registers) up to N = 36;
// 128 above (two blocks, 8 warps, <= 255 registers: the column sums no longer fit 168).
int glynn_fx_block(int n) { return ((n + 3) & ~3) <= 36 ? 192 : 128; }

int glynn_fx_mixed_columns(int n) {
  const int N = (n + 3) & ~3;
  return N >= 40 ? 0 : mixed_columns(N);
}

int glynn_fx_blocks_per_sm(int n, int block, bool mixed, bool pair) {
  void* k = pair ? pick_pair(n) : pick(n, mixed, false);
  if (!k) return 0;
  const size_t smem = smem_bytes(n);
  if (smem > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_fx_prep(const SweepArgs& a, FxTable* tab, cudaStream_t stream) {
  fx_prep_kernel<<<1, 64, 0, stream>>>(a, tab);
  return cudaGetLastError();
}

cudaError_t launch_glynn_fx(const SweepArgs& a, FxTable* tab, const LaunchCfg& c, bool want_abs, bool mixed,
                            bool pair) {
  if (pair && (want_abs || !mixed || c.block != kPairBlock)) return cudaErrorInvalidValue;
  void* k = pair ? pick_pair(a.n) : pick(a.n, mixed, want_abs);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = launch_fx_prep(a, tab, c.stream);
  if (e != cudaSuccess) return e;
  const size_t smem = smem_bytes(a.n);
  if (smem > 32 * 1024) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  SweepArgs args = a;
  const FxTable* tp = tab;
  void* params[] = {&args, &tp};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), params, smem, c.stream);
}

}  // namespace perm
