// Rectangular Glynn (m < n) for real input on the integer pipes, with the padding
// rows of Eq. glynn_filled_matrix summed in closed form.
//
// Eq. glynn_rectangle pads A with n - m rows of ones.  A padding sign vector enters a
// term only through its number t of -1 signs (column sums shifted by x = n - m - 2t),
// so the padding sum over t is the (n-m)-th finite difference (step 2) of the
// polynomial  P(x) = prod_j (c_j + x) = sum_r e_{n-r}(c) x^r,  c_j = sum_{i<m} d_i a_ij.
// With k = n - m, the k-th difference sum_t (-1)^t C(k, t) f(x - 2t) annihilates x^r
// for r < k and maps x^k to 2^k k!; the terms x^r with r > k carry e_{n-r}(c), a
// polynomial of degree n - r < m in the sign vector d, which vanishes in the sum over
// d weighted by prod_i d_i.  What survives, after the normalisation 2^(n-1) k!, is
//     per(A) = 2^-(m-1) sum_{d in {+-1}^m, d_0 = +1} (prod_i d_i) e_m(c(d)),
// the sum over the m-column subsets S of Glynn's formula for the square A_S.  The
// padding rows' 2^(n-m) sign vectors and their cancellation are gone: where the
// padded sum cancels by 10^15 or more (m << n, entries of both signs) this one
// cancels like the square formula on the m x m blocks.
//
// Arithmetic:
//   * c_j in fixed point as in glynn_fx.cu, column j scaled by 2^e_j so that
//     sum_i |a_ij| 2^e_j < 2^60 (real rows only), the Gray-code flips exact int64
//     additions of +-2 q_ij, held per thread in shared memory;
//   * e_0..e_m by the recurrence E_s += c_j E_{s-1} (s descending) over the columns, only
//     for the s that are reachable (s <= j + 1) and can still reach m (s >= m - (n-1-j)):
//     m (n - m + 1) multiply-adds per sign vector instead of m n; the band depends on the
//     loop indices only, so the warp stays converged.  The recurrence runs in
//     a software float with a signed 64-bit mantissa of magnitude [2^62, 2^63] and an
//     int exponent: product = high half of the 128-bit product (truncation < 2^-60),
//     sum = both halves aligned and added (< 2^-61 each), renormalised with clz;
//   * the signed e_m of each sign vector goes into the 192-bit accumulator of
//     fixed_common.cuh.
// With an error bound asked for (ABS), the same recurrence runs on |c_j|
// (G = e_m(|c|), no cancellation) and, if the quantisation of A was inexact, on the
// difference F = e_m(|c| + eta) - e_m(|c|) (eta_j = m/2 quantisation units, each
// entry rounded by at most half a unit): |e_m(c_true) - e_m(c)| <= F.
#include "device_common.cuh"
#include "fixed_common.cuh"
#include "internal.h"

namespace perm {

namespace {

constexpr int kMaxM = 32;             // rows of the DP kernels (1..kMaxM)
constexpr int kZeroExp = -(1 << 28);  // exponent of a software-float zero
constexpr int kEsymBlock = 128;

// software float: value = m * 2^e, |m| in [2^62 - 1, 2^63] or m == 0 (e = kZeroExp)
struct sf {
  long long m;
  int e;
};

__device__ __forceinline__ sf sf_from_int(long long q, int scale_exp) {
  // q * 2^-scale_exp with |q| < 2^62
  if (q == 0) return sf{0, kZeroExp};
  // one's-complement magnitude (|q| - 1 for q < 0) only picks the shift: a negative
  // power of two lands on -2^63, every other value in [2^62, 2^63)
  const u64 mag = (u64)(q ^ (q >> 63));
  const int l = __clzll((long long)(mag | 1ull)) - 1;
  return sf{q << l, -scale_exp - l};
}

__device__ __forceinline__ sf sf_mul(sf a, sf b) {
  const long long h = __mul64hi(a.m, b.m);  // floor(a.m b.m / 2^64), |h| in [2^60 - 1, 2^62]
  if (h == 0 || h == -1) return sf{0, kZeroExp};  // only for a zero factor
  const int l = __clzll((long long)((u64)(h ^ (h >> 63)) | 1ull)) - 1;
  return sf{h << l, a.e + b.e + 64 - l};
}

__device__ __forceinline__ sf sf_add(sf a, sf b) {
  // align on the larger exponent, add the halves (no overflow), renormalise
  if (a.e < b.e) {
    const sf t = a;
    a = b;
    b = t;
  }
  const int d = a.e - b.e;
  const long long bs = d >= 62 ? (b.m >> 63) : (b.m >> (d + 1));
  const long long s = (a.m >> 1) + bs;
  if (s == 0) return sf{0, kZeroExp};
  const int l = __clzll((long long)((u64)(s ^ (s >> 63)) | 1ull)) - 1;
  return sf{s << l, a.e + 1 - l};
}

// One block, one thread per column: scales (real rows only), the +-2q table, flags.
__global__ void esym_prep_kernel(SweepArgs a, EsymTable* tab) {
  const int n = a.n, m = a.m;
  const double* A = static_cast<const double*>(a.A);
  __shared__ int bad, inexact;
  if (threadIdx.x == 0) {
    bad = 0;
    inexact = 0;
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j < n) {
    double colabs = 0.0, scaled = 0.0;  // scaled: the same sum times 2^-64 (no overflow)
    for (int i = 0; i < m; ++i) {
      const double v = A[i * a.rs + j * a.cs];
      if (!isfinite(v)) bad = 1;
      colabs += fabs(v);
      scaled += ldexp(fabs(v), -64);
    }
    int x = 0;
    if (colabs > 0.0 && isfinite(colabs)) {
      frexp(colabs, &x);  // colabs < 2^x
    } else if (scaled > 0.0 && isfinite(scaled)) {
      frexp(scaled, &x);
      x += 64;
    }
    // sum_i |q_ij| <= 2^61 + m / 2: one bit below x for the rounding of colabs itself
    const int e = 60 - x;
    tab->e[j] = e;
    for (int i = 0; i < m; ++i) {
      const double s = ldexp(A[i * a.rs + j * a.cs], e);
      const double r = rint(s);
      if (r != s && isfinite(s)) inexact = 1;
      tab->d[i * 64 + j] = isfinite(s) ? 2 * (long long)r : 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    tab->bad = bad;
    tab->inexact = inexact;
    tab->eta = (m + 1) / 2;
  }
}

// sum over the sign vectors g in [g_begin, g_end) (Gray code, bit b <-> row m-1-b,
// term sign (-1)^g) of sign * e_m(c); records {sum.hi, sum.lo, G.hi, G.lo, F.hi, F.lo}
// (G, F only with ABS), unnormalised (the caller divides by 2^(m-1)).
template <int M, bool ABS>
__global__ void __launch_bounds__(kEsymBlock) glynn_esym_kernel(SweepArgs a, const EsymTable* __restrict__ tab) {
  extern __shared__ long long smem_es[];
  __shared__ dd scratch[3 * (kEsymBlock / 32)];
  const int n = a.n;
  const int nt = blockDim.x;
  long long* sP = smem_es;                  // +2 q_ij, M x n
  long long* sC = smem_es + M * n;          // per-thread column sums: sC[j * nt + tid]
  __shared__ int s_e[64];
  for (int idx = threadIdx.x; idx < M * n; idx += nt) {
    const int i = idx / n, j = idx - i * n;
    sP[idx] = tab->d[i * 64 + j];
  }
  for (int j = threadIdx.x; j < n; j += nt) s_e[j] = tab->e[j];
  const bool use_f = ABS && tab->inexact != 0;
  const long long eta = tab->eta;
  __syncthreads();
  long long* myC = sC + threadIdx.x;

  const int lane = threadIdx.x & 31;
  const uint64_t L = 1ull << a.chunk_log2;
  const uint64_t c_first = a.g_begin >> a.chunk_log2;
  const uint64_t c_end = (a.g_end + L - 1) >> a.chunk_log2;
  const uint64_t rounds = (c_end - c_first + 31) / 32;
  const uint64_t warps = (uint64_t)gridDim.x * (nt >> 5);
  const uint64_t warp = (uint64_t)blockIdx.x * (nt >> 5) + (threadIdx.x >> 5);

  int e_lo = 0;
  bool anchored = false;
  u64 a0 = 0, a1 = 0, a2 = 0;
  u64 b0 = 0, b1 = 0, b2 = 0;  // sum of G (ABS)
  u64 f0 = 0, f1 = 0, f2 = 0;  // sum of F (ABS, inexact quantisation)

  // add the software float v (sign flipped if neg) into the accumulator (x0, x1, x2)
  auto accumulate = [&](u64& x0, u64& x1, u64& x2, sf v, unsigned neg) {
    if (v.m == 0) return;
    const unsigned vneg = (unsigned)((u64)v.m >> 63) ^ neg;
    const u64 P = v.m < 0 ? (u64)0 - (u64)v.m : (u64)v.m;  // in [2^62 - 1, 2^63]
    if (!anchored) {
      e_lo = v.e + 63 - kAnchorBit;
      anchored = true;
    }
    int p = v.e - e_lo;
    if (p > kMaxLsb) {
      shr192(a0, a1, a2, p - kMaxLsb);
      if (ABS) {
        shr192(b0, b1, b2, p - kMaxLsb);
        shr192(f0, f1, f2, p - kMaxLsb);
      }
      e_lo += p - kMaxLsb;
      p = kMaxLsb;
    }
    if (p >= 0) {
      acc_add_nb(x0, x1, x2, P, p, vneg);
    } else {
      acc_add(x0, x1, x2, P, p, vneg);
    }
  };

  for (uint64_t r = warp; r < rounds; r += warps) {
    const uint64_t chunk = c_first + 32 * r + lane;
    uint64_t ga = chunk << a.chunk_log2, gb = ga + L;
    if (ga < a.g_begin) ga = a.g_begin;
    if (gb > a.g_end) gb = a.g_end;
    if (chunk >= c_end) ga = gb = a.g_end;  // idle lane
    for (uint64_t g = ga; g < gb; ++g) {
      if (g == ga) {
        const uint64_t gray = g ^ (g >> 1);
        for (int j = 0; j < n; ++j) {
          long long s = 0;
#pragma unroll 4
          for (int i = 0; i < M; ++i) {
            const long long v = sP[i * n + j];
            s += ((gray >> (M - 1 - i)) & 1u) ? -v : v;
          }
          myC[j * nt] = s >> 1;  // sum of +-2q is even
        }
      } else {
        // delta of row m-1-b flips; it becomes -1 when bit b+1 of g is 0 (see the
        // Gray-code bookkeeping of the square sweeps)
        const int b = ctz64(g);
        const long long* row = sP + (M - 1 - b) * n;
        const bool plus = ((g >> (b + 1)) & 1u) != 0;
        for (int j = 0; j < n; ++j) myC[j * nt] += plus ? row[j] : -row[j];
      }

      sf E[M + 1];
      E[0] = sf{1ll << 62, -62};
#pragma unroll
      for (int s = 1; s <= M; ++s) E[s] = sf{0, kZeroExp};
      for (int j = 0; j < n; ++j) {
        const sf c = sf_from_int(myC[j * nt], s_e[j]);
        const int lo = M - (n - 1 - j), hi = j + 1;  // the band that can still reach e_m
#pragma unroll
        for (int s = M; s >= 1; --s)
          if (s >= lo && s <= hi) E[s] = sf_add(E[s], sf_mul(c, E[s - 1]));
      }
      accumulate(a0, a1, a2, E[M], (unsigned)(g & 1u));
      if (ABS) {
        sf G[M + 1], F[M + 1];
        G[0] = sf{1ll << 62, -62};
        F[0] = sf{0, kZeroExp};
#pragma unroll
        for (int s = 1; s <= M; ++s) G[s] = F[s] = sf{0, kZeroExp};
        for (int j = 0; j < n; ++j) {
          const long long q = myC[j * nt];
          const sf c = sf_from_int(q < 0 ? -q : q, s_e[j]);
          const int lo = M - (n - 1 - j), hi = j + 1;
          if (use_f) {
            const sf ce = sf_from_int((q < 0 ? -q : q) + eta, s_e[j]);
            const sf h = sf_from_int(eta, s_e[j]);
#pragma unroll
            for (int s = M; s >= 1; --s)
              if (s >= lo && s <= hi) F[s] = sf_add(F[s], sf_add(sf_mul(ce, F[s - 1]), sf_mul(h, G[s - 1])));
          }
#pragma unroll
          for (int s = M; s >= 1; --s)
            if (s >= lo && s <= hi) G[s] = sf_add(G[s], sf_mul(c, G[s - 1]));
        }
        accumulate(b0, b1, b2, G[M], 0u);
        if (use_f) accumulate(f0, f1, f2, F[M], 0u);
      }
    }
  }

  dd v[3] = {to_dd(a0, a1, a2, e_lo), ABS ? to_dd(b0, b1, b2, e_lo) : dd{0.0, 0.0},
             ABS ? to_dd(f0, f1, f2, e_lo) : dd{0.0, 0.0}};
  block_sum_dd<3>(v, scratch);
  if (threadIdx.x == 0) {
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * kCplxRecord;
    const bool bad = tab->bad != 0;
    rec[0] = bad ? __longlong_as_double(0x7ff8000000000000ll) : v[0].hi;
    rec[1] = bad ? 0.0 : v[0].lo;
    rec[2] = v[1].hi;
    rec[3] = v[1].lo;
    rec[4] = v[2].hi;
    rec[5] = v[2].lo;
  }
}

// Sum of the block records, divided by 2^(m-1) (exact); err = coef G + F (1 + 2^-50)
// plus the rounding of the result to double.
__global__ void esym_finish_kernel(const double* rec, int nrec, int pow2, double coef, double* out, double* err) {
  __shared__ dd scratch[3 * 8];
  dd v[3] = {dd{0.0, 0.0}, dd{0.0, 0.0}, dd{0.0, 0.0}};
  for (int r = threadIdx.x; r < nrec; r += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = dd_add(v[k], dd{rec[kCplxRecord * r + 2 * k], rec[kCplxRecord * r + 2 * k + 1]});
  }
  block_sum_dd<3>(v, scratch);
  if (threadIdx.x != 0) return;
  const dd s = dd_ldexp(v[0], -pow2);
  const double r = __dadd_rn(s.hi, s.lo);
  out[0] = r;
  if (err) {
    const double G = scalbn(v[1].hi, -pow2), F = scalbn(v[2].hi, -pow2);
    err[0] = coef * G + F * (1.0 + 0x1p-50) + fabs(__dsub_rn(r, s.hi) - s.lo);
  }
}

template <int M, bool ABS>
void* kernel_m() {
  return (void*)glynn_esym_kernel<M, ABS>;
}

template <bool ABS>
void* pick(int m) {
  switch (m) {
#define ESYM_CASE(k) \
  case k: return kernel_m<k, ABS>();
    ESYM_CASE(1) ESYM_CASE(2) ESYM_CASE(3) ESYM_CASE(4) ESYM_CASE(5) ESYM_CASE(6) ESYM_CASE(7) ESYM_CASE(8)
    ESYM_CASE(9) ESYM_CASE(10) ESYM_CASE(11) ESYM_CASE(12) ESYM_CASE(13) ESYM_CASE(14) ESYM_CASE(15)
    ESYM_CASE(16) ESYM_CASE(17) ESYM_CASE(18) ESYM_CASE(19) ESYM_CASE(20) ESYM_CASE(21) ESYM_CASE(22)
    ESYM_CASE(23) ESYM_CASE(24) ESYM_CASE(25) ESYM_CASE(26) ESYM_CASE(27) ESYM_CASE(28) ESYM_CASE(29)
    ESYM_CASE(30) ESYM_CASE(31) ESYM_CASE(32)
#undef ESYM_CASE
    default: return nullptr;
  }
}

void* pick_kernel(int m, bool abs) { return abs ? pick<true>(m) : pick<false>(m); }

size_t smem_bytes(int m, int n, int block) { return ((size_t)m * n + (size_t)n * block) * sizeof(long long); }

}  // namespace

int glynn_esym_max_m() { return kMaxM; }
int glynn_esym_block() { return kEsymBlock; }

int glynn_esym_blocks_per_sm(int m, int n, int block, bool want_abs) {
  void* k = pick_kernel(m, want_abs);
  if (!k || n > 64 || m >= n) return 0;
  const size_t smem = smem_bytes(m, n, block);
  if (smem > 32 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_glynn_esym(const SweepArgs& a, EsymTable* tab, const LaunchCfg& c, bool want_abs) {
  if (a.m < 1 || a.m >= a.n || a.n > 64 || c.block > kEsymBlock || c.block % 32) return cudaErrorInvalidValue;
  void* k = pick_kernel(a.m, want_abs);
  if (!k) return cudaErrorInvalidValue;
  esym_prep_kernel<<<1, 64, 0, c.stream>>>(a, tab);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = smem_bytes(a.m, a.n, c.block);
  if (smem > 32 * 1024) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  SweepArgs args = a;
  const EsymTable* tp = tab;
  void* params[] = {&args, &tp};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), params, smem, c.stream);
}

cudaError_t launch_esym_finish(const double* rec, int nrec, int m, double coef, double* out, double* err,
                               cudaStream_t s) {
  esym_finish_kernel<<<1, 256, 0, s>>>(rec, nrec, m - 1, coef, out, err);
  return cudaGetLastError();
}

size_t glynn_esym_table_bytes() { return sizeof(EsymTable); }

}  // namespace perm
