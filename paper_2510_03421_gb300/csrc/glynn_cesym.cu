// Rectangular Glynn (m < n) for complex input on the integer pipes, with the padding
// rows of Eq. glynn_filled_matrix summed in closed form (the derivation is in
// glynn_esym.cu):
//     per(A) = 2^-(m-1) sum_{d in {+-1}^m, d_0 = +1} (prod_i d_i) e_m(c(d)),
// e_m the m-th elementary symmetric polynomial of the column sums c_j = sum_i d_i a_ij.
// The padded walk cancels 10^6 .. 10^14-fold on complex Gaussian rectangles; this sum
// cancels like Glynn's formula on the square m x m blocks.
//
// Arithmetic: column sums in fixed point (column j scaled by 2^e_j so that
// sum_i (|re a_ij| + |im a_ij|) 2^e_j < 2^60), updated by exact int64 additions; the
// recurrence E_s += c_j E_{s-1} in a complex software float whose two signed 64-bit
// components share one exponent (the larger magnitude in [2^61, 2^62), as in
// glynn_cfx.cu): a product takes the high halves of four 64x64-bit products, a sum
// aligns the smaller operand; each operation errs by a few units in 2^-60 of the
// larger component.  The signed e_m of each sign vector goes into two 192-bit
// accumulators (real, imaginary).  No error bound is stated (as for the complex
// integer-pipe square sweep); calls that ask for one take the FP64 sweep.
#include "device_common.cuh"
#include "fixed_common.cuh"
#include "internal.h"

namespace perm {

namespace {

constexpr int kMaxM = 32;
constexpr int kZeroExp = -(1 << 28);
constexpr int kBlock = 128;

// value = (re + i im) 2^e, max(|re|, |im|) in [2^61, 2^62), or zero (e = kZeroExp)
struct csf {
  long long re, im;
  int e;
};

__device__ __forceinline__ csf csf_from_int(long long qr, long long qi, int scale_exp) {
  if ((qr | qi) == 0) return csf{0, 0, kZeroExp};
  const int l = norm_shift(qr, qi);
  return csf{qr << l, qi << l, -scale_exp - l};
}

__device__ __forceinline__ csf csf_mul(const csf& a, const csf& b) {
  const long long re = __mul64hi(a.re, b.re) - __mul64hi(a.im, b.im);
  const long long im = __mul64hi(a.re, b.im) + __mul64hi(a.im, b.re);
  if ((re | im) == 0 || (a.e == kZeroExp) || (b.e == kZeroExp)) return csf{0, 0, kZeroExp};
  const int l = norm_shift(re, im);
  return csf{re << l, im << l, a.e + b.e + 64 - l};
}

__device__ __forceinline__ csf csf_add(csf a, csf b) {
  if (a.e < b.e) {
    const csf t = a;
    a = b;
    b = t;
  }
  const int d = a.e - b.e;
  const long long br = d >= 62 ? (b.re >> 63) : (b.re >> (d + 1));
  const long long bi = d >= 62 ? (b.im >> 63) : (b.im >> (d + 1));
  const long long sr = (a.re >> 1) + br, si = (a.im >> 1) + bi;
  if ((sr | si) == 0) return csf{0, 0, kZeroExp};
  const int l = norm_shift(sr, si);
  return csf{sr << l, si << l, a.e + 1 - l};
}

// One block, one thread per column: scales, the +-2q table (re, im interleaved), flags.
__global__ void cesym_prep_kernel(SweepArgs a, CesymTable* tab) {
  const int n = a.n, m = a.m;
  const double* A = static_cast<const double*>(a.A);  // (re, im) pairs
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < n) {
    double colabs = 0.0, scaled = 0.0;
    for (int i = 0; i < m; ++i) {
      const int64_t e = 2 * (i * a.rs + j * a.cs);
      const double re = A[e], im = A[e + 1];
      if (!isfinite(re) || !isfinite(im)) bad = 1;
      colabs += fabs(re) + fabs(im);
      scaled += ldexp(fabs(re), -64) + ldexp(fabs(im), -64);
    }
    int x = 0;
    if (colabs > 0.0 && isfinite(colabs)) {
      frexp(colabs, &x);
    } else if (scaled > 0.0 && isfinite(scaled)) {
      frexp(scaled, &x);
      x += 64;
    }
    const int e = 60 - x;
    tab->e[j] = e;
    for (int i = 0; i < m; ++i) {
      const int64_t k = 2 * (i * a.rs + j * a.cs);
      const double sr = ldexp(A[k], e), si = ldexp(A[k + 1], e);
      tab->d[2 * (i * 64 + j)] = isfinite(sr) ? 2 * (long long)rint(sr) : 0;
      tab->d[2 * (i * 64 + j) + 1] = isfinite(si) ? 2 * (long long)rint(si) : 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) tab->bad = bad;
}

// Records {re.hi, re.lo, im.hi, im.lo, 0, 0} per block, unnormalised.
template <int M>
__global__ void __launch_bounds__(kBlock) glynn_cesym_kernel(SweepArgs a, const CesymTable* __restrict__ tab) {
  extern __shared__ long long smem_ce[];
  __shared__ dd scratch[3 * (kBlock / 32)];
  __shared__ int s_e[64];
  const int n = a.n;
  const int nt = blockDim.x;
  long long* sP = smem_ce;                // (re, im) of +2 q_ij, M x n pairs
  long long* sC = smem_ce + 2 * M * n;    // per-thread column sums: re at [2 j nt + tid], im at + nt
  for (int idx = threadIdx.x; idx < M * n; idx += nt) {
    const int i = idx / n, j = idx - i * n;
    sP[2 * idx] = tab->d[2 * (i * 64 + j)];
    sP[2 * idx + 1] = tab->d[2 * (i * 64 + j) + 1];
  }
  for (int j = threadIdx.x; j < n; j += nt) s_e[j] = tab->e[j];
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
  u64 r0 = 0, r1 = 0, r2 = 0, i0 = 0, i1 = 0, i2 = 0;
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
          long long sr = 0, si = 0;
          for (int i = 0; i < M; ++i) {
            const bool minus = ((gray >> (M - 1 - i)) & 1u) != 0;
            const long long vr = sP[2 * (i * n + j)], vi = sP[2 * (i * n + j) + 1];
            sr += minus ? -vr : vr;
            si += minus ? -vi : vi;
          }
          myC[2 * j * nt] = sr >> 1;
          myC[2 * j * nt + nt] = si >> 1;
        }
      } else {
        const int b = ctz64(g);
        const long long* row = sP + 2 * (M - 1 - b) * n;
        const bool plus = ((g >> (b + 1)) & 1u) != 0;
        for (int j = 0; j < n; ++j) {
          myC[2 * j * nt] += plus ? row[2 * j] : -row[2 * j];
          myC[2 * j * nt + nt] += plus ? row[2 * j + 1] : -row[2 * j + 1];
        }
      }
      csf E[M + 1];
      E[0] = csf{1ll << 61, 0, -61};
#pragma unroll
      for (int s = 1; s <= M; ++s) E[s] = csf{0, 0, kZeroExp};
      for (int j = 0; j < n; ++j) {
        const csf c = csf_from_int(myC[2 * j * nt], myC[2 * j * nt + nt], s_e[j]);
        const int lo = M - (n - 1 - j), hi = j + 1;  // the band that can still reach e_m
#pragma unroll
        for (int s = M; s >= 1; --s)
          if (s >= lo && s <= hi) E[s] = csf_add(E[s], csf_mul(c, E[s - 1]));
      }
      const csf v = E[M];
      if ((v.re | v.im) != 0) {
        long long pr = v.re, pi = v.im;
        if (g & 1u) {
          pr = -pr;
          pi = -pi;
        }
        if (!anchored) {
          e_lo = v.e + 62 - kAnchorBit;
          anchored = true;
        }
        int p = v.e - e_lo;
        if (p > kMaxLsb) {
          shr192(r0, r1, r2, p - kMaxLsb);
          shr192(i0, i1, i2, p - kMaxLsb);
          e_lo += p - kMaxLsb;
          p = kMaxLsb;
        }
        add192(r0, r1, r2, pr, p);
        add192(i0, i1, i2, pi, p);
      }
    }
  }
  dd v[3] = {to_dd(r0, r1, r2, e_lo), to_dd(i0, i1, i2, e_lo), dd{0.0, 0.0}};
  block_sum_dd<3>(v, scratch);
  if (threadIdx.x == 0) {
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * kCplxRecord;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const bool bad = tab->bad != 0;
    rec[0] = bad ? nan : v[0].hi;
    rec[1] = bad ? 0.0 : v[0].lo;
    rec[2] = bad ? nan : v[1].hi;
    rec[3] = bad ? 0.0 : v[1].lo;
    rec[4] = 0.0;
    rec[5] = 0.0;
  }
}

void* pick(int m) {
  switch (m) {
#define CESYM_CASE(k) \
  case k: return (void*)glynn_cesym_kernel<k>;
    CESYM_CASE(1) CESYM_CASE(2) CESYM_CASE(3) CESYM_CASE(4) CESYM_CASE(5) CESYM_CASE(6) CESYM_CASE(7)
    CESYM_CASE(8) CESYM_CASE(9) CESYM_CASE(10) CESYM_CASE(11) CESYM_CASE(12) CESYM_CASE(13) CESYM_CASE(14)
    CESYM_CASE(15) CESYM_CASE(16) CESYM_CASE(17) CESYM_CASE(18) CESYM_CASE(19) CESYM_CASE(20) CESYM_CASE(21)
    CESYM_CASE(22) CESYM_CASE(23) CESYM_CASE(24) CESYM_CASE(25) CESYM_CASE(26) CESYM_CASE(27) CESYM_CASE(28)
    CESYM_CASE(29) CESYM_CASE(30) CESYM_CASE(31) CESYM_CASE(32)
#undef CESYM_CASE
    default: return nullptr;
  }
}

size_t smem_bytes(int m, int n, int block) { return (2 * (size_t)m * n + 2 * (size_t)n * block) * sizeof(long long); }

}  // namespace

int glynn_cesym_max_m() { return kMaxM; }
int glynn_cesym_block() { return kBlock; }

int glynn_cesym_blocks_per_sm(int m, int n, int block) {
  void* k = pick(m);
  if (!k || n > 64 || m >= n) return 0;
  const size_t smem = smem_bytes(m, n, block);
  if (smem > 32 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_glynn_cesym(const SweepArgs& a, CesymTable* tab, const LaunchCfg& c) {
  if (a.m < 1 || a.m >= a.n || a.n > 64 || c.block > kBlock || c.block % 32) return cudaErrorInvalidValue;
  void* k = pick(a.m);
  if (!k) return cudaErrorInvalidValue;
  cesym_prep_kernel<<<1, 64, 0, c.stream>>>(a, tab);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = smem_bytes(a.m, a.n, c.block);
  if (smem > 32 * 1024) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  SweepArgs args = a;
  const CesymTable* tp = tab;
  void* params[] = {&args, &tp};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), params, smem, c.stream);
}

}  // namespace perm
