// Glynn's formula (Eq. glynn, Eq. glynn_rectangle) for complex input on the integer
// pipes, the complex counterpart of glynn_fx.cu:
//   * column j is held in fixed point with its own scale 2^e_j, chosen so that
//     sum_i (|re a'_ij| + |im a'_ij|) 2^e_j <= 2^61; real and imaginary parts are
//     rounded once to int64, and the +-2q updates of the walk are exact;
//   * the running product is a complex software float: two signed 64-bit mantissas
//     (re, im) with one shared exponent, the larger magnitude kept in [2^61, 2^62).
//     Each factor is normalised the same way, the four partial products are the high
//     halves of signed 64x64-bit products (truncation error < 2^-60 of the larger
//     component), and the result is renormalised by clz of the larger component;
//   * the signed terms go into two 192-bit fixed-point accumulators (re, im) sharing a
//     window anchored on the thread's first nonzero term, moved up if a later term
//     would overflow it.
#include "device_common.cuh"
#include "fixed_common.cuh"
#include "internal.h"

namespace perm {
namespace {

// One block, one thread per column: scales and the quantised +-2q table (re, im).
__global__ void cfx_prep_kernel(SweepArgs a, CfxTable* tab) {
  const int n = a.n, m = a.m;
  const double* A = static_cast<const double*>(a.A);
  __shared__ int es[64];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < n) {
    double colabs = (double)(n - m);
    for (int i = 0; i < m; ++i) {
      const int64_t e = 2 * (i * a.rs + j * a.cs);
      if (!isfinite(A[e]) || !isfinite(A[e + 1])) bad = 1;
      colabs += fabs(A[e]) + fabs(A[e + 1]);
    }
    int x = 0;
    if (colabs > 0.0) frexp(colabs, &x);
    const int e = 61 - x;
    es[j] = e;
    for (int i = 0; i < n; ++i) {
      long long qr = 0, qi = 0;
      if (i < m) {
        const int64_t el = 2 * (i * a.rs + j * a.cs);
        qr = llrint(ldexp(A[el], e));
        qi = llrint(ldexp(A[el + 1], e));
      } else {
        qr = llrint(ldexp(1.0, e));
      }
      tab->d[2 * (i * 64 + j)] = 2 * qr;
      tab->d[2 * (i * 64 + j) + 1] = 2 * qi;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int esum = 0;
    for (int k = 0; k < n; ++k) esum += es[k];
    tab->e_sum = esum;
    tab->bad = bad;
  }
}

// The column sums of every thread live in shared memory (sS[j][thread], re and im),
// so the column loop is a rolled loop over the actual n columns: the kernel body stays
// small enough for the instruction cache.  The table row update of a step is fused
// into the product loop.
template <bool SHARE>
__global__ void __launch_bounds__(128) glynn_cfx_kernel(SweepArgs a, const CfxTable* __restrict__ tab) {
  extern __shared__ long long smem_cfx[];
  __shared__ dd scratch[3 * 32];
  const int n = a.n;
  const int T = blockDim.x;
  long long* sP = smem_cfx;            // +2q: row i, column j at 2 (i n + j) (re, im)
  long long* sM = sP + 2 * n * n;      // -2q
  long long* sS = sM + 2 * n * n;      // column sums: column j of thread t at 2 (j T + t)
  for (int idx = threadIdx.x; idx < n * n; idx += T) {
    const int i = idx / n, j = idx - i * n;
    const long long vr = tab->d[2 * (i * 64 + j)];
    const long long vi = tab->d[2 * (i * 64 + j) + 1];
    sP[2 * idx] = vr;
    sP[2 * idx + 1] = vi;
    sM[2 * idx] = -vr;
    sM[2 * idx + 1] = -vi;
  }
  const int e_sum = tab->e_sum;
  __syncthreads();
  long long* mine = sS + 2 * threadIdx.x;  // column j at mine[2 j T]
  const int nint = SHARE ? n - a.fp64_cols : n;  // columns on the integer pipes (>= 1)

  // aligned chunks of 2^chunk_log2 terms, 32 consecutive chunks per warp per round
  const int lane = threadIdx.x & 31;
  const uint64_t L = 1ull << a.chunk_log2;
  const uint64_t c_first = a.g_begin >> a.chunk_log2;
  const uint64_t c_end = (a.g_end + L - 1) >> a.chunk_log2;
  const uint64_t rounds = (c_end - c_first + 31) / 32;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);

  int e_lo = 0;
  bool anchored = false;
  u64 r0 = 0, r1 = 0, r2 = 0, i0 = 0, i1 = 0, i2 = 0;
  for (uint64_t rr = warp; rr < rounds; rr += warps) {
    const uint64_t chunk = c_first + 32 * rr + lane;
    uint64_t ga = chunk << a.chunk_log2, gb = ga + L;
    if (ga < a.g_begin) ga = a.g_begin;
    if (gb > a.g_end) gb = a.g_end;
    if (chunk >= c_end) ga = gb = a.g_end;  // idle lane
    for (uint64_t g = ga; g < gb; ++g) {
      const long long* row = nullptr;  // update row of this step (null at a rebuild)
      if (g == ga) {
        const uint64_t gray = g ^ (g >> 1);
        for (int j = 0; j < n; ++j) {
          long long sr = 0, si = 0;
          for (int i = 0; i < n; ++i) {
            const long long* t = (((gray >> (n - 1 - i)) & 1u) ? sM : sP) + 2 * (i * n + j);
            sr += t[0];
            si += t[1];
          }
          mine[2 * j * T] = sr >> 1;
          mine[2 * j * T + 1] = si >> 1;
        }
      } else {
        const int b = ctz64(g);
        row = (((g >> (b + 1)) & 1u) ? sP : sM) + 2 * (n - 1 - b) * n;
      }
      // product over the columns, (pr + i pi) 2^(E - 62), larger component in [2^61, 2^62);
      // the last K columns (mixed) on the FP64 unit as a complex double dr + i di
      long long pr = 0, pi = 0;
      int E = 0;
      double dr = 1.0, di = 0.0;
#pragma unroll 2
      for (int j = 0; j < n; ++j) {
        long long sr = mine[2 * j * T], si = mine[2 * j * T + 1];
        if (row) {
          sr += row[2 * j];
          si += row[2 * j + 1];
          mine[2 * j * T] = sr;
          mine[2 * j * T + 1] = si;
        }
        if (!SHARE || j < nint) {
          const int l = norm_shift(sr, si);
          sr <<= l;
          si <<= l;
          if (j == 0) {
            pr = sr;
            pi = si;
            E = 62 - l;
          } else {
            cmul_step(pr, pi, E, sr, si, l);
          }
        } else {
          const double xr = (double)sr, xi = (double)si;  // rounded once (|s| <= 2^61)
          const double nr = __fma_rn(dr, xr, -__dmul_rn(di, xi));
          const double ni = __fma_rn(dr, xi, __dmul_rn(di, xr));
          dr = nr;
          di = ni;
        }
      }
      if (SHARE && nint < n && (pr != 0 || pi != 0)) cfold_double(pr, pi, E, dr, di);
      if (pr != 0 || pi != 0) {
        if (g & 1u) {
          pr = -pr;
          pi = -pi;
        }
        if (!anchored) {
          e_lo = E - e_sum - kAnchorBit - 1;
          anchored = true;
        }
        // a component's lsb has weight 2^(E - 62 - e_sum): bit p of the accumulators
        int p = E - 62 - e_sum - e_lo;
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
    const bool bad = tab->bad != 0;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * kCplxRecord;
    rec[0] = bad ? nan : v[0].hi;
    rec[1] = bad ? 0.0 : v[0].lo;
    rec[2] = bad ? nan : v[1].hi;
    rec[3] = bad ? 0.0 : v[1].lo;
    rec[4] = 0.0;
    rec[5] = 0.0;
  }
}

// Rectangular Glynn (Eq. glynn_rectangle) with the n - m padding rows of ones grouped
// by their number t of -1 signs: the column sums shift by (n - m - 2t) u_j (u_j the
// quantised 1 of column j, real), the sign by (-1)^t, and C(n - m, t) padding sign
// vectors share each t.  The walk runs over the 2^(m-1) sign vectors of the real rows
// (Gray code, bit b <-> row m-1-b, term sign (-1)^g); at each it takes the n - m + 1
// values of t, up for even g and down for odd g.  The product is multiplied by
// C(n - m, t) (truncation < 2^-61) before the 192-bit accumulation.
__global__ void __launch_bounds__(128) glynn_cfxg_kernel(SweepArgs a, const CfxTable* __restrict__ tab) {
  extern __shared__ long long smem_cfx[];
  __shared__ dd scratch[3 * 32];
  __shared__ long long s_wm[64];  // C(n - m, t) = s_wm[t] 2^(1 - s_wl[t]), s_wm in [2^62, 2^63)
  __shared__ int s_wl[64];
  const int n = a.n, m = a.m, k = n - m;
  const int R = m + 1;  // the real rows and one padding row
  const int T = blockDim.x;
  long long* sP = smem_cfx;            // +2q: row i, column j at 2 (i n + j) (re, im)
  long long* sM = sP + 2 * R * n;      // -2q
  long long* sS = sM + 2 * R * n;      // column sums: column j of thread t at 2 (j T + t)
  for (int idx = threadIdx.x; idx < R * n; idx += T) {
    const int i = idx / n, j = idx - i * n;
    const long long vr = tab->d[2 * (i * 64 + j)];
    const long long vi = tab->d[2 * (i * 64 + j) + 1];
    sP[2 * idx] = vr;
    sP[2 * idx + 1] = vi;
    sM[2 * idx] = -vr;
    sM[2 * idx + 1] = -vi;
  }
  for (int t = threadIdx.x; t <= k; t += T) {
    unsigned __int128 c = 1;
    for (int i = 1; i <= t; ++i) c = c * (unsigned __int128)(k - t + i) / (unsigned __int128)i;
    const int l = __clzll((long long)(unsigned long long)c);  // c < 2^60: l >= 4
    s_wm[t] = (long long)((unsigned long long)c << (l - 1));
    s_wl[t] = l;
  }
  const int e_sum = tab->e_sum;
  __syncthreads();
  long long* mine = sS + 2 * threadIdx.x;
  const long long* padP = sP + 2 * m * n;
  const long long* padM = sM + 2 * m * n;

  const int lane = threadIdx.x & 31;
  const uint64_t L = 1ull << a.chunk_log2;
  const uint64_t c_first = a.g_begin >> a.chunk_log2;
  const uint64_t c_end = (a.g_end + L - 1) >> a.chunk_log2;
  const uint64_t rounds = (c_end - c_first + 31) / 32;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);

  int e_lo = 0;
  bool anchored = false;
  u64 r0 = 0, r1 = 0, r2 = 0, i0 = 0, i1 = 0, i2 = 0;
  for (uint64_t rr = warp; rr < rounds; rr += warps) {
    const uint64_t chunk = c_first + 32 * rr + lane;
    uint64_t ga = chunk << a.chunk_log2, gb = ga + L;
    if (ga < a.g_begin) ga = a.g_begin;
    if (gb > a.g_end) gb = a.g_end;
    if (chunk >= c_end) ga = gb = a.g_end;
    for (uint64_t g = ga; g < gb; ++g) {
      const bool up = (g & 1u) == 0;
      const long long* row = nullptr;  // real-row update of this step (null at a rebuild)
      if (g == ga) {
        const uint64_t gray = g ^ (g >> 1);
        const long long* pad = up ? padP : padM;  // padding sum +(n-m) or -(n-m)
        for (int j = 0; j < n; ++j) {
          long long sr = (long long)k * pad[2 * j], si = (long long)k * pad[2 * j + 1];
          for (int i = 0; i < m; ++i) {
            const long long* t = (((gray >> (m - 1 - i)) & 1u) ? sM : sP) + 2 * (i * n + j);
            sr += t[0];
            si += t[1];
          }
          mine[2 * j * T] = sr >> 1;
          mine[2 * j * T + 1] = si >> 1;
        }
      } else {
        const int b = ctz64(g);
        row = (((g >> (b + 1)) & 1u) ? sP : sM) + 2 * (m - 1 - b) * n;
      }
      for (int st = 0; st <= k; ++st) {
        const long long* upd = row;  // the real-row flip goes with the first t of the step
        if (st > 0) upd = up ? padM : padP;
        long long pr = 0, pi = 0;
        int E = 0;
#pragma unroll 2
        for (int j = 0; j < n; ++j) {
          long long sr = mine[2 * j * T], si = mine[2 * j * T + 1];
          if (upd) {
            sr += upd[2 * j];
            si += upd[2 * j + 1];
            mine[2 * j * T] = sr;
            mine[2 * j * T + 1] = si;
          }
          const int l = norm_shift(sr, si);
          sr <<= l;
          si <<= l;
          if (j == 0) {
            pr = sr;
            pi = si;
            E = 62 - l;
          } else {
            cmul_step(pr, pi, E, sr, si, l);
          }
        }
        if (pr != 0 || pi != 0) {
          const int t = up ? st : k - st;
          const long long hr = __mul64hi(pr, s_wm[t]), hi = __mul64hi(pi, s_wm[t]);
          const int l2 = norm_shift(hr, hi);
          pr = hr << l2;
          pi = hi << l2;
          E += 65 - s_wl[t] - l2;
          if (((unsigned)(g & 1u) ^ (unsigned)(t & 1)) != 0u) {
            pr = -pr;
            pi = -pi;
          }
          if (!anchored) {
            e_lo = E - e_sum - kAnchorBit - 1;
            anchored = true;
          }
          int p = E - 62 - e_sum - e_lo;
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
  }

  dd v[3] = {to_dd(r0, r1, r2, e_lo), to_dd(i0, i1, i2, e_lo), dd{0.0, 0.0}};
  block_sum_dd<3>(v, scratch);
  if (threadIdx.x == 0) {
    const bool bad = tab->bad != 0;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * kCplxRecord;
    rec[0] = bad ? nan : v[0].hi;
    rec[1] = bad ? 0.0 : v[0].lo;
    rec[2] = bad ? nan : v[1].hi;
    rec[3] = bad ? 0.0 : v[1].lo;
    rec[4] = 0.0;
    rec[5] = 0.0;
  }
}

size_t smem_bytes_grouped(int m, int n, int block) {
  return (4u * (size_t)(m + 1) * n + 2u * (size_t)n * block) * sizeof(long long);
}

size_t smem_bytes(int n, int block) { return (4u * (size_t)n * n + 2u * (size_t)n * block) * sizeof(long long); }

}  // namespace

int glynn_cfx_max_n() { return 64; }

int glynn_cfx_blocks_per_sm(int m, int n, int block, bool grouped) {
  const void* k = grouped ? (const void*)glynn_cfxg_kernel : (const void*)glynn_cfx_kernel<false>;
  const size_t smem = grouped ? smem_bytes_grouped(m, n, block) : smem_bytes(n, block);
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_glynn_cfx(const SweepArgs& a, CfxTable* tab, const LaunchCfg& c, bool grouped) {
  if (grouped && (a.m < 1 || a.m >= a.n)) return cudaErrorInvalidValue;
  cfx_prep_kernel<<<1, 64, 0, c.stream>>>(a, tab);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const void* k = grouped ? (const void*)glynn_cfxg_kernel
                          : (a.fp64_cols > 0 ? (const void*)glynn_cfx_kernel<true> : (const void*)glynn_cfx_kernel<false>);
  const size_t smem = grouped ? smem_bytes_grouped(a.m, a.n, c.block) : smem_bytes(a.n, c.block);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  SweepArgs args = a;
  const CfxTable* tp = tab;
  void* params[] = {&args, &tp};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), params, smem, c.stream);
}

}  // namespace perm
