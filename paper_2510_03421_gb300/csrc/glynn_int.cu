// Glynn's formula (Eq. glynn, Eq. glynn_rectangle) for integer input (uint8 0/1
// matrices or int64), exact: column sums are int64 and stay exact under the +-2 a'_rj
// updates (so no periodic rebuild is needed beyond the start of each thread's
// slice), products and the signed sum are taken modulo 2^128 in unsigned 128-bit
// integers.  Wrap-around is exact modulo 2^128, so the final sum equals
// 2^(n-1) (n-m)! per(A) whenever that value fits in a signed 128-bit integer; the
// a-priori bound kernel below flags inputs for which that is not guaranteed.
#include "device_common.cuh"
#include "int_bound.cuh"
#include "internal.h"

namespace perm {
namespace {

typedef unsigned __int128 u128;

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int off) {
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  lo = __shfl_down_sync(0xffffffffu, lo, off);
  hi = __shfl_down_sync(0xffffffffu, hi, off);
  return ((u128)hi << 64) | lo;
}

// P * s modulo 2^128 for a signed 64-bit s.
__device__ __forceinline__ u128 mul_s64(u128 P, long long s) { return P * (u128)(__int128)s; }

template <typename T>
__device__ __forceinline__ long long load_int(const void* A, int64_t e) {
  return (long long)static_cast<const T*>(A)[e];
}

template <int N, typename T>
__global__ void __launch_bounds__(256) glynn_int_kernel(SweepArgs a) {
  extern __shared__ long long smem_i[];
  __shared__ u128 scratch[32];
  const int n = a.n, m = a.m;
  long long* sP = smem_i;          // +2 a'_ij
  long long* sM = smem_i + n * N;  // -2 a'_ij
  for (int idx = threadIdx.x; idx < n * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    long long v = 0;
    if (j < n) v = (i < m) ? load_int<T>(a.A, i * a.rs + j * a.cs) : 1;
    sP[idx] = 2 * v;
    sM[idx] = -2 * v;
  }
  __syncthreads();

  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t g, len;
  split_range(a.g_begin, a.g_end, nt, tid, &g, &len);

  u128 acc = 0;
  long long S[N];
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0) {
      const uint64_t gray = g ^ (g >> 1);
#pragma unroll
      for (int j = 0; j < N; ++j) S[j] = 0;
      for (int i = 0; i < n; ++i) {
        const long long* row = (((gray >> (n - 1 - i)) & 1u) ? sM : sP) + i * N;
#pragma unroll
        for (int j = 0; j < N; ++j) S[j] += row[j];
      }
#pragma unroll
      for (int j = 0; j < N; ++j) S[j] = (j < n) ? S[j] / 2 : 1;
    } else {
      const int b = ctz64(g);
      const long long* row = (((g >> (b + 1)) & 1u) ? sP : sM) + (n - 1 - b) * N;
#pragma unroll
      for (int j = 0; j < N; ++j) S[j] += row[j];
    }
    u128 P = (u128)(__int128)S[0];
#pragma unroll
    for (int j = 1; j < N; ++j) P = mul_s64(P, S[j]);
    if (g & 1u) acc -= P; else acc += P;
  }

#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += shfl_down_u128(acc, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) scratch[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    u128 x = (lane < nw) ? scratch[lane] : (u128)0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += shfl_down_u128(x, off);
    if (lane == 0) {
      unsigned long long* rec = static_cast<unsigned long long*>(a.partials) + (size_t)blockIdx.x * kIntRecord;
      rec[0] = (unsigned long long)x;
      rec[1] = (unsigned long long)(x >> 64);
    }
  }
}

// Rectangular Glynn (Eq. glynn_rectangle) with the n - m padding rows of ones grouped
// by their number t of -1 signs: column sums shifted by n - m - 2t, sign (-1)^t,
// multiplicity C(n - m, t) (an exact integer weight).  The walk runs over the
// 2^(m-1) sign vectors of the real rows (bit b of gray(g) <-> row m-1-b, term sign
// (-1)^g); at each it takes the n - m + 1 values of t, up for even g and down for odd
// g, one padding update (+-2 per column) apart.  Products, weights and the signed sum
// are exact modulo 2^128, so the total is the same sum as the ungrouped walk's.
template <int N, typename T>
__global__ void __launch_bounds__(256) glynn_intg_kernel(SweepArgs a) {
  extern __shared__ long long smem_i[];
  __shared__ u128 scratch[32];
  __shared__ unsigned long long s_w[64];  // C(n - m, t)
  const int n = a.n, m = a.m, k = n - m;
  const int R = m + 1;                    // the real rows and one padding row
  long long* sP = smem_i;                 // +2 a'_ij
  long long* sM = smem_i + R * N;         // -2 a'_ij
  for (int idx = threadIdx.x; idx < R * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    long long v = 0;
    if (j < n) v = (i < m) ? load_int<T>(a.A, i * a.rs + j * a.cs) : 1;
    sP[idx] = 2 * v;
    sM[idx] = -2 * v;
  }
  for (int t = threadIdx.x; t <= k; t += blockDim.x) {
    u128 c = 1;
    for (int i = 1; i <= t; ++i) c = c * (u128)(k - t + i) / (u128)i;
    s_w[t] = (unsigned long long)c;
  }
  __syncthreads();
  const long long* padP = sP + m * N;
  const long long* padM = sM + m * N;

  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t g, len;
  split_range(a.g_begin, a.g_end, nt, tid, &g, &len);

  u128 acc = 0;
  long long S[N];
  for (uint64_t s = 0; s < len; ++s, ++g) {
    const bool up = (g & 1u) == 0;
    if (s == 0) {
      const uint64_t gray = g ^ (g >> 1);
#pragma unroll
      for (int j = 0; j < N; ++j) S[j] = 0;
      for (int i = 0; i < m; ++i) {
        const long long* row = (((gray >> (m - 1 - i)) & 1u) ? sM : sP) + i * N;
#pragma unroll
        for (int j = 0; j < N; ++j) S[j] += row[j];
      }
      const long long* pad = up ? padP : padM;  // padding sum +k (t = 0) or -k (t = k)
#pragma unroll
      for (int j = 0; j < N; ++j) S[j] = (j < n) ? (S[j] + (long long)k * pad[j]) / 2 : 1;
    } else {
      const int b = ctz64(g);
      const long long* row = (((g >> (b + 1)) & 1u) ? sP : sM) + (m - 1 - b) * N;
#pragma unroll
      for (int j = 0; j < N; ++j) S[j] += row[j];
    }
    for (int st = 0; st <= k; ++st) {
      if (st > 0) {
        const long long* pad = up ? padM : padP;
#pragma unroll
        for (int j = 0; j < N; ++j) S[j] += pad[j];
      }
      const int t = up ? st : k - st;
      u128 P = (u128)(__int128)S[0];
#pragma unroll
      for (int j = 1; j < N; ++j) P = mul_s64(P, S[j]);
      P *= (u128)s_w[t];
      if (((unsigned)(g & 1u) ^ (unsigned)(t & 1)) != 0u) acc -= P; else acc += P;
    }
  }

#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += shfl_down_u128(acc, off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) scratch[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    u128 x = (lane < nw) ? scratch[lane] : (u128)0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += shfl_down_u128(x, off);
    if (lane == 0) {
      unsigned long long* rec = static_cast<unsigned long long*>(a.partials) + (size_t)blockIdx.x * kIntRecord;
      rec[0] = (unsigned long long)x;
      rec[1] = (unsigned long long)(x >> 64);
    }
  }
}

template <int N>
void* kernel_for_grouped(int dtype) {
  return dtype == 2 ? (void*)glynn_intg_kernel<N, unsigned char> : (void*)glynn_intg_kernel<N, long long>;
}

void* pick_grouped(int n, int dtype) {
  switch ((n + 3) & ~3) {
    case 4: return kernel_for_grouped<4>(dtype);
    case 8: return kernel_for_grouped<8>(dtype);
    case 12: return kernel_for_grouped<12>(dtype);
    case 16: return kernel_for_grouped<16>(dtype);
    case 20: return kernel_for_grouped<20>(dtype);
    case 24: return kernel_for_grouped<24>(dtype);
    case 28: return kernel_for_grouped<28>(dtype);
    case 32: return kernel_for_grouped<32>(dtype);
    case 36: return kernel_for_grouped<36>(dtype);
    case 40: return kernel_for_grouped<40>(dtype);
    case 44: return kernel_for_grouped<44>(dtype);
    case 48: return kernel_for_grouped<48>(dtype);
    case 52: return kernel_for_grouped<52>(dtype);
    case 56: return kernel_for_grouped<56>(dtype);
    case 60: return kernel_for_grouped<60>(dtype);
    case 64: return kernel_for_grouped<64>(dtype);
    default: return nullptr;
  }
}

// Gaussian integers (dtype 4): the same walk with complex column sums (int64 real and
// imaginary parts) and complex products and sums modulo 2^128 per component.  The
// per-block records are written as two arrays of int128: the real parts at records
// [0, grid), the imaginary parts at [grid, 2 grid).
template <int N>
__global__ void __launch_bounds__(128) glynn_cint_kernel(SweepArgs a) {
  extern __shared__ long long smem_i[];
  __shared__ u128 scratch[2 * 32];
  const int n = a.n, m = a.m;
  long long* sP = smem_i;              // +2 a'_ij as (re, im) at 2 (i N + j)
  long long* sM = smem_i + 2 * n * N;  // -2 a'_ij
  const long long* A = static_cast<const long long*>(a.A);
  for (int idx = threadIdx.x; idx < n * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    long long vr = 0, vi = 0;
    if (j < n) {
      if (i < m) {
        vr = A[2 * (i * a.rs + j * a.cs)];
        vi = A[2 * (i * a.rs + j * a.cs) + 1];
      } else {
        vr = 1;
      }
    }
    sP[2 * idx] = 2 * vr;
    sP[2 * idx + 1] = 2 * vi;
    sM[2 * idx] = -2 * vr;
    sM[2 * idx + 1] = -2 * vi;
  }
  __syncthreads();

  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t g, len;
  split_range(a.g_begin, a.g_end, nt, tid, &g, &len);

  u128 acc_r = 0, acc_i = 0;
  long long Sr[N], Si[N];
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0) {
      const uint64_t gray = g ^ (g >> 1);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        Sr[j] = 0;
        Si[j] = 0;
      }
      for (int i = 0; i < n; ++i) {
        const long long* row = (((gray >> (n - 1 - i)) & 1u) ? sM : sP) + 2 * i * N;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          Sr[j] += row[2 * j];
          Si[j] += row[2 * j + 1];
        }
      }
#pragma unroll
      for (int j = 0; j < N; ++j) {
        Sr[j] = (j < n) ? Sr[j] / 2 : 1;
        Si[j] = (j < n) ? Si[j] / 2 : 0;
      }
    } else {
      const int b = ctz64(g);
      const long long* row = (((g >> (b + 1)) & 1u) ? sP : sM) + 2 * (n - 1 - b) * N;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        Sr[j] += row[2 * j];
        Si[j] += row[2 * j + 1];
      }
    }
    u128 pr = (u128)(__int128)Sr[0], pi = (u128)(__int128)Si[0];
#pragma unroll
    for (int j = 1; j < N; ++j) {
      const u128 nr = mul_s64(pr, Sr[j]) - mul_s64(pi, Si[j]);
      const u128 ni = mul_s64(pr, Si[j]) + mul_s64(pi, Sr[j]);
      pr = nr;
      pi = ni;
    }
    if (g & 1u) {
      acc_r -= pr;
      acc_i -= pi;
    } else {
      acc_r += pr;
      acc_i += pi;
    }
  }

#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    acc_r += shfl_down_u128(acc_r, off);
    acc_i += shfl_down_u128(acc_i, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) {
    scratch[warp] = acc_r;
    scratch[32 + warp] = acc_i;
  }
  __syncthreads();
  if (warp == 0) {
    u128 xr = (lane < nw) ? scratch[lane] : (u128)0;
    u128 xi = (lane < nw) ? scratch[32 + lane] : (u128)0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      xr += shfl_down_u128(xr, off);
      xi += shfl_down_u128(xi, off);
    }
    if (lane == 0) {
      unsigned long long* rec = static_cast<unsigned long long*>(a.partials);
      rec[kIntRecord * blockIdx.x] = (unsigned long long)xr;
      rec[kIntRecord * blockIdx.x + 1] = (unsigned long long)(xr >> 64);
      rec[kIntRecord * (gridDim.x + blockIdx.x)] = (unsigned long long)xi;
      rec[kIntRecord * (gridDim.x + blockIdx.x) + 1] = (unsigned long long)(xi >> 64);
    }
  }
}

void* pick_gaussian(int n) {
  switch ((n + 3) & ~3) {
    case 4: return (void*)glynn_cint_kernel<4>;
    case 8: return (void*)glynn_cint_kernel<8>;
    case 12: return (void*)glynn_cint_kernel<12>;
    case 16: return (void*)glynn_cint_kernel<16>;
    case 20: return (void*)glynn_cint_kernel<20>;
    case 24: return (void*)glynn_cint_kernel<24>;
    case 28: return (void*)glynn_cint_kernel<28>;
    case 32: return (void*)glynn_cint_kernel<32>;
    default: return nullptr;
  }
}

template <int N>
void* kernel_for(int dtype) {
  return dtype == 2 ? (void*)glynn_int_kernel<N, unsigned char> : (void*)glynn_int_kernel<N, long long>;
}

void* pick(int n, int dtype) {
  switch ((n + 3) & ~3) {
    case 4: return kernel_for<4>(dtype);
    case 8: return kernel_for<8>(dtype);
    case 12: return kernel_for<12>(dtype);
    case 16: return kernel_for<16>(dtype);
    case 20: return kernel_for<20>(dtype);
    case 24: return kernel_for<24>(dtype);
    case 28: return kernel_for<28>(dtype);
    case 32: return kernel_for<32>(dtype);
    case 36: return kernel_for<36>(dtype);
    case 40: return kernel_for<40>(dtype);
    case 44: return kernel_for<44>(dtype);
    case 48: return kernel_for<48>(dtype);
    case 52: return kernel_for<52>(dtype);
    case 56: return kernel_for<56>(dtype);
    case 60: return kernel_for<60>(dtype);
    case 64: return kernel_for<64>(dtype);
    default: return nullptr;
  }
}

size_t smem_bytes(int n) { return 2u * (size_t)n * (size_t)((n + 3) & ~3) * sizeof(long long); }

// A-priori bound on |2^(n-1) (n-m)! per(A)|: log2 of 2^(n-1) (n-m)! prod_i sum_j |a_ij|
// and, for 0/1 matrices, of 2^(n-1) times Bregman's bound prod_i (r_i!)^(1/r_i) on
// the permanent of the padded matrix A' (pad rows have n ones).  Also guards the
// int64 column sums.  Sets *status = PERM_EOVERFLOW (3) if exactness is not assured.
// |a| of element e (Gaussian integers: |re| + |im|, an upper bound of the modulus).
__device__ __forceinline__ double mag_of(const void* A, int dtype, int64_t e) {
  if (dtype == 2) return (double)static_cast<const unsigned char*>(A)[e];
  const long long* p = static_cast<const long long*>(A);
  if (dtype == 4) return fabs((double)p[2 * e]) + fabs((double)p[2 * e + 1]);
  return fabs((double)p[e]);
}

// glynn: the bound of the Glynn and Ryser sums, 2^(n-1) (n-m)! per(|A|) (Bregman for 0/1
// input, and the column sums' headroom); otherwise that of the plain sum of products
// (the combinatoric algorithm), per(|A|) <= prod_i sum_j |a_ij|.
__global__ void int_bound_kernel(const void* A, int dtype, int m, int n, int64_t rs, int64_t cs, int* status,
                                 bool glynn) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double lrow = 0.0, lbreg = 0.0;
  bool binary = true, zero_row = false, col_overflow = false;
  for (int i = 0; i < m; ++i) {
    double rsum = 0.0;
    for (int j = 0; j < n; ++j) {
      const int64_t e = i * rs + j * cs;
      const double v = mag_of(A, dtype, e);
      if (v > 1.0 || dtype == 4) binary = false;
      rsum += v;
    }
    if (rsum == 0.0) zero_row = true;
    else {
      lrow += log2(rsum);
      lbreg += bregman_log2_term(rsum);
    }
  }
  for (int j = 0; j < n; ++j) {
    double csum = 0.0;
    for (int i = 0; i < m; ++i) {
      const int64_t e = i * rs + j * cs;
      csum += mag_of(A, dtype, e);
    }
    if (column_sum_overflows(csum, m, n)) col_overflow = true;
  }
  if (!glynn) {
    if (!zero_row && lrow >= kInt128Bits) *status = 3;
    return;
  }
  if (zero_row) {
    if (col_overflow) *status = 3;
    return;
  }
  if (glynn_sum_log2_bound(m, n, lrow, lbreg, binary) >= kInt128Bits || col_overflow) *status = 3;
}

}  // namespace

int glynn_int_blocks_per_sm(int n, int dtype, int block, bool grouped) {
  void* k = grouped ? pick_grouped(n, dtype) : pick(n, dtype);
  if (!k) return 0;
  size_t smem = smem_bytes(n);  // at least the grouped walk's (m + 1) rows
  if (smem > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_glynn_int(const SweepArgs& a, int dtype, const LaunchCfg& c, bool grouped) {
  if (grouped && (a.m < 1 || a.m >= a.n)) return cudaErrorInvalidValue;
  void* k = grouped ? pick_grouped(a.n, dtype) : pick(a.n, dtype);
  if (!k) return cudaErrorInvalidValue;
  size_t smem = grouped ? 2u * (size_t)(a.m + 1) * (size_t)((a.n + 3) & ~3) * sizeof(long long) : smem_bytes(a.n);
  if (smem > 32 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  SweepArgs args = a;
  void* params[] = {&args};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), params, smem, c.stream);
}

int glynn_gaussian_max_n() { return 32; }

int glynn_gaussian_blocks_per_sm(int n, int block) {
  void* k = pick_gaussian(n);
  if (!k) return 0;
  const size_t smem = 4u * (size_t)n * (size_t)((n + 3) & ~3) * sizeof(long long);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_glynn_gaussian(const SweepArgs& a, const LaunchCfg& c) {
  void* k = pick_gaussian(a.n);
  if (!k) return cudaErrorInvalidValue;
  const size_t smem = 4u * (size_t)a.n * (size_t)((a.n + 3) & ~3) * sizeof(long long);  // <= 32 KiB
  SweepArgs args = a;
  void* params[] = {&args};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), params, smem, c.stream);
}

cudaError_t launch_int_bound(const void* A, int dtype, int m, int n, int64_t rs, int64_t cs, int* status,
                             cudaStream_t s, bool glynn) {
  int_bound_kernel<<<1, 32, 0, s>>>(A, dtype, m, n, rs, cs, status, glynn);
  return cudaGetLastError();
}

}  // namespace perm
