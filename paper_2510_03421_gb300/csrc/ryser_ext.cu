// Ryser's formula (Eq. ryser_square; Eq. ryser_rectangle in its subset-size form) for
// complex input (FP64, Kahan-compensated) and for integer and Gaussian-integer input
// (exact, modulo 2^128).
// Same walk as ryser_f64.cu: the 2^n column subsets in reflected Gray-code order,
// subset(g) = set bits of gray(g), one column added or removed per step, the m row
// sums updated by +-a_ic, and the term weighted by (-1)^(m-|S|) C(n-|S|, m-|S|).
#include "device_common.cuh"
#include "internal.h"

namespace perm {
namespace {

typedef unsigned __int128 u128;

__device__ __forceinline__ void kahan_add(double& acc, double& comp, double x) {
  const double y = __dsub_rn(x, comp);
  const double s = __dadd_rn(acc, y);
  comp = __dsub_rn(__dsub_rn(s, acc), y);
  acc = s;
}

template <int M, bool WEIGHTED>
__global__ void __launch_bounds__(128) ryser_c128_kernel(SweepArgs a, SizeWeights weights) {
  extern __shared__ double smem[];
  __shared__ dd scratch[3 * 32];
  __shared__ double w[65];
  const int n = a.n, m = a.m;
  double2* sP = reinterpret_cast<double2*>(smem);  // sP[c * M + i] = +a_ic
  double2* sM = sP + n * M;
  const double* A = static_cast<const double*>(a.A);
  for (int idx = threadIdx.x; idx < n * M; idx += blockDim.x) {
    const int c = idx / M, i = idx - c * M;
    double2 v = make_double2(0.0, 0.0);
    if (i < m) {
      const int64_t e = 2 * (i * a.rs + c * a.cs);
      v = make_double2(A[e], A[e + 1]);
    }
    sP[idx] = v;
    sM[idx] = make_double2(-v.x, -v.y);
  }
  for (int s = threadIdx.x; s <= n; s += blockDim.x) w[s] = weights.w[s];
  __syncthreads();

  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t g, len;
  split_range(a.g_begin, a.g_end, nt, tid, &g, &len);
  const uint64_t mask = (a.chunk_log2 >= 63) ? ~0ull : ((1ull << a.chunk_log2) - 1);
  double ar = 0.0, cr = 0.0, ai = 0.0, ci = 0.0;
  double Rr[M], Ri[M];
  int size = 0;
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0 || (g & mask) == 0) {
      const uint64_t gray = g ^ (g >> 1);
      size = __popcll(gray);
#pragma unroll
      for (int i = 0; i < M; ++i) Rr[i] = Ri[i] = 0.0;
      for (int c = 0; c < n; ++c) {
        if (!((gray >> c) & 1u)) continue;
        const double2* col = sP + c * M;
#pragma unroll
        for (int i = 0; i < M; ++i) {
          Rr[i] = __dadd_rn(Rr[i], col[i].x);
          Ri[i] = __dadd_rn(Ri[i], col[i].y);
        }
      }
#pragma unroll
      for (int i = 0; i < M; ++i)
        if (i >= m) {
          Rr[i] = 1.0;
          Ri[i] = 0.0;
        }
    } else {
      const int c = ctz64(g);
      const bool added = !((g >> (c + 1)) & 1u);
      size += added ? 1 : -1;
      const double2* col = (added ? sP : sM) + c * M;
#pragma unroll
      for (int i = 0; i < M; ++i) {
        Rr[i] = __dadd_rn(Rr[i], col[i].x);
        Ri[i] = __dadd_rn(Ri[i], col[i].y);
      }
    }
    double pr = Rr[0], pi = Ri[0];
#pragma unroll
    for (int i = 1; i < M; ++i) {
      const double nr = __fma_rn(pr, Rr[i], -__dmul_rn(pi, Ri[i]));
      const double ni = __fma_rn(pr, Ri[i], __dmul_rn(pi, Rr[i]));
      pr = nr;
      pi = ni;
    }
    double wt;
    if (WEIGHTED) {
      wt = w[size];
    } else {
      wt = (g & 1u) ? -1.0 : 1.0;
    }
    kahan_add(ar, cr, __dmul_rn(pr, wt));
    kahan_add(ai, ci, __dmul_rn(pi, wt));
  }
  dd v[3] = {two_sum(ar, -cr), two_sum(ai, -ci), dd{0.0, 0.0}};
  block_sum_dd<3>(v, scratch);
  if (threadIdx.x == 0) {
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * kCplxRecord;
    rec[0] = v[0].hi;
    rec[1] = v[0].lo;
    rec[2] = v[1].hi;
    rec[3] = v[1].lo;
    rec[4] = 0.0;
    rec[5] = 0.0;
  }
}

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int off) {
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
  lo = __shfl_down_sync(0xffffffffu, lo, off);
  hi = __shfl_down_sync(0xffffffffu, hi, off);
  return ((u128)hi << 64) | lo;
}

template <int M, typename T>
__global__ void __launch_bounds__(256) ryser_int_kernel(SweepArgs a, IntWeights weights) {
  extern __shared__ long long smem_i[];
  __shared__ u128 scratch[32];
  __shared__ u128 w[65];
  const int n = a.n, m = a.m;
  long long* sP = smem_i;  // sP[c * M + i] = +a_ic
  long long* sM = smem_i + n * M;
  for (int idx = threadIdx.x; idx < n * M; idx += blockDim.x) {
    const int c = idx / M, i = idx - c * M;
    const long long v = (i < m) ? (long long)static_cast<const T*>(a.A)[i * a.rs + c * a.cs] : 0;
    sP[idx] = v;
    sM[idx] = -v;
  }
  for (int s = threadIdx.x; s <= n; s += blockDim.x) w[s] = ((u128)weights.hi[s] << 64) | weights.lo[s];
  __syncthreads();

  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t g, len;
  split_range(a.g_begin, a.g_end, nt, tid, &g, &len);
  u128 acc = 0;
  long long R[M];
  int size = 0;
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0) {
      const uint64_t gray = g ^ (g >> 1);
      size = __popcll(gray);
#pragma unroll
      for (int i = 0; i < M; ++i) R[i] = 0;
      for (int c = 0; c < n; ++c) {
        if (!((gray >> c) & 1u)) continue;
#pragma unroll
        for (int i = 0; i < M; ++i) R[i] += sP[c * M + i];
      }
#pragma unroll
      for (int i = 0; i < M; ++i)
        if (i >= m) R[i] = 1;
    } else {
      const int c = ctz64(g);
      const bool added = !((g >> (c + 1)) & 1u);
      size += added ? 1 : -1;
      const long long* col = (added ? sP : sM) + c * M;
#pragma unroll
      for (int i = 0; i < M; ++i) R[i] += col[i];
    }
    u128 P = (u128)(__int128)R[0];
#pragma unroll
    for (int i = 1; i < M; ++i) P *= (u128)(__int128)R[i];
    acc += P * w[size];  // weights carry the sign, modulo 2^128
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

// Gaussian integers (dtype 4): (re, im) row sums in int64, the product and the sums as
// two 128-bit parts modulo 2^128.  Records: real parts at [0, grid), imaginary parts at
// [grid, 2 grid), kIntRecord words each.
template <int M>
__global__ void __launch_bounds__(256) ryser_cint_kernel(SweepArgs a, IntWeights weights) {
  extern __shared__ long long smem_i[];
  __shared__ u128 scratch[2][32];
  __shared__ u128 w[65];
  const int n = a.n, m = a.m;
  long long* sP = smem_i;  // sP[2 (c M + i)] = (re, im) of +a_ic
  long long* sM = smem_i + 2 * n * M;
  const long long* A = static_cast<const long long*>(a.A);
  for (int idx = threadIdx.x; idx < n * M; idx += blockDim.x) {
    const int c = idx / M, i = idx - c * M;
    long long re = 0, im = 0;
    if (i < m) {
      const int64_t e = 2 * (i * a.rs + c * a.cs);
      re = A[e];
      im = A[e + 1];
    }
    sP[2 * idx] = re;
    sP[2 * idx + 1] = im;
    sM[2 * idx] = -re;
    sM[2 * idx + 1] = -im;
  }
  for (int s = threadIdx.x; s <= n; s += blockDim.x) w[s] = ((u128)weights.hi[s] << 64) | weights.lo[s];
  __syncthreads();

  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t g, len;
  split_range(a.g_begin, a.g_end, nt, tid, &g, &len);
  u128 acc_re = 0, acc_im = 0;
  long long Rr[M], Ri[M];
  int size = 0;
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0) {
      const uint64_t gray = g ^ (g >> 1);
      size = __popcll(gray);
#pragma unroll
      for (int i = 0; i < M; ++i) Rr[i] = Ri[i] = 0;
      for (int c = 0; c < n; ++c) {
        if (!((gray >> c) & 1u)) continue;
#pragma unroll
        for (int i = 0; i < M; ++i) {
          Rr[i] += sP[2 * (c * M + i)];
          Ri[i] += sP[2 * (c * M + i) + 1];
        }
      }
#pragma unroll
      for (int i = 0; i < M; ++i)
        if (i >= m) {
          Rr[i] = 1;
          Ri[i] = 0;
        }
    } else {
      const int c = ctz64(g);
      const bool added = !((g >> (c + 1)) & 1u);
      size += added ? 1 : -1;
      const long long* col = (added ? sP : sM) + 2 * c * M;
#pragma unroll
      for (int i = 0; i < M; ++i) {
        Rr[i] += col[2 * i];
        Ri[i] += col[2 * i + 1];
      }
    }
    u128 pr = (u128)(__int128)Rr[0], pi = (u128)(__int128)Ri[0];
#pragma unroll
    for (int i = 1; i < M; ++i) {
      const u128 xr = (u128)(__int128)Rr[i], xi = (u128)(__int128)Ri[i];
      const u128 nr = pr * xr - pi * xi;
      pi = pr * xi + pi * xr;
      pr = nr;
    }
    acc_re += pr * w[size];
    acc_im += pi * w[size];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    acc_re += shfl_down_u128(acc_re, off);
    acc_im += shfl_down_u128(acc_im, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) {
    scratch[0][warp] = acc_re;
    scratch[1][warp] = acc_im;
  }
  __syncthreads();
  if (warp == 0) {
    u128 xr = (lane < nw) ? scratch[0][lane] : (u128)0;
    u128 xi = (lane < nw) ? scratch[1][lane] : (u128)0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      xr += shfl_down_u128(xr, off);
      xi += shfl_down_u128(xi, off);
    }
    if (lane == 0) {
      unsigned long long* rec = static_cast<unsigned long long*>(a.partials);
      rec[(size_t)blockIdx.x * kIntRecord] = (unsigned long long)xr;
      rec[(size_t)blockIdx.x * kIntRecord + 1] = (unsigned long long)(xr >> 64);
      rec[(size_t)(gridDim.x + blockIdx.x) * kIntRecord] = (unsigned long long)xi;
      rec[(size_t)(gridDim.x + blockIdx.x) * kIntRecord + 1] = (unsigned long long)(xi >> 64);
    }
  }
}

template <int M>
void* cplx_for(bool weighted) {
  return weighted ? (void*)ryser_c128_kernel<M, true> : (void*)ryser_c128_kernel<M, false>;
}

template <int M>
void* int_for(int dtype) {
  return dtype == 2 ? (void*)ryser_int_kernel<M, unsigned char> : (void*)ryser_int_kernel<M, long long>;
}

void* pick(int m, int dtype, bool weighted) {
  const int M = (m + 3) & ~3;
  if (dtype == 1) {
    weighted = true;  // square input uses the weights (-1)^(n-|S|): no final sign
    switch (M) {
      case 4: return cplx_for<4>(weighted);
      case 8: return cplx_for<8>(weighted);
      case 12: return cplx_for<12>(weighted);
      case 16: return cplx_for<16>(weighted);
      case 20: return cplx_for<20>(weighted);
      case 24: return cplx_for<24>(weighted);
      case 28: return cplx_for<28>(weighted);
      case 32: return cplx_for<32>(weighted);
      case 36: return cplx_for<36>(weighted);
      case 40: return cplx_for<40>(weighted);
      default: return nullptr;
    }
  }
  if (dtype == 4) {
    switch (M) {
      case 4: return (void*)ryser_cint_kernel<4>;
      case 8: return (void*)ryser_cint_kernel<8>;
      case 12: return (void*)ryser_cint_kernel<12>;
      case 16: return (void*)ryser_cint_kernel<16>;
      case 20: return (void*)ryser_cint_kernel<20>;
      case 24: return (void*)ryser_cint_kernel<24>;
      case 28: return (void*)ryser_cint_kernel<28>;
      case 32: return (void*)ryser_cint_kernel<32>;
      default: return nullptr;
    }
  }
  switch (M) {
    case 4: return int_for<4>(dtype);
    case 8: return int_for<8>(dtype);
    case 12: return int_for<12>(dtype);
    case 16: return int_for<16>(dtype);
    case 20: return int_for<20>(dtype);
    case 24: return int_for<24>(dtype);
    case 28: return int_for<28>(dtype);
    case 32: return int_for<32>(dtype);
    case 36: return int_for<36>(dtype);
    case 40: return int_for<40>(dtype);
    case 44: return int_for<44>(dtype);
    case 48: return int_for<48>(dtype);
    case 52: return int_for<52>(dtype);
    case 56: return int_for<56>(dtype);
    case 60: return int_for<60>(dtype);
    case 64: return int_for<64>(dtype);
    default: return nullptr;
  }
}

size_t smem_bytes(int m, int n, int dtype) {
  return 2u * (size_t)n * (size_t)((m + 3) & ~3) * (dtype == 1 || dtype == 4 ? 16 : 8);
}

}  // namespace

int ryser_ext_blocks_per_sm(int m, int n, int dtype, int block) {
  void* k = pick(m, dtype, m < n);
  if (!k) return 0;
  size_t smem = smem_bytes(m, n, dtype);
  if (smem > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_ryser_ext(const SweepArgs& a, int dtype, const SizeWeights& fw, const IntWeights& iw,
                             const LaunchCfg& c) {
  void* k = pick(a.m, dtype, a.m < a.n);
  if (!k) return cudaErrorInvalidValue;
  size_t smem = smem_bytes(a.m, a.n, dtype);
  if (smem > 32 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  SweepArgs args = a;
  SizeWeights f = fw;
  IntWeights iwv = iw;
  void* params_c[] = {&args, &f};
  void* params_i[] = {&args, &iwv};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), dtype == 1 ? params_c : params_i, smem, c.stream);
}

}  // namespace perm
