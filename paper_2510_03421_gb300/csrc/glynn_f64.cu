// Glynn's formula (Eq. glynn) with the rectangular padding of Eq. glynn_filled_matrix /
// Eq. glynn_rectangle, real input, FP64 arithmetic on the FP64 pipe.
//
// Term g (0 <= g < 2^(n-1)) has sign vector delta(g): delta_i = -1 iff bit (n-1-i)
// of gray(g) = g ^ (g >> 1) is set (row 0 is never flipped), and contributes
// (-1)^g prod_j S_j(g) with S_j(g) = sum_i delta_i a'_ij, where a' is A with n - m
// rows of ones appended.  Going from term g-1 to g flips one row, r = n-1-ctz(g),
// so every column sum moves by +-2 a'_rj: n additions instead of n^2.
//
// Work split: the term range is cut into one contiguous, equal slice per thread.
// A thread rebuilds its column sums exactly at the start of its slice and at every
// multiple of 2^chunk_log2 (bounding the drift of the incremental updates), walks
// the Gray code in between, and sums (-1)^g * prod in a Kahan-compensated FP64
// accumulator.  Block partials are double-double; the final reduction is a fixed
// order double-double sum (reduce.cu), so the result is deterministic.
//
// Columns are padded to N (a multiple of 4, compile time) so the sums live in
// registers; padded columns hold S_j = 1 and zero update rows.  Shared memory holds
// +2a' and -2a' (2 n N doubles).
#include "device_common.cuh"
#include "internal.h"

namespace perm {
namespace {


template <int N, bool ABS>
__global__ void __launch_bounds__(256) glynn_f64_kernel(SweepArgs a) {
  extern __shared__ double smem[];
  __shared__ dd scratch[3 * 32];
  __shared__ double s_eps[ABS ? N : 1];
  const int n = a.n, m = a.m;
  double* sP = smem;          // +2 a'_ij
  double* sM = smem + n * N;  // -2 a'_ij
  const double* A = static_cast<const double*>(a.A);
  for (int idx = threadIdx.x; idx < n * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    double v = 0.0;
    if (j < n) v = (i < m) ? A[i * a.rs + j * a.cs] : 1.0;
    sP[idx] = 2.0 * v;
    sM[idx] = -2.0 * v;
  }
  if (ABS) {
    // the rebuilt column sum errs by at most (n - 1) u sum_i |a'_ij| and each of the at
    // most 2^chunk_log2 - 1 later updates by u |S_j| <= u sum_i |a'_ij| (first order)
    const double steps = (double)n + ldexp(1.0, a.chunk_log2 < 62 ? a.chunk_log2 : 62);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      double colabs = 0.0;
      if (j < n)
        for (int i = 0; i < n; ++i) colabs += fabs((i < m) ? A[i * a.rs + j * a.cs] : 1.0);
      s_eps[j] = steps * 0x1p-53 * colabs * (1.0 + 0x1p-40);
    }
  }
  __syncthreads();

  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t g, len;
  split_range(a.g_begin, a.g_end, nt, tid, &g, &len);
  const uint64_t mask = (a.chunk_log2 >= 63) ? ~0ull : ((1ull << a.chunk_log2) - 1);

  double acc = 0.0, comp = 0.0, absacc = 0.0, diffacc = 0.0;
  double S[N];
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0 || (g & mask) == 0) {
      // exact rebuild: S_j = 1/2 * sum_i (delta_i * 2 a'_ij)
      const uint64_t gray = g ^ (g >> 1);
#pragma unroll
      for (int j = 0; j < N; ++j) S[j] = 0.0;
      for (int i = 0; i < n; ++i) {
        const double* row = (((gray >> (n - 1 - i)) & 1u) ? sM : sP) + i * N;
#pragma unroll
        for (int j = 0; j < N; ++j) S[j] = __dadd_rn(S[j], row[j]);
      }
#pragma unroll
      for (int j = 0; j < N; ++j) S[j] = (j < n) ? 0.5 * S[j] : 1.0;
    } else {
      const int b = ctz64(g);
      const double* row = (((g >> (b + 1)) & 1u) ? sP : sM) + (n - 1 - b) * N;
#pragma unroll
      for (int j = 0; j < N; ++j) S[j] = __dadd_rn(S[j], row[j]);
    }
    const double t = product_tree(S);
    const double st = __longlong_as_double(__double_as_longlong(t) ^ (long long)((g & 1ull) << 63));
    const double y = __dsub_rn(st, comp);
    const double sum = __dadd_rn(acc, y);
    comp = __dsub_rn(__dsub_rn(sum, acc), y);
    acc = sum;
    if (ABS) {
      absacc = __dadd_rn(absacc, fabs(t));
      // prod (|S_j| + eps_j) - |prod S_j| bounds the effect of the column sums' errors
      double pe = 1.0;
#pragma unroll
      for (int j = 0; j < N; ++j) pe = __dmul_rn(pe, __dadd_rn(fabs(S[j]), s_eps[j]));
      diffacc = __dadd_rn(diffacc, __dsub_rn(pe, fabs(t)));
    }
  }

  // records {sum, sum |term|, sum of the widened differences} (the last two with ABS)
  dd v[3] = {two_sum(acc, -comp), dd{absacc, 0.0}, dd{diffacc, 0.0}};
  block_sum_dd<3>(v, scratch);
  if (threadIdx.x == 0) {
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * (ABS ? kCplxRecord : kRealRecord);
    rec[0] = v[0].hi;
    rec[1] = v[0].lo;
    rec[2] = v[1].hi;
    rec[3] = v[1].lo;
    if (ABS) {
      rec[4] = v[2].hi;
      rec[5] = v[2].lo;
    }
  }
}

template <int N>
void* kernel_for(bool abs) {
  return abs ? (void*)glynn_f64_kernel<N, true> : (void*)glynn_f64_kernel<N, false>;
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

size_t smem_bytes(int n) { return 2u * (size_t)n * (size_t)((n + 3) & ~3) * sizeof(double); }

}  // namespace

int glynn_f64_blocks_per_sm(int n, int block, bool want_abs) {
  void* k = pick(n, want_abs);
  if (!k) return 0;
  size_t smem = smem_bytes(n);
  if (smem > 32 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_glynn_f64(const SweepArgs& a, const LaunchCfg& c, bool want_abs) {
  void* k = pick(a.n, want_abs);
  if (!k) return cudaErrorInvalidValue;
  size_t smem = smem_bytes(a.n);
  if (smem > 32 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  SweepArgs args = a;
  void* params[] = {&args};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), params, smem, c.stream);
}

}  // namespace perm
