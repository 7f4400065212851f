// Ryser's inclusion-exclusion formula, real input, FP64 arithmetic.
//
// Written for an m x n matrix (m <= n) in the subset-size form of Eq. ryser_rectangle:
//     per(A) = sum_{S subset of columns, |S| <= m} (-1)^(m-|S|) C(n-|S|, m-|S|) prod_i R_i(S),
//     R_i(S) = sum_{j in S} a_ij,
// which for m = n is Eq. ryser_square (all weights +-1).  The 2^n column subsets are
// visited in reflected Gray-code order: subset(g) = set bits of gray(g) = g ^ (g >> 1)
// (bit c <-> column c); step g adds or removes column c = ctz(g), so each of the m
// row sums moves by +-a_ic.  Each thread walks a contiguous slice of g, rebuilding
// its row sums exactly at the slice start and at every multiple of 2^chunk_log2.
// For m = n the sign of a term is (-1)^(n-|S|) = (-1)^n (-1)^g; for m < n the weight
// (sign included) is read from a table indexed by |S|, which the walk tracks.
#include "device_common.cuh"
#include "internal.h"

namespace perm {
namespace {


template <int M, bool WEIGHTED, bool ABS>
__global__ void __launch_bounds__(256) ryser_f64_kernel(SweepArgs a, SizeWeights weights) {
  extern __shared__ double smem[];
  __shared__ dd scratch[3 * 32];
  __shared__ double w[65];
  __shared__ double s_eps[ABS ? M : 1];
  const int n = a.n, m = a.m;
  double* sP = smem;          // sP[c * M + i] = +a_ic
  double* sM = smem + n * M;  // -a_ic
  const double* A = static_cast<const double*>(a.A);
  for (int idx = threadIdx.x; idx < n * M; idx += blockDim.x) {
    const int c = idx / M, i = idx - c * M;
    const double v = (i < m) ? A[i * a.rs + c * a.cs] : 0.0;
    sP[idx] = v;
    sM[idx] = -v;
  }
  if (WEIGHTED)
    for (int s = threadIdx.x; s <= n; s += blockDim.x) w[s] = weights.w[s];
  if (ABS) {
    // a rebuilt row sum errs by at most (n - 1) u sum_j |a_ij|, each of the at most
    // 2^chunk_log2 - 1 later updates by u sum_j |a_ij| (first order)
    const double steps = (double)n + ldexp(1.0, a.chunk_log2 < 62 ? a.chunk_log2 : 62);
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      double rowabs = 0.0;
      if (i < m)
        for (int c = 0; c < n; ++c) rowabs += fabs(A[i * a.rs + c * a.cs]);
      s_eps[i] = steps * 0x1p-53 * rowabs * (1.0 + 0x1p-40);
    }
  }
  __syncthreads();

  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t g, len;
  split_range(a.g_begin, a.g_end, nt, tid, &g, &len);
  const uint64_t mask = (a.chunk_log2 >= 63) ? ~0ull : ((1ull << a.chunk_log2) - 1);

  double acc = 0.0, comp = 0.0, absacc = 0.0, diffacc = 0.0;
  double R[M];
  int size = 0;
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0 || (g & mask) == 0) {
      const uint64_t gray = g ^ (g >> 1);
      size = __popcll(gray);
#pragma unroll
      for (int i = 0; i < M; ++i) R[i] = 0.0;
      for (int c = 0; c < n; ++c) {
        if (!((gray >> c) & 1u)) continue;
        const double* col = sP + c * M;
#pragma unroll
        for (int i = 0; i < M; ++i) R[i] = __dadd_rn(R[i], col[i]);
      }
#pragma unroll
      for (int i = 0; i < M; ++i) R[i] = (i < m) ? R[i] : 1.0;
    } else {
      const int c = ctz64(g);
      const bool added = !((g >> (c + 1)) & 1u);
      size += added ? 1 : -1;
      const double* col = (added ? sP : sM) + c * M;
#pragma unroll
      for (int i = 0; i < M; ++i) R[i] = __dadd_rn(R[i], col[i]);
    }
    double t = product_tree(R);
    if (WEIGHTED) {
      t = __dmul_rn(t, w[size]);
    } else {
      t = __longlong_as_double(__double_as_longlong(t) ^ (long long)((g & 1ull) << 63));
    }
    const double y = __dsub_rn(t, comp);
    const double sum = __dadd_rn(acc, y);
    comp = __dsub_rn(__dsub_rn(sum, acc), y);
    acc = sum;
    if (ABS) {
      absacc = __dadd_rn(absacc, fabs(t));
      // |weight| (prod (|R_i| + eps_i) - prod |R_i|): the row sums' own errors
      double pe = 1.0, pa = 1.0;
#pragma unroll
      for (int i = 0; i < M; ++i) {
        pe = __dmul_rn(pe, __dadd_rn(fabs(R[i]), s_eps[i]));
        pa = __dmul_rn(pa, fabs(R[i]));
      }
      const double aw = WEIGHTED ? fabs(w[size]) : 1.0;
      diffacc = __dadd_rn(diffacc, __dmul_rn(aw, __dsub_rn(pe, pa)));
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

template <int M>
void* kernel_for(bool weighted, bool abs) {
  if (weighted) return abs ? (void*)ryser_f64_kernel<M, true, true> : (void*)ryser_f64_kernel<M, true, false>;
  return abs ? (void*)ryser_f64_kernel<M, false, true> : (void*)ryser_f64_kernel<M, false, false>;
}

void* pick(int m, bool weighted, bool abs) {
  switch ((m + 3) & ~3) {
    case 4: return kernel_for<4>(weighted, abs);
    case 8: return kernel_for<8>(weighted, abs);
    case 12: return kernel_for<12>(weighted, abs);
    case 16: return kernel_for<16>(weighted, abs);
    case 20: return kernel_for<20>(weighted, abs);
    case 24: return kernel_for<24>(weighted, abs);
    case 28: return kernel_for<28>(weighted, abs);
    case 32: return kernel_for<32>(weighted, abs);
    case 36: return kernel_for<36>(weighted, abs);
    case 40: return kernel_for<40>(weighted, abs);
    case 44: return kernel_for<44>(weighted, abs);
    case 48: return kernel_for<48>(weighted, abs);
    case 52: return kernel_for<52>(weighted, abs);
    case 56: return kernel_for<56>(weighted, abs);
    case 60: return kernel_for<60>(weighted, abs);
    case 64: return kernel_for<64>(weighted, abs);
    default: return nullptr;
  }
}

size_t smem_bytes(int m, int n) { return 2u * (size_t)n * (size_t)((m + 3) & ~3) * sizeof(double); }

}  // namespace

int ryser_f64_blocks_per_sm(int m, int n, int block, bool weighted, bool want_abs) {
  void* k = pick(m, weighted, want_abs);
  if (!k) return 0;
  size_t smem = smem_bytes(m, n);
  if (smem > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_ryser_f64(const SweepArgs& a, const SizeWeights& weights, const LaunchCfg& c, bool want_abs) {
  const bool weighted = a.m < a.n;
  void* k = pick(a.m, weighted, want_abs);
  if (!k) return cudaErrorInvalidValue;
  size_t smem = smem_bytes(a.m, a.n);
  if (smem > 32 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  SweepArgs args = a;
  SizeWeights wt = weights;
  void* params[] = {&args, &wt};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), params, smem, c.stream);
}

}  // namespace perm
