// Rectangular Ryser (Eq. ryser_rectangle) by subset size, real input, FP64:
//     per(A) = sum_{s=1..m} (-1)^(m-s) C(n-s, m-s) sum_{|S|=s} prod_i sum_{j in S} a_ij.
// Only the subsets of size <= m are visited (sum_s C(n, s) of them, far fewer than
// 2^n when m << n).  The subsets of one size are taken in colex order: subset x (a
// bitmask) is followed by Gosper's successor, which swaps a few columns in and out,
// and the m row sums are updated for exactly those columns.  The global index runs
// over sizes 1..m in turn; a thread's slice starts at a rank that is unranked with
// the combinatorial number system (rank r of an s-subset c_s > ... > c_1 in colex
// order is sum_k C(c_k, k)).  Row sums are rebuilt exactly at the slice start, at
// each size change and every 2^chunk_log2 subsets.
#include "device_common.cuh"
#include "internal.h"

namespace perm {
namespace {

__device__ __forceinline__ uint64_t binom(int a, int b) {
  if (b < 0 || b > a) return 0;
  unsigned __int128 r = 1;
  for (int i = 1; i <= b; ++i) r = r * (unsigned __int128)(a - b + i) / (unsigned __int128)i;
  return (uint64_t)r;
}

// The s-subset of {0..n-1} of colex rank r, as a bitmask.
__device__ uint64_t colex_unrank(uint64_t r, int s, int n) {
  uint64_t x = 0;
  int hi = n - 1;
  for (int k = s; k >= 1; --k) {
    int c = hi;
    while (c >= k && binom(c, k) > r) --c;  // largest c with C(c, k) <= r
    r -= binom(c, k);
    x |= 1ull << c;
    hi = c - 1;
  }
  return x;
}

template <int M>
__global__ void __launch_bounds__(256) ryser_colex_kernel(SweepArgs a, SizeWeights weights, SizeCounts cum) {
  extern __shared__ double smem[];
  __shared__ dd scratch[2 * 32];
  const int n = a.n, m = a.m;
  double* sA = smem;  // sA[c * M + i] = a_ic
  const double* A = static_cast<const double*>(a.A);
  for (int idx = threadIdx.x; idx < n * M; idx += blockDim.x) {
    const int c = idx / M, i = idx - c * M;
    sA[idx] = (i < m) ? A[i * a.rs + c * a.cs] : 0.0;
  }
  __syncthreads();

  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t idx, len;
  split_range(a.g_begin, a.g_end, nt, tid, &idx, &len);
  const uint64_t mask = (a.chunk_log2 >= 63) ? ~0ull : ((1ull << a.chunk_log2) - 1);
  const uint64_t full = (n == 64) ? ~0ull : ((1ull << n) - 1);

  double acc = 0.0, comp = 0.0;
  double R[M];
  uint64_t x = 0;
  int s = 0;
  uint64_t since = 0;
  for (uint64_t t = 0; t < len; ++t, ++idx) {
    bool rebuild = false;
    if (t == 0) {
      s = 1;
      while (s < m && cum.c[s + 1] <= idx) ++s;
      x = colex_unrank(idx - cum.c[s], s, n);
      rebuild = true;
    } else {
      // Gosper's successor within size s; past the last s-subset, the first (s+1)-subset
      const uint64_t u = x & (~x + 1);
      const uint64_t v = x + u;
      uint64_t nx = v | ((((v ^ x) >> 2)) >> (__ffsll((long long)u) - 1));
      if (v == 0 || (nx & ~full) != 0) {
        ++s;
        nx = (s >= 64) ? ~0ull : ((1ull << s) - 1);
        x = nx;
        rebuild = true;
      } else if ((++since & mask) == 0) {
        x = nx;
        rebuild = true;
      } else {
        uint64_t rem = x & ~nx, add = nx & ~x;
        while (rem) {
          const int c = __ffsll((long long)rem) - 1;
          rem &= rem - 1;
#pragma unroll
          for (int i = 0; i < M; ++i) R[i] = __dsub_rn(R[i], sA[c * M + i]);
        }
        while (add) {
          const int c = __ffsll((long long)add) - 1;
          add &= add - 1;
#pragma unroll
          for (int i = 0; i < M; ++i) R[i] = __dadd_rn(R[i], sA[c * M + i]);
        }
        x = nx;
      }
    }
    if (rebuild) {
#pragma unroll
      for (int i = 0; i < M; ++i) R[i] = 0.0;
      uint64_t bits = x;
      while (bits) {
        const int c = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
#pragma unroll
        for (int i = 0; i < M; ++i) R[i] = __dadd_rn(R[i], sA[c * M + i]);
      }
#pragma unroll
      for (int i = 0; i < M; ++i)
        if (i >= m) R[i] = 1.0;
    }
    const double term = __dmul_rn(product_tree(R), weights.w[s]);
    const double y = __dsub_rn(term, comp);
    const double sum = __dadd_rn(acc, y);
    comp = __dsub_rn(__dsub_rn(sum, acc), y);
    acc = sum;
  }

  dd v[2] = {two_sum(acc, -comp), dd{0.0, 0.0}};
  block_sum_dd<2>(v, scratch);
  if (threadIdx.x == 0) {
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * kRealRecord;
    rec[0] = v[0].hi;
    rec[1] = v[0].lo;
    rec[2] = 0.0;
    rec[3] = 0.0;
  }
}

void* pick(int m) {
  switch ((m + 3) & ~3) {
    case 4: return (void*)ryser_colex_kernel<4>;
    case 8: return (void*)ryser_colex_kernel<8>;
    case 12: return (void*)ryser_colex_kernel<12>;
    case 16: return (void*)ryser_colex_kernel<16>;
    case 20: return (void*)ryser_colex_kernel<20>;
    case 24: return (void*)ryser_colex_kernel<24>;
    case 28: return (void*)ryser_colex_kernel<28>;
    case 32: return (void*)ryser_colex_kernel<32>;
    case 36: return (void*)ryser_colex_kernel<36>;
    case 40: return (void*)ryser_colex_kernel<40>;
    case 44: return (void*)ryser_colex_kernel<44>;
    case 48: return (void*)ryser_colex_kernel<48>;
    case 52: return (void*)ryser_colex_kernel<52>;
    case 56: return (void*)ryser_colex_kernel<56>;
    case 60: return (void*)ryser_colex_kernel<60>;
    case 64: return (void*)ryser_colex_kernel<64>;
    default: return nullptr;
  }
}

size_t smem_bytes(int m, int n) { return (size_t)n * (size_t)((m + 3) & ~3) * sizeof(double); }

}  // namespace

int ryser_colex_blocks_per_sm(int m, int n, int block) {
  void* k = pick(m);
  if (!k) return 0;
  size_t smem = smem_bytes(m, n);
  if (smem > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_ryser_colex(const SweepArgs& a, const SizeWeights& w, const SizeCounts& cum, const LaunchCfg& c) {
  void* k = pick(a.m);
  if (!k) return cudaErrorInvalidValue;
  size_t smem = smem_bytes(a.m, a.n);
  if (smem > 32 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  SweepArgs args = a;
  SizeWeights wv = w;
  SizeCounts cv = cum;
  void* params[] = {&args, &wv, &cv};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), params, smem, c.stream);
}

}  // namespace perm
