// Glynn's formula (Eq. glynn, Eq. glynn_rectangle), real input, FP64, with the
// column sums at the chunk starts formed on the FP64 tensor cores.
//
// The term range is cut into chunks aligned to multiples of L = 2^chunk_log2.  A
// warp takes 32 consecutive chunks at a time (one per lane).  Their 32 starting
// sign vectors form a +-1 matrix Delta (32 x n, row l = delta(gray(start of chunk l)));
// the 32 starting column-sum vectors are the contraction S = Delta A' (32 x n),
// computed with mma.sync.m8n8k4 in FP64 (4 row tiles of 8 chunks, n/4 k-steps, N/8
// column tiles).  Each lane then receives its row of S by shuffles and walks its chunk
// with the incremental +-2 a'_rj updates of glynn_f64.cu.  All lanes of a warp walk
// chunks of the same length, so the warp stays converged.
//
// mma.m8n8k4 f64 fragments (one double of A and of B, two of C per lane):
//   A (8 x 4, row major): row = lane / 4, col = lane % 4
//   B (4 x 8, col major): row = lane % 4, col = lane / 4
//   C (8 x 8):            row = lane / 4, cols 2 (lane % 4) and 2 (lane % 4) + 1
#include "device_common.cuh"
#include "internal.h"

namespace perm {
namespace {

__device__ __forceinline__ void dmma(double& c0, double& c1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c0), "+d"(c1)
               : "d"(a), "d"(b));
}

template <int N, bool ABS>
__global__ void __launch_bounds__(256) glynn_dmma_kernel(SweepArgs a) {
  constexpr int NT = (N + 7) / 8;  // column tiles
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
    // a contracted column sum errs by at most (n - 1) u sum_i |a'_ij| (n exact +-a
    // products summed), each of the at most 2^chunk_log2 - 1 later updates by
    // u sum_i |a'_ij| (first order), as in glynn_f64.cu
    const double steps = (double)n + ldexp(1.0, a.chunk_log2 < 62 ? a.chunk_log2 : 62);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      double colabs = 0.0;
      if (j < n)
        for (int i = 0; i < n; ++i) colabs += fabs((i < m) ? A[i * a.rs + j * a.cs] : 1.0);
      s_eps[j] = steps * 0x1p-53 * colabs * (1.0 + 0x1p-40);
    }
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const uint64_t L = 1ull << a.chunk_log2;
  const uint64_t c_first = a.g_begin >> a.chunk_log2;
  const uint64_t c_end = (a.g_end + L - 1) >> a.chunk_log2;  // one past the last chunk
  const uint64_t rounds = (c_end - c_first + 31) / 32;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);

  double acc = 0.0, comp = 0.0, absacc = 0.0, diffacc = 0.0;
  double S[N];
  for (uint64_t r = warp; r < rounds; r += warps) {
    const uint64_t chunk = c_first + 32 * r + lane;
    uint64_t ga = chunk << a.chunk_log2, gb = ga + L;
    if (ga < a.g_begin) ga = a.g_begin;
    if (gb > a.g_end) gb = a.g_end;
    if (chunk >= c_end) ga = gb = a.g_end;  // idle lane
    const uint64_t gray = ga ^ (ga >> 1);

    // S (32 x N) = Delta (32 x n) * A' (n x N), one 8-row tile at a time
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
      const uint64_t gr = __shfl_sync(0xffffffffu, gray, mt * 8 + (lane >> 2));
      double c[NT][2];
#pragma unroll
      for (int t = 0; t < NT; ++t) c[t][0] = c[t][1] = 0.0;
      for (int kt = 0; kt < (n + 3) / 4; ++kt) {
        const int i = kt * 4 + (lane & 3);
        const double av = (i < n) ? (((gr >> (n - 1 - i)) & 1u) ? -1.0 : 1.0) : 0.0;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const int j = t * 8 + (lane >> 2);
          const double bv = (i < n && j < N) ? 0.5 * sP[i * N + j] : 0.0;
          dmma(c[t][0], c[t][1], av, bv);
        }
      }
      // lane l (l / 8 == mt) takes row l % 8 of the tile: element (row, col) sits in
      // lane 4 row + (col % 8) / 2, register col % 2
#pragma unroll
      for (int t = 0; t < NT; ++t)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int col = t * 8 + 2 * q + h;
            const double v = __shfl_sync(0xffffffffu, c[t][h], (lane & 7) * 4 + q);
            if (col < N && (lane >> 3) == mt) S[col] = v;
          }
    }
#pragma unroll
    for (int j = 0; j < N; ++j)
      if (j >= n) S[j] = 1.0;

    // walk the chunk
    for (uint64_t g = ga; g < gb; ++g) {
      if (g != ga) {
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
        double pe = 1.0;  // prod (|S_j| + eps_j): the column sums' own errors
#pragma unroll
        for (int j = 0; j < N; ++j) pe = __dmul_rn(pe, __dadd_rn(fabs(S[j]), s_eps[j]));
        diffacc = __dadd_rn(diffacc, __dsub_rn(pe, fabs(t)));
      }
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
  return abs ? (void*)glynn_dmma_kernel<N, true> : (void*)glynn_dmma_kernel<N, false>;
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
    default: return nullptr;
  }
}

size_t smem_bytes(int n) { return 2u * (size_t)n * (size_t)((n + 3) & ~3) * sizeof(double); }

}  // namespace

int glynn_dmma_max_n() { return 48; }

int glynn_dmma_blocks_per_sm(int n, int block, bool want_abs) {
  void* k = pick(n, want_abs);
  if (!k) return 0;
  size_t smem = smem_bytes(n);
  if (smem > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_glynn_dmma(const SweepArgs& a, const LaunchCfg& c, bool want_abs) {
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
