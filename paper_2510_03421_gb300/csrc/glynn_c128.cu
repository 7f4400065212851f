// Glynn's formula (Eq. glynn, Eq. glynn_rectangle) for complex input, FP64
// arithmetic.  Same Gray-code walk as the real kernel (glynn_f64.cu): each thread
// owns a contiguous slice of the 2^(n-1) terms, rebuilds its column sums exactly at
// the start of the slice and at every multiple of 2^chunk_log2, and otherwise moves
// every column sum by +-2 a'_rj when row r flips.  Complex products use two FMAs
// per component; real and imaginary parts are summed in separate Kahan pairs.
#include "device_common.cuh"
#include "internal.h"

namespace perm {
namespace {

struct cd {
  double re, im;
};

__device__ __forceinline__ cd cmul(cd a, cd b) {
  return {__fma_rn(a.re, b.re, -__dmul_rn(a.im, b.im)), __fma_rn(a.re, b.im, __dmul_rn(a.im, b.re))};
}

template <int N>
__device__ __forceinline__ cd cproduct_tree(const double (&Sr)[N], const double (&Si)[N]) {
  constexpr int H = (N + 1) / 2;
  cd p[H];
#pragma unroll
  for (int j = 0; j < H; ++j)
    p[j] = (2 * j + 1 < N) ? cmul(cd{Sr[2 * j], Si[2 * j]}, cd{Sr[2 * j + 1], Si[2 * j + 1]}) : cd{Sr[2 * j], Si[2 * j]};
#pragma unroll
  for (int w = 1; w < H; w *= 2)
#pragma unroll
    for (int j = 0; j + w < H; j += 2 * w) p[j] = cmul(p[j], p[j + w]);
  return p[0];
}

template <int N, bool ABS>
__global__ void __launch_bounds__(128) glynn_c128_kernel(SweepArgs a) {
  extern __shared__ double smem[];
  __shared__ dd scratch[3 * 32];
  __shared__ double s_eps[ABS ? N : 1];
  const int n = a.n, m = a.m;
  // interleaved (re, im) pairs: +2 a'_ij then -2 a'_ij
  double2* sP = reinterpret_cast<double2*>(smem);
  double2* sM = sP + n * N;
  const double* A = static_cast<const double*>(a.A);  // (re, im) pairs, 8-byte aligned
  for (int idx = threadIdx.x; idx < n * N; idx += blockDim.x) {
    const int i = idx / N, j = idx - i * N;
    double2 v = make_double2(0.0, 0.0);
    if (j < n) {
      const int64_t e = 2 * (i * a.rs + j * a.cs);
      v = (i < m) ? make_double2(A[e], A[e + 1]) : make_double2(1.0, 0.0);
    }
    sP[idx] = make_double2(2.0 * v.x, 2.0 * v.y);
    sM[idx] = make_double2(-2.0 * v.x, -2.0 * v.y);
  }
  if (ABS) {
    // modulus of a column sum's error: the rebuild ((n - 1) u) and the at most
    // 2^chunk_log2 - 1 later updates (u each), per component, against
    // sum_i |re a'_ij| + |im a'_ij| (first order)
    const double steps = (double)n + ldexp(1.0, a.chunk_log2 < 62 ? a.chunk_log2 : 62);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      double colabs = 0.0;
      if (j < n)
        for (int i = 0; i < n; ++i) {
          const int64_t e = 2 * (i * a.rs + j * a.cs);
          colabs += (i < m) ? fabs(A[e]) + fabs(A[e + 1]) : 1.0;
        }
      s_eps[j] = steps * 0x1p-53 * colabs * (1.0 + 0x1p-40);
    }
  }
  // per term of the bound variant: the products' rounding (3n + 6) u and the FP64
  // evaluation of the widened product 2 (n + 1) u, against |re t| + |im t|
  const double cr = ldexp(3.0 * n + 6.0 + 2.0 * (n + 1.0), -53);
  __syncthreads();

  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t g, len;
  split_range(a.g_begin, a.g_end, nt, tid, &g, &len);
  const uint64_t mask = (a.chunk_log2 >= 63) ? ~0ull : ((1ull << a.chunk_log2) - 1);

  double accr = 0.0, compr = 0.0, acci = 0.0, compi = 0.0, absacc = 0.0;
  double Sr[N], Si[N];
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0 || (g & mask) == 0) {
      const uint64_t gray = g ^ (g >> 1);
#pragma unroll
      for (int j = 0; j < N; ++j) Sr[j] = Si[j] = 0.0;
      for (int i = 0; i < n; ++i) {
        const double2* row = (((gray >> (n - 1 - i)) & 1u) ? sM : sP) + i * N;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const double2 v = row[j];
          Sr[j] = __dadd_rn(Sr[j], v.x);
          Si[j] = __dadd_rn(Si[j], v.y);
        }
      }
#pragma unroll
      for (int j = 0; j < N; ++j) {
        Sr[j] = (j < n) ? 0.5 * Sr[j] : 1.0;
        Si[j] = (j < n) ? 0.5 * Si[j] : 0.0;
      }
    } else {
      const int b = ctz64(g);
      const double2* row = (((g >> (b + 1)) & 1u) ? sP : sM) + (n - 1 - b) * N;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const double2 v = row[j];
        Sr[j] = __dadd_rn(Sr[j], v.x);
        Si[j] = __dadd_rn(Si[j], v.y);
      }
    }
    cd t = cproduct_tree(Sr, Si);
    const long long flip = (long long)((g & 1ull) << 63);
    const double tr = __longlong_as_double(__double_as_longlong(t.re) ^ flip);
    const double ti = __longlong_as_double(__double_as_longlong(t.im) ^ flip);
    double y = __dsub_rn(tr, compr), sum = __dadd_rn(accr, y);
    compr = __dsub_rn(__dsub_rn(sum, accr), y);
    accr = sum;
    y = __dsub_rn(ti, compi);
    sum = __dadd_rn(acci, y);
    compi = __dsub_rn(__dsub_rn(sum, acci), y);
    acci = sum;
    if (ABS) {
      // bound of this term's error: cr |t|_1 plus prod (|S_j|_1 + eps_j) - prod |S_j|_1,
      // which bounds the effect of the column sums' errors (|.|_1 >= the modulus, and
      // the widened difference grows with the sums it is formed from)
      const double t1 = __dadd_rn(fabs(t.re), fabs(t.im));
      double pe = 1.0, pa = 1.0;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const double sa = __dadd_rn(fabs(Sr[j]), fabs(Si[j]));
        pe = __dmul_rn(pe, __dadd_rn(sa, s_eps[j]));
        pa = __dmul_rn(pa, sa);
      }
      const double d = fmax(__dsub_rn(pe, pa), 0.0);
      absacc = __dadd_rn(absacc, __fma_rn(cr, fmax(t1, pa) + d, d * (1.0 + 0x1p-25)));
    }
  }

  dd v[3] = {two_sum(accr, -compr), two_sum(acci, -compi), dd{absacc, 0.0}};
  block_sum_dd<3>(v, scratch);
  if (threadIdx.x == 0) {
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * kCplxRecord;
    rec[0] = v[0].hi;
    rec[1] = v[0].lo;
    rec[2] = v[1].hi;
    rec[3] = v[1].lo;
    rec[4] = v[2].hi;
    rec[5] = v[2].lo;
  }
}

template <int N>
void* kernel_for(bool abs) {
  return abs ? (void*)glynn_c128_kernel<N, true> : (void*)glynn_c128_kernel<N, false>;
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

size_t smem_bytes(int n) { return 2u * (size_t)n * (size_t)((n + 3) & ~3) * 2 * sizeof(double); }

}  // namespace

int glynn_c128_max_n() { return 48; }

int glynn_c128_blocks_per_sm(int n, int block, bool want_abs) {
  void* k = pick(n, want_abs);
  if (!k) return 0;
  size_t smem = smem_bytes(n);
  if (smem > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_glynn_c128(const SweepArgs& a, const LaunchCfg& c, bool want_abs) {
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
