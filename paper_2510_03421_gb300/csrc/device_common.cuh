// Device helpers shared by the permanent kernels: double-double arithmetic,
// Gray-code bookkeeping and block reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace perm {

// ---------------------------------------------------------------- double-double
// A value hi + lo with |lo| <= ulp(hi)/2.  Error-free transformations after
// Knuth (TwoSum) and Dekker (FastTwoSum); products use the FMA form of TwoProd.
struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ dd fast_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double e = __dsub_rn(b, __dsub_rn(s, a));
  return {s, e};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo = __dadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __dadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}

// (hi + lo) * d for a double d (TwoProd by FMA), about 2^-104 relative error.
__device__ __forceinline__ dd dd_mul_d(dd a, double d) {
  const double p = __dmul_rn(a.hi, d);
  const double e = __fma_rn(a.hi, d, -p);
  return fast_two_sum(p, __fma_rn(a.lo, d, e));
}

// (hi + lo) * 2^e, exact barring under/overflow.
__device__ __forceinline__ dd dd_ldexp(dd a, int e) { return {scalbn(a.hi, e), scalbn(a.lo, e)}; }

// (hi + lo) / d for a double d, about 2^-104 relative error.
__device__ __forceinline__ dd dd_div_d(dd a, double d) {
  double q1 = a.hi / d;
  double r = __fma_rn(-q1, d, a.hi);
  r = __dadd_rn(r, a.lo);
  double q2 = r / d;
  return fast_two_sum(q1, q2);
}

__device__ __forceinline__ dd shfl_down_dd(dd v, int off) {
  return {__shfl_down_sync(0xffffffffu, v.hi, off), __shfl_down_sync(0xffffffffu, v.lo, off)};
}

// Deterministic block-wide double-double sum of K values per thread (fixed tree
// order).  `scratch` holds at least K * blockDim.x / 32 dd.  Thread 0 gets the result.
template <int K>
__device__ __forceinline__ void block_sum_dd(dd (&v)[K], dd* scratch) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = dd_add(v[k], shfl_down_dd(v[k], off));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) scratch[k * nw + warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      dd x = (lane < nw) ? scratch[k * nw + lane] : dd{0.0, 0.0};
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x = dd_add(x, shfl_down_dd(x, off));
      v[k] = x;
    }
  }
}

// ---------------------------------------------------------------- products
// prod_j x_j as a balanced tree of FP64 multiplications (N - 1 of them).
template <int N>
__device__ __forceinline__ double product_tree(const double (&x)[N]) {
  constexpr int H = (N + 1) / 2;
  double p[H];
#pragma unroll
  for (int j = 0; j < H; ++j) p[j] = (2 * j + 1 < N) ? __dmul_rn(x[2 * j], x[2 * j + 1]) : x[2 * j];
#pragma unroll
  for (int w = 1; w < H; w *= 2)
#pragma unroll
    for (int j = 0; j + w < H; j += 2 * w) p[j] = __dmul_rn(p[j], p[j + w]);
  return p[0];
}

// ---------------------------------------------------------------- work split
// Split [g_begin, g_end) into `parts` nearly equal contiguous ranges; range `t`
// is [*lo, *lo + *len).
__device__ __forceinline__ void split_range(uint64_t g_begin, uint64_t g_end, uint64_t parts, uint64_t t,
                                            uint64_t* lo, uint64_t* len) {
  uint64_t total = g_end - g_begin;
  uint64_t base = total / parts, rem = total % parts;
  *lo = g_begin + t * base + (t < rem ? t : rem);
  *len = base + (t < rem ? 1u : 0u);
}

// Index of the lowest set bit of g (g != 0).
__device__ __forceinline__ int ctz64(uint64_t g) { return __ffsll((long long)g) - 1; }

}  // namespace perm
