// Fixed-point helpers shared by the complex integer-pipe sweeps (glynn_cfx.cu,
// batched_fx.cu): normalisation of a complex software float whose two signed 64-bit
// components share one exponent, and signed 192-bit fixed-point accumulators.
#pragma once

#include "device_common.cuh"

namespace perm {

typedef unsigned long long u64;

__device__ __forceinline__ u64 uabs(long long v) { return v < 0 ? (u64)(-v) : (u64)v; }

// Shift count that brings max(|x|, |y|) into [2^61, 2^62) (0 if both are zero).
__device__ __forceinline__ int norm_shift(long long x, long long y) {
  const u64 mx = uabs(x) | uabs(y);  // same leading bit as the max
  return (__clzll((long long)mx) - 2) & 63;
}

__device__ __forceinline__ void add192(u64& a0, u64& a1, u64& a2, long long v, int p) {
  // a += v * 2^p for a signed 64-bit v (|v| < 2^62), p <= kMaxLsb
  const bool neg = v < 0;
  const u64 P = neg ? (u64)(-v) : (u64)v;
  u64 t0, t1, t2;
  if (p >= 64) {
    const int q = p - 64;
    t0 = 0;
    t1 = P << q;
    t2 = q ? (P >> (64 - q)) : 0;
  } else if (p >= 0) {
    t0 = P << p;
    t1 = p ? (P >> (64 - p)) : 0;
    t2 = 0;
  } else if (p > -64) {
    t0 = P >> (-p);
    t1 = 0;
    t2 = 0;
  } else {
    t0 = t1 = t2 = 0;
  }
  if (neg) {
    asm("sub.cc.u64 %0, %0, %3;\n\tsubc.cc.u64 %1, %1, %4;\n\tsubc.u64 %2, %2, %5;"
        : "+l"(a0), "+l"(a1), "+l"(a2)
        : "l"(t0), "l"(t1), "l"(t2));
  } else {
    asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
        : "+l"(a0), "+l"(a1), "+l"(a2)
        : "l"(t0), "l"(t1), "l"(t2));
  }
}

__device__ __forceinline__ void shr192(u64& a0, u64& a1, u64& a2, int s) {
  const u64 sgn = (u64)((long long)a2 >> 63);
  while (s >= 64) {
    a0 = a1;
    a1 = a2;
    a2 = sgn;
    s -= 64;
  }
  if (s > 0) {
    a0 = (a0 >> s) | (a1 << (64 - s));
    a1 = (a1 >> s) | (a2 << (64 - s));
    a2 = (u64)((long long)a2 >> s);
  }
}

__device__ __forceinline__ dd to_dd(u64 a0, u64 a1, u64 a2, int e_lo) {
  const bool negative = (long long)a2 < 0;
  if (negative) {
    asm("sub.cc.u64 %0, 0, %0;\n\tsubc.cc.u64 %1, 0, %1;\n\tsubc.u64 %2, 0, %2;" : "+l"(a0), "+l"(a1), "+l"(a2));
  }
  const u64 mask = (1ull << 48) - 1;
  dd r = dd{scalbn((double)(a2 >> 16), e_lo + 144), 0.0};
  r = dd_add(r, dd{scalbn((double)(((a1 >> 32) | (a2 << 32)) & mask), e_lo + 96), 0.0});
  r = dd_add(r, dd{scalbn((double)(((a0 >> 48) | (a1 << 16)) & mask), e_lo + 48), 0.0});
  r = dd_add(r, dd{scalbn((double)(a0 & mask), e_lo), 0.0});
  if (negative) {
    r.hi = -r.hi;
    r.lo = -r.lo;
  }
  return r;
}

// One step of the complex software-float product: (pr + i pi) 2^(E - 62) times the
// column sum (sr + i si) (already normalised by `l`).
__device__ __forceinline__ void cmul_step(long long& pr, long long& pi, int& E, long long sr, long long si, int l) {
  const long long re = __mul64hi(pr, sr) - __mul64hi(pi, si);
  const long long im = __mul64hi(pr, si) + __mul64hi(pi, sr);
  const int l2 = norm_shift(re, im);
  pr = re << l2;
  pi = im << l2;
  E += 64 - l - l2;
}

}  // namespace perm
