// Fixed-point helpers shared by the integer-pipe sweeps (glynn_fx.cu, glynn_fxg.cu,
// glynn_cfx.cu): the real software-float product of column sums, the normalisation of
// a complex software float whose two signed 64-bit components share one exponent,
// and signed 192-bit fixed-point accumulators.
#pragma once

#include "device_common.cuh"

namespace perm {

typedef unsigned long long u64;

constexpr int kAnchorBit = 120;  // leading bit of a thread's first term in its accumulator
constexpr int kMaxLsb = 87;      // a term's lsb may sit at most here (leading bit <= 150)

// Full 64 x 64 -> 128-bit unsigned product as one carry chain of 32-bit multiply-adds.
__device__ __forceinline__ void mul_wide(u64 a, u64 b, u64& lo, u64& hi) {
  asm("{\n\t.reg .u32 a0, a1, b0, b1, r0, r1, r2, r3;\n\t"
      "mov.b64 {a0, a1}, %2;\n\t"
      "mov.b64 {b0, b1}, %3;\n\t"
      "mul.lo.u32 r0, a0, b0;\n\t"
      "mul.hi.u32 r1, a0, b0;\n\t"
      "mad.lo.cc.u32 r1, a0, b1, r1;\n\t"
      "madc.hi.u32 r2, a0, b1, 0;\n\t"
      "mad.lo.cc.u32 r1, a1, b0, r1;\n\t"
      "madc.hi.cc.u32 r2, a1, b0, r2;\n\t"
      "madc.hi.u32 r3, a1, b1, 0;\n\t"
      "mad.lo.cc.u32 r2, a1, b1, r2;\n\t"
      "addc.u32 r3, r3, 0;\n\t"
      "mov.b64 %0, {r0, r1};\n\t"
      "mov.b64 %1, {r2, r3};\n\t}"
      : "=l"(lo), "=l"(hi)
      : "l"(a), "l"(b));
}

// value = sign * P * 2^(E - 63) * 2^(-e_sum); P == 0 iff some factor is zero.
// Columns [0, N - K) are taken in pairs: the product of two column sums (each at
// most 2^61 in magnitude) is formed exactly in 128 bits and its leading 64 bits mc
// (normalised, value mc 2^(64 - lz)) are multiplied into P with the high half of a
// 64x64-bit product: P mc 2^(E - 63 + 64 - lz) = h2 2^(E + 65 - lz), so P = h2 and
// E += 128 - lz.  h2 >= P / 2, so P is renormalised (clz) only every fourth pair and
// after the last one.  Columns [N - K, N) are multiplied on the FP64 unit and the
// double product is folded in once (its exponent field ed: value md 2^(ed - 1086)).
// EXACT: magnitudes by two's complement (one more instruction per column), for the
// variants that state an error bound; otherwise one's complement (below).
template <int N, int K, bool EXACT = false>
__device__ __forceinline__ void soft_product(const long long (&S)[N], u64& P, int& E, unsigned& neg) {
  static_assert((N - K) % 2 == 0, "integer columns are taken in pairs");
  P = 1ull << 63;  // the value 1
  E = 0;
  neg = 0;
#pragma unroll
  for (int j = 0; j < N - K; j += 2) {
    const long long qa = S[j], qb = S[j + 1];
    const u64 sa = (u64)(qa >> 63), sb = (u64)(qb >> 63);
    neg ^= (unsigned)(sa ^ sb);
    // magnitudes by one's complement: |q| or |q| - 1, an error of one unit in a value
    // of up to 2^61 (relative 2^-58 or less for all but vanishing column sums)
    const u64 aa = EXACT ? ((u64)qa ^ sa) - sa : (u64)qa ^ sa, ab = EXACT ? ((u64)qb ^ sb) - sb : (u64)qb ^ sb;
    u64 lo, hi;
    mul_wide(aa, ab, lo, hi);
    // hi < 2^59, so lz >= 5; a pair product below 2^64 (vanishing column sums) keeps
    // the bits of lo that fit, the value stays exact
    const int lz = __clzll((long long)(hi | 1ull));
    const u64 mc = (hi << lz) | (lo >> (64 - lz));
    P = __umul64hi(P, mc);
    E += 128 - lz;
    if ((j / 2) % 4 == 3 || j + 2 >= N - K) {
      const int l = __clzll((long long)(P | 1ull));  // P == 0 stays 0
      P <<= l;
      E -= l;
    }
  }
  if (K > 0) {
    double d[K > 0 ? K : 1];
#pragma unroll
    for (int k = 0; k < K; ++k) d[k] = (double)S[N - K + k];  // exact below 2^53, else rounded once
#pragma unroll
    for (int w = 1; w < K; w *= 2)
#pragma unroll
      for (int k = 0; k + w < K; k += 2 * w) d[k] = __dmul_rn(d[k], d[k + w]);
    // |d| < 2^(61 K) <= 2^976 (K <= 16) and |d| >= 1 unless some factor is 0: no overflow,
    // no subnormals, and ed == 0 exactly when the product is zero
    const u64 bits = (u64)__double_as_longlong(d[0]);
    neg ^= (unsigned)(bits >> 63);
    const int ed = (int)((bits >> 52) & 0x7ff);
    const u64 md = (bits << 11) | (1ull << 63);
    const u64 h2 = __umul64hi(P, md);
    const int top = (int)(h2 >> 63);
    P = ed ? (top ? h2 : (h2 << 1)) : 0ull;
    E += ed - 1023 + top;
  }
  neg &= 1u;
}

// Product of (|S_j| + eta) over the first `nreal` sums (the others taken as they are),
// computed in place with S restored afterwards: when every sum may be off by eta units
// (the rounding of A to fixed point), |prod S_true - prod S| <= prod (|S| + eta) - prod |S|.
template <int N, int K>
__device__ __forceinline__ void soft_product_eta(long long (&S)[N], int nreal, long long eta, u64& P, int& E) {
  u64 sg = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (j < nreal) {
      if (S[j] < 0) {
        sg |= 1ull << j;
        S[j] = -S[j];
      }
      S[j] += eta;
    }
  }
  unsigned ng;
  soft_product<N, K, true>(S, P, E, ng);
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (j < nreal) {
      S[j] -= eta;
      if ((sg >> j) & 1u) S[j] = -S[j];
    }
  }
}

// acc += (-1)^neg * P * 2^p (p = position of P's lsb in the accumulator, p <= 127)
__device__ __forceinline__ void acc_add(u64& a0, u64& a1, u64& a2, u64 P, int p, unsigned neg) {
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

// acc += (-1)^neg * P * 2^p for 0 <= p <= 127 without branches: the lanes of a warp add
// terms of different signs and positions at the same step, so a branch on either
// diverges.  The three shifted words are chosen by masks; the sign enters as the
// two's complement ~t + 1, with the + 1 as the carry into the lowest word (set by
// adding the all-ones mask to itself).
__device__ __forceinline__ void acc_add_nb(u64& a0, u64& a1, u64& a2, u64 P, int p, unsigned neg) {
  const int s = p & 63;
  const u64 lo = P << s;
  const u64 hi = (P >> 1) >> (63 - s);  // P >> (64 - s), and 0 for s = 0
  const u64 up = (u64)0 - (u64)(p >> 6);  // all ones when p >= 64
  const u64 m = (u64)0 - (u64)(neg & 1u);
  const u64 t0 = (lo & ~up) ^ m;
  const u64 t1 = ((hi & ~up) | (lo & up)) ^ m;
  const u64 t2 = (hi & up) ^ m;
  asm("{\n\t.reg .u64 c;\n\t"
      "add.cc.u64 c, %3, %3;\n\t"
      "addc.cc.u64 %0, %0, %4;\n\t"
      "addc.cc.u64 %1, %1, %5;\n\t"
      "addc.u64 %2, %2, %6;\n\t}"
      : "+l"(a0), "+l"(a1), "+l"(a2)
      : "l"(m), "l"(t0), "l"(t1), "l"(t2));
}

// u64 binomial coefficient C(a, b), a <= 63 (exact: every partial product is a
// binomial coefficient times b, below 2^70, kept in 128 bits).
__device__ __forceinline__ u64 binom_u64(int a, int b) {
  unsigned __int128 r = 1;
  for (int i = 1; i <= b; ++i) r = r * (unsigned __int128)(a - b + i) / (unsigned __int128)i;
  return (u64)r;
}

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

// Fold a complex double d = dr + i di (the FP64 part of a mixed product) into the
// complex software float (pr + i pi) 2^(E - 62): both components are put on the
// larger one's exponent as signed integers of at most 53 bits (the smaller loses the
// bits below that exponent's ulp), normalised, and multiplied in as one factor.
__device__ __forceinline__ void cfold_double(long long& pr, long long& pi, int& E, double dr, double di) {
  const u64 br = (u64)__double_as_longlong(dr), bi = (u64)__double_as_longlong(di);
  const int er = (int)((br >> 52) & 0x7ff), ei = (int)((bi >> 52) & 0x7ff);
  const int em = er > ei ? er : ei;
  if (em == 0) {  // the FP64 factor is zero (its columns are integers: no subnormals)
    pr = 0;
    pi = 0;
    return;
  }
  // value of component c: (2^52 + frac) 2^(e - 1075) for a normal e; 0 when e == 0
  const long long mr0 = er ? (long long)((br & ((1ull << 52) - 1)) | (1ull << 52)) : 0;
  const long long mi0 = ei ? (long long)((bi & ((1ull << 52) - 1)) | (1ull << 52)) : 0;
  const int shr = em - er, shi = em - ei;
  long long mr = shr >= 63 ? 0 : (mr0 >> shr), mi = shi >= 63 ? 0 : (mi0 >> shi);
  if (br >> 63) mr = -mr;
  if (bi >> 63) mi = -mi;
  // the factor is (mr + i mi) 2^(em - 1075); normalise it like a column sum
  const int l = norm_shift(mr, mi);
  const long long sr = mr << l, si = mi << l;
  const long long re = __mul64hi(pr, sr) - __mul64hi(pi, si);
  const long long im = __mul64hi(pr, si) + __mul64hi(pi, sr);
  const int l2 = norm_shift(re, im);
  pr = re << l2;
  pi = im << l2;
  // (pr + i pi) 2^(E-62) (sr + i si) 2^(em-1075-l) = (re + i im) 2^(E+2+em-1075-l), and
  // pr' = re << l2 makes the exponent of pr' 2^(E'-62): E' = E + em - 1011 - l - l2
  E += em - 1011 - l - l2;
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
