// Multi-limb binary floating point for the Cauchy path (cauchy.cu).
//
// A value is (-1)^s * 0.m * 2^e: the mantissa m is L 64-bit limbs, m[0] the most
// significant, with the top bit of m[0] set unless the value is zero (z = 1); the
// exponent is a 32-bit integer, so values far outside the double range (the
// determinants of large Cauchy matrices) stay representable.  L is a compile-time
// precision and every limb loop is unrolled, so a value lives in registers; shifts by
// a run-time number of limbs go through a barrel shifter (one conditional stage per
// bit of the count) instead of an indexed array, which would live in local memory.
//
// Every operation truncates toward zero after working with at least one guard limb,
// so each result carries a relative error below 2^(2 - 64 L).  The functions are
// host-and-device so that the arithmetic can also run on the CPU.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstring>

namespace perm {

constexpr int kBigLimbs = 16;  // longest precision: 1024-bit mantissas

template <int L>
struct Big {
  uint64_t m[L];
  int e;
  int s;
  int z;
};

__host__ __device__ __forceinline__ uint64_t big_mulhi(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

__host__ __device__ __forceinline__ int big_clz(uint64_t v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

template <int L>
__host__ __device__ __forceinline__ void big_set_zero(Big<L>& a) {
#pragma unroll
  for (int i = 0; i < L; ++i) a.m[i] = 0;
  a.e = 0;
  a.s = 0;
  a.z = 1;
}

// Exact conversion of a finite double.
template <int L>
__host__ __device__ __forceinline__ void big_from_double(Big<L>& a, double v) {
#pragma unroll
  for (int i = 0; i < L; ++i) a.m[i] = 0;
  if (v == 0.0) {
    a.e = 0;
    a.s = 0;
    a.z = 1;
    return;
  }
  a.s = v < 0.0;
  a.z = 0;
  const double av = ::fabs(v);
#ifdef __CUDA_ARCH__
  const uint64_t bits = (uint64_t)__double_as_longlong(av);
#else
  uint64_t bits;
  std::memcpy(&bits, &av, sizeof bits);
#endif
  const int ex = (int)(bits >> 52) & 0x7ff;
  const uint64_t mant = bits & ((1ull << 52) - 1);
  if (ex == 0) {  // subnormal: mant * 2^-1074
    const int lz = big_clz(mant);
    a.m[0] = mant << lz;
    a.e = 64 - lz - 1074;
  } else {  // (2^52 + mant) * 2^(ex - 1075), the 53 bits placed at the top of m[0]
    a.m[0] = (mant | (1ull << 52)) << 11;
    a.e = ex - 1022;
  }
}

// Round to the nearest double (ties to even); |a| beyond the double range gives +-inf or 0.
template <int L>
__host__ __device__ __forceinline__ double big_to_double(const Big<L>& a) {
  if (a.z) return 0.0;
  uint64_t q = a.m[0] >> 11;
  const uint64_t rem = a.m[0] & 0x7ff;
  bool sticky = false;
#pragma unroll
  for (int i = 1; i < L; ++i) sticky |= a.m[i] != 0;
  if (rem > 0x400 || (rem == 0x400 && (sticky || (q & 1)))) ++q;
  int e = a.e;
  if (q == (1ull << 53)) {
    q >>= 1;
    ++e;
  }
  const double r = ::ldexp((double)q, e - 53);
  return a.s ? -r : r;
}

// -1, 0, 1 as |a| <, ==, > |b|
template <int L>
__host__ __device__ __forceinline__ int big_cmp_abs(const Big<L>& a, const Big<L>& b) {
  if (a.z || b.z) return a.z && b.z ? 0 : (a.z ? -1 : 1);
  if (a.e != b.e) return a.e > b.e ? 1 : -1;
  int c = 0;
#pragma unroll
  for (int i = L - 1; i >= 0; --i)
    if (a.m[i] != b.m[i]) c = a.m[i] > b.m[i] ? 1 : -1;
  return c;
}

// r = a * b.  Product scanning over the anti-diagonals i + j = t of limb pairs, from
// t = L down to 0, with a 192-bit column accumulator; pairs with i + j > L only reach
// below the guard limb and are left out.  r may alias a or b.
template <int L>
__host__ __device__ __forceinline__ void big_mul(Big<L>& r, const Big<L>& a, const Big<L>& b) {
  const int z = a.z | b.z;
  uint64_t p[L + 1];
  uint64_t c0 = 0, c1 = 0, c2 = 0;  // accumulator in units of limb t + 1
#pragma unroll
  for (int t = L; t >= 0; --t) {
#pragma unroll
    for (int i = (t - (L - 1) > 0 ? t - (L - 1) : 0); i <= (t < L - 1 ? t : L - 1); ++i) {
      const uint64_t x = a.m[i], y = b.m[t - i];
      const uint64_t lo = x * y, hi = big_mulhi(x, y);
      c0 += lo;
      const uint64_t k0 = c0 < lo;
      c1 += k0;
      c2 += c1 < k0;
      c1 += hi;
      c2 += c1 < hi;
    }
    if (t + 1 <= L) p[t + 1] = c0;
    c0 = c1;
    c1 = c2;
    c2 = 0;
  }
  p[0] = c0;
  int e = a.e + b.e;
  if (!(p[0] >> 63)) {  // product of two mantissas in [1/2, 1) lies in [1/4, 1)
#pragma unroll
    for (int i = 0; i < L; ++i) p[i] = (p[i] << 1) | (p[i + 1] >> 63);
    --e;
  }
  const int s = a.s ^ b.s;
#pragma unroll
  for (int i = 0; i < L; ++i) r.m[i] = z ? 0 : p[i];
  r.e = z ? 0 : e;
  r.s = z ? 0 : s;
  r.z = z;
}

// r = a + b (negb = 0) or a - b (negb = 1), with two guard limbs.  r may alias a or b.
template <int L>
__host__ __device__ __forceinline__ void big_add(Big<L>& r, const Big<L>& a, const Big<L>& b, int negb) {
  constexpr int W = L + 2;
  const int bs = b.s ^ negb;
  if (b.z) {
    r = a;
    return;
  }
  if (a.z) {
    r = b;
    r.s = bs;
    return;
  }
  const bool a_big = big_cmp_abs(a, b) >= 0;
  uint64_t X[W], Y[W];
#pragma unroll
  for (int k = 0; k < W; ++k) {
    X[k] = k < L ? (a_big ? a.m[k] : b.m[k]) : 0;
    Y[k] = k < L ? (a_big ? b.m[k] : a.m[k]) : 0;
  }
  const int xs = a_big ? a.s : bs;
  const int ys = a_big ? bs : a.s;
  const int xe = a_big ? a.e : b.e;
  const int d = a_big ? a.e - b.e : b.e - a.e;  // >= 0
  if (d >= 64 * W) {
#pragma unroll
    for (int i = 0; i < L; ++i) r.m[i] = X[i];
    r.e = xe;
    r.s = xs;
    r.z = 0;
    return;
  }
  // Y >>= d bits: whole limbs through the barrel shifter, then the bits
  const int q = d >> 6, sh = d & 63;
#pragma unroll
  for (int b2 = 1; b2 < W; b2 <<= 1) {
    if (q & b2) {
#pragma unroll
      for (int k = W - 1; k >= 0; --k) Y[k] = k >= b2 ? Y[k - b2] : 0;
    }
  }
  if (sh) {
#pragma unroll
    for (int k = W - 1; k >= 0; --k) Y[k] = (Y[k] >> sh) | (k > 0 ? Y[k - 1] << (64 - sh) : 0);
  }
  uint64_t carry = 0;
  int e = xe;
  if (xs == ys) {
#pragma unroll
    for (int k = W - 1; k >= 0; --k) {
      const uint64_t s1 = X[k] + Y[k];
      const uint64_t c1 = s1 < X[k];
      const uint64_t s2 = s1 + carry;
      carry = c1 | (s2 < s1);
      X[k] = s2;
    }
    if (carry) {
#pragma unroll
      for (int k = W - 1; k > 0; --k) X[k] = (X[k] >> 1) | (X[k - 1] << 63);
      X[0] = (X[0] >> 1) | (1ull << 63);
      ++e;
    }
  } else {
#pragma unroll
    for (int k = W - 1; k >= 0; --k) {
      const uint64_t d1 = X[k] - Y[k];
      const uint64_t b1 = X[k] < Y[k];
      const uint64_t d2 = d1 - carry;
      carry = b1 | (d1 < carry);
      X[k] = d2;
    }
    int k0 = W;
#pragma unroll
    for (int k = W - 1; k >= 0; --k)
      if (X[k]) k0 = k;
    if (k0 == W) {
      big_set_zero(r);
      return;
    }
    // X <<= 64 k0 + clz bits: limbs through the barrel shifter, then the bits
#pragma unroll
    for (int b2 = 1; b2 < W; b2 <<= 1) {
      if (k0 & b2) {
#pragma unroll
        for (int k = 0; k < W; ++k) X[k] = k + b2 < W ? X[k + b2] : 0;
      }
    }
    const int lz = big_clz(X[0]);
    if (lz) {
#pragma unroll
      for (int k = 0; k < W; ++k) X[k] = (X[k] << lz) | (k + 1 < W ? X[k + 1] >> (64 - lz) : 0);
    }
    e -= 64 * k0 + lz;
  }
#pragma unroll
  for (int i = 0; i < L; ++i) r.m[i] = X[i];
  r.e = e;
  r.s = xs;
  r.z = 0;
}

// r = 1 / a (a != 0): a double-double reciprocal of the top 106 bits of the mantissa
// (one Newton step on the FP64 unit, about 2^-104 relative), then Newton steps
// x <- x + x (1 - a x) in L limbs, each doubling the correct bits, until they cover 64 L.
template <int L>
__host__ __device__ __forceinline__ void big_recip(Big<L>& r, const Big<L>& a) {
  const double h = (double)(a.m[0] >> 11) * 0x1p-53;  // in [1/2, 1)
  const uint64_t next = (a.m[0] << 53) | (L > 1 ? a.m[1] >> 11 : 0);
  const double l = (double)(next >> 11) * 0x1p-106;    // the following 53 bits
  const double x0 = 1.0 / h;
#ifdef __CUDA_ARCH__
  const double e = __dsub_rn(__fma_rn(-h, x0, 1.0), __dmul_rn(l, x0));  // 1 - (h + l) x0
  const double x1 = __dmul_rn(x0, e);
#else
  const double e = std::fma(-h, x0, 1.0) - l * x0;
  const double x1 = x0 * e;
#endif
  Big<L> x, t, one;
  big_from_double(x, x0);
  big_from_double(t, x1);
  big_add(x, x, t, 0);
  x.e -= a.e;
  x.s = a.s;
  big_from_double(one, 1.0);
#pragma unroll 1
  for (int bits = 100; bits < 64 * L + 8; bits *= 2) {
    big_mul(t, a, x);
    big_add(t, one, t, 1);
    big_mul(t, x, t);
    big_add(x, x, t, 0);
  }
  r = x;
}

// Stored form: word 0 = e (low 32 bits) | s << 32 | z << 33, words 1 .. L the limbs;
// word w of value `idx` at p[w * stride + idx] (structure of arrays, so that
// consecutive threads touching consecutive values read consecutive addresses).
template <int L>
__host__ __device__ __forceinline__ void big_store(uint64_t* p, size_t stride, size_t idx, const Big<L>& a) {
  p[idx] = (uint64_t)(uint32_t)a.e | ((uint64_t)a.s << 32) | ((uint64_t)a.z << 33);
#pragma unroll
  for (int i = 0; i < L; ++i) p[(size_t)(1 + i) * stride + idx] = a.m[i];
}

template <int L>
__host__ __device__ __forceinline__ void big_load(Big<L>& a, const uint64_t* p, size_t stride, size_t idx) {
  const uint64_t h = p[idx];
  a.e = (int)(uint32_t)h;
  a.s = (int)((h >> 32) & 1);
  a.z = (int)((h >> 33) & 1);
#pragma unroll
  for (int i = 0; i < L; ++i) a.m[i] = p[(size_t)(1 + i) * stride + idx];
}

}  // namespace perm
