// Multi-limb binary floating point for the Cauchy path (cauchy.cu).
//
// A value is (-1)^s * 0.m * 2^e: the mantissa m is L 64-bit limbs, m[0] the most
// significant, with the top bit of m[0] set unless the value is zero (z = 1); the
// exponent is a 32-bit integer, so values far outside the double range (the
// determinants of large Cauchy matrices) stay representable.  L is a run-time
// precision (2 <= L <= kBigLimbs); limbs at index >= L are ignored.
//
// Every operation truncates toward zero after working with at least one guard limb,
// so each result carries a relative error below 2^(2 - 64 L).  The functions are
// host-and-device so that the arithmetic can also run on the CPU.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

namespace perm {

constexpr int kBigLimbs = 16;            // 1024-bit mantissas at most
constexpr int kBigWords = kBigLimbs + 1; // stored value: header word + limbs

struct Big {
  uint64_t m[kBigLimbs];
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

__host__ __device__ inline void big_set_zero(Big& a, int L) {
  for (int i = 0; i < L; ++i) a.m[i] = 0;
  a.e = 0;
  a.s = 0;
  a.z = 1;
}

// Exact conversion of a finite double.
__host__ __device__ inline void big_from_double(Big& a, double v, int L) {
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
  uint64_t mant = bits & ((1ull << 52) - 1);
  if (ex == 0) {  // subnormal: mant * 2^-1074
    const int lz = big_clz(mant);
    a.m[0] = mant << lz;
    a.e = 64 - lz - 1074;
  } else {  // (2^52 + mant) * 2^(ex - 1075); the 53 bits at the top of m[0] weigh 2^-53 ..
    a.m[0] = (mant | (1ull << 52)) << 11;
    a.e = ex - 1022;
  }
}

// Round to the nearest double (ties to even); |a| beyond the double range gives +-inf or 0.
__host__ __device__ inline double big_to_double(const Big& a, int L) {
  if (a.z) return 0.0;
  uint64_t q = a.m[0] >> 11;
  const uint64_t rem = a.m[0] & 0x7ff;
  bool sticky = false;
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
__host__ __device__ inline int big_cmp_abs(const Big& a, const Big& b, int L) {
  if (a.z || b.z) return a.z && b.z ? 0 : (a.z ? -1 : 1);
  if (a.e != b.e) return a.e > b.e ? 1 : -1;
  for (int i = 0; i < L; ++i)
    if (a.m[i] != b.m[i]) return a.m[i] > b.m[i] ? 1 : -1;
  return 0;
}

// r = a * b.  Product scanning over the anti-diagonals i + j = t of limb pairs, from
// t = L down to 0, with a 192-bit column accumulator; pairs with i + j > L only reach
// below the guard limb and are left out.  r may alias a or b.
__host__ __device__ inline void big_mul(Big& r, const Big& a, const Big& b, int L) {
  if (a.z || b.z) {
    big_set_zero(r, L);
    return;
  }
  uint64_t p[kBigLimbs + 1];
  uint64_t c0 = 0, c1 = 0, c2 = 0;  // accumulator in units of limb t + 1
  for (int t = L; t >= 0; --t) {
    const int ilo = t - (L - 1) > 0 ? t - (L - 1) : 0;
    const int ihi = t < L - 1 ? t : L - 1;
    for (int i = ilo; i <= ihi; ++i) {
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
    for (int i = 0; i < L; ++i) p[i] = (p[i] << 1) | (p[i + 1] >> 63);
    --e;
  }
  for (int i = 0; i < L; ++i) r.m[i] = p[i];
  r.e = e;
  r.s = a.s ^ b.s;
  r.z = 0;
}

// r = a + b (negb = 0) or a - b (negb = 1), with two guard limbs.  r may alias a or b.
__host__ __device__ inline void big_add(Big& r, const Big& a, const Big& b, int negb, int L) {
  const int bs = b.s ^ negb;
  if (b.z) {
    if (&r != &a) r = a;
    return;
  }
  if (a.z) {
    if (&r != &b) r = b;
    r.s = bs;
    return;
  }
  const bool a_big = big_cmp_abs(a, b, L) >= 0;
  const Big& x = a_big ? a : b;
  const Big& y = a_big ? b : a;
  const int xs = a_big ? a.s : bs;
  const int ys = a_big ? bs : a.s;
  const int xe = x.e;
  const int d = x.e - y.e;  // >= 0
  const int W = L + 2;
  uint64_t S[kBigLimbs + 2];
  if (d >= 64 * W) {
    if (&r != &x) {
      for (int i = 0; i < L; ++i) r.m[i] = x.m[i];
      r.e = xe;
      r.z = 0;
    }
    r.s = xs;
    return;
  }
  const int q = d >> 6, sh = d & 63;
  uint64_t carry = 0;
  if (xs == ys) {
    for (int k = W - 1; k >= 0; --k) {
      const int src = k - q;
      uint64_t yk = (src >= 0 && src < L) ? (y.m[src] >> sh) : 0;
      if (sh && src - 1 >= 0 && src - 1 < L) yk |= y.m[src - 1] << (64 - sh);
      const uint64_t xk = k < L ? x.m[k] : 0;
      const uint64_t s1 = xk + yk;
      const uint64_t c1 = s1 < xk;
      const uint64_t s2 = s1 + carry;
      carry = c1 | (s2 < s1);
      S[k] = s2;
    }
    int e = xe;
    if (carry) {
      for (int k = W - 1; k > 0; --k) S[k] = (S[k] >> 1) | (S[k - 1] << 63);
      S[0] = (S[0] >> 1) | (1ull << 63);
      ++e;
    }
    for (int i = 0; i < L; ++i) r.m[i] = S[i];
    r.e = e;
  } else {
    for (int k = W - 1; k >= 0; --k) {
      const int src = k - q;
      uint64_t yk = (src >= 0 && src < L) ? (y.m[src] >> sh) : 0;
      if (sh && src - 1 >= 0 && src - 1 < L) yk |= y.m[src - 1] << (64 - sh);
      const uint64_t xk = k < L ? x.m[k] : 0;
      const uint64_t d1 = xk - yk;
      const uint64_t b1 = xk < yk;
      const uint64_t d2 = d1 - carry;
      carry = b1 | (d1 < carry);
      S[k] = d2;
    }
    int k0 = 0;
    while (k0 < W && S[k0] == 0) ++k0;
    if (k0 == W) {
      big_set_zero(r, L);
      return;
    }
    const int lz = big_clz(S[k0]);
    const int shift = 64 * k0 + lz;
    const int qq = shift >> 6, ss = shift & 63;
    for (int i = 0; i < L; ++i) {
      const int s0 = i + qq;
      uint64_t v = s0 < W ? (S[s0] << ss) : 0;
      if (ss && s0 + 1 < W) v |= S[s0 + 1] >> (64 - ss);
      r.m[i] = v;
    }
    r.e = xe - shift;
  }
  r.s = xs;
  r.z = 0;
}

// r = 1 / a (a != 0): a double reciprocal of the top 53 bits, then Newton steps
// x <- x + x (1 - a x), each doubling the correct bits, until they cover 64 L.
__host__ __device__ inline void big_recip(Big& r, const Big& a, int L) {
  const double top = (double)(a.m[0] >> 11) * 0x1p-53;  // in [1/2, 1)
  Big x, one, t;
  big_from_double(x, 1.0 / top, L);
  x.e -= a.e;
  x.s = a.s;
  big_from_double(one, 1.0, L);
  for (int bits = 50; bits < 64 * L + 8; bits *= 2) {
    big_mul(t, a, x, L);
    big_add(t, one, t, 1, L);
    big_mul(t, x, t, L);
    big_add(x, x, t, 0, L);
  }
  r = x;
}

// Stored form in device memory: word 0 = e (low 32 bits) | s << 32 | z << 33, words
// 1 .. L the limbs.
__host__ __device__ inline void big_store(uint64_t* p, const Big& a, int L) {
  p[0] = (uint64_t)(uint32_t)a.e | ((uint64_t)a.s << 32) | ((uint64_t)a.z << 33);
  for (int i = 0; i < L; ++i) p[1 + i] = a.m[i];
}

__host__ __device__ inline void big_load(Big& a, const uint64_t* p, int L) {
  const uint64_t h = p[0];
  a.e = (int)(uint32_t)h;
  a.s = (int)((h >> 32) & 1);
  a.z = (int)((h >> 33) & 1);
  for (int i = 0; i < L; ++i) a.m[i] = p[1 + i];
}

}  // namespace perm
