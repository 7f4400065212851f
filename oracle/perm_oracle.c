/*
 * perm_oracle.c -- plain, slow, serial CPU oracle for the permanent of an m x n
 * matrix (real, complex or integer), written from the paper's definitions and
 * algorithms (Eq. permanent_definition, Eq. rectangular_permanent_definition,
 * Eq. ryser_rectangle, Eq. ryser_square, Eq. glynn, Eq. glynn_rectangle and the
 * four base algorithms of the appendix).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA library, and the CUDA library never calls it.
 *
 * Precisions:
 *   *_ld   long double (80-bit extended on x86-64, IEEE binary128 on aarch64;
 *          oracle_ldbl_mant_dig() reports which) -- the reference precision.
 *   *_f64  the same code in double -- only used as the timed CPU baseline.
 *   *_i128 exact integer arithmetic in wrapping unsigned 128-bit integers; the
 *          result is exact whenever the unnormalised sum fits in a signed
 *          128-bit integer (wrap-around is exact modulo 2^128).
 *
 * Every function requires 0 <= m <= n <= 64 (n <= 28 for the subset DP; the full
 * sums are only practical for small n, the partial sums take any n); the
 * Python wrapper applies per(A) = per(A^T) for m > n and per(0 x n) = 1.
 *
 * Functions: the definition, Glynn (square and rectangular, the appendix
 * algorithms), Glynn with the padding rows of ones grouped by their number of -1
 * signs (Eq. glynn_rectangle, same terms), square and rectangular Ryser, the
 * exact subset DP, and partial sums over ranges of Glynn / Ryser terms.
 *
 * Parity pins (tests/test_oracle_*.py): the worked 3x3 example of the usage
 * section, per(J_n) = n!, all-ones m x n = n!/(n-m)!, padded identity = 1,
 * derangement numbers, Fibonacci numbers for tridiagonal ones, triangular
 * matrices, rank-one closed form, Cauchy/Borchardt in exact rationals, row/column
 * permutation, transpose, multilinearity, Laplace expansion, perfect-matching
 * counts by brute force, and the focus-pointer flip sequence.
 */
#include <complex.h>
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

int oracle_ldbl_mant_dig(void) { return LDBL_MANT_DIG; }

/* One step of the focus-pointer generator of the Glynn algorithms: given the
 * pointer array and the current pos (the row that was just flipped is
 * bound - pos), return the next pos.  The statements are those of the
 * "generate next permutation" block of Algorithm "Glynn's Algorithm for
 * Square Matrices". */
static int focus_pointer_next(int* perm, int pos) {
  perm[0] = 0;
  perm[pos] = perm[pos + 1];
  pos = pos + 1;
  perm[pos] = pos;
  return perm[0];
}

/* The sequence of rows flipped by the focus-pointer generator for an n x n
 * matrix: flips[t] = bound - pos at step t, t = 0 .. 2^(n-1) - 2. */
int oracle_glynn_flips(int n, int* flips, int64_t capacity) {
  int perm[64];
  for (int i = 0; i < n; ++i) perm[i] = i;
  int bound = n - 1, pos = 0;
  int64_t t = 0;
  while (pos != bound) {
    if (t < capacity) flips[t] = bound - pos;
    ++t;
    pos = focus_pointer_next(perm, pos);
  }
  return (int)t;
}

/* C(a, b) by the multiplicative formula; exact for the sizes used here. */
static uint64_t binomial_u64(int a, int b) {
  if (b < 0 || b > a) return 0;
  u128 r = 1;
  for (int i = 1; i <= b; ++i) r = r * (u128)(a - b + i) / (u128)i;
  return (uint64_t)r;
}

/* Advance comb[0..s-1] (strictly increasing, values in 0..n-1) to the next
 * combination in lexicographic order; returns 0 after the last one. */
static int next_combination(int* comb, int s, int n) {
  int i = s - 1;
  while (i >= 0 && comb[i] == n - s + i) --i;
  if (i < 0) return 0;
  comb[i] += 1;
  for (int t = i + 1; t < s; ++t) comb[t] = comb[t - 1] + 1;
  return 1;
}

#define REAL long double
#define SFX(name) name##_ld
#define SQRT_REAL sqrtl
#include "oracle_real.inc"
#undef REAL
#undef SFX
#undef SQRT_REAL

#define REAL double
#define SFX(name) name##_f64
#define SQRT_REAL sqrt
#include "oracle_real.inc"
#undef REAL
#undef SFX
#undef SQRT_REAL

/* ===========================================================================
 * Exact integer versions.  Input: int64 entries, row-major with ld.  Output:
 * a two's-complement 128-bit integer written as out[0] = low 64 bits,
 * out[1] = high 64 bits.
 * ========================================================================= */
static void put_i128(u128 x, uint64_t* out) {
  out[0] = (uint64_t)x;
  out[1] = (uint64_t)(x >> 64);
}

static void def_rec_i(int m, int n, const int64_t* A, int64_t ld, int i, int* sigma, int* used, u128* acc) {
  if (i == m) {
    u128 p = 1;
    for (int r = 0; r < m; ++r) p *= (u128)(i128)A[r * ld + sigma[r]];
    *acc += p;
    return;
  }
  for (int j = 0; j < n; ++j) {
    if (used[j]) continue;
    used[j] = 1;
    sigma[i] = j;
    def_rec_i(m, n, A, ld, i + 1, sigma, used, acc);
    used[j] = 0;
  }
}

/* Definition (Eq. rectangular_permanent_definition) in wrapping 128-bit. */
void oracle_definition_i128(int m, int n, const int64_t* A, int64_t ld, uint64_t* out) {
  int sigma[64], used[64] = {0};
  u128 acc = 0;
  def_rec_i(m, n, A, ld, 0, sigma, used, &acc);
  put_i128(acc, out);
}

static u128 glynn_term_i(int m, int n, const int64_t* A, int64_t ld, const int* delta) {
  u128 prod = 1;
  for (int j = 0; j < n; ++j) {
    i128 sum = 0;
    for (int i = 0; i < m; ++i) sum += (i128)A[i * ld + j] * delta[i];
    for (int k = m; k < n; ++k) sum += delta[k];
    prod *= (u128)sum;
  }
  return prod;
}

/* Glynn (Algorithms "Glynn's Algorithm for Square / Rectangular Matrices") in
 * wrapping 128-bit integers, then the exact division by 2^(n-1) (n-m)!. */
void oracle_glynn_i128(int m, int n, const int64_t* A, int64_t ld, uint64_t* out) {
  int delta[64] = {0}, perm[64] = {0};
  for (int i = 0; i < n; ++i) { delta[i] = 1; perm[i] = i; }
  u128 acc = glynn_term_i(m, n, A, ld, delta);
  int bound = n - 1, pos = 0, sign = 1;
  while (pos != bound) {
    sign = -sign;
    delta[bound - pos] = -delta[bound - pos];
    u128 t = glynn_term_i(m, n, A, ld, delta);
    if (sign < 0) acc -= t; else acc += t;
    pos = focus_pointer_next(perm, pos);
  }
  i128 v = (i128)acc;
  i128 norm = (i128)1 << bound;
  for (int i = 2; i <= n - m; ++i) norm *= i;
  put_i128((u128)(v / norm), out);
}

/* ---------------------------------------------------------------------------
 * Gaussian integers (complex entries with int64 real and imaginary parts, stored
 * as interleaved pairs, ld counted in complex elements): the same two algorithms
 * with every product and sum taken componentwise in wrapping 128-bit integers.
 * Output: out[0..1] = real part, out[2..3] = imaginary part (low, high words).
 * ------------------------------------------------------------------------- */
typedef struct {
  u128 re, im;
} ci128;

static ci128 ci_mul(ci128 a, ci128 b) {
  ci128 r;
  r.re = a.re * b.re - a.im * b.im;
  r.im = a.re * b.im + a.im * b.re;
  return r;
}

static void def_rec_ci(int m, int n, const int64_t* A, int64_t ld, int i, int* sigma, int* used, ci128* acc) {
  if (i == m) {
    ci128 p = {1, 0};
    for (int r = 0; r < m; ++r) {
      const int64_t* e = A + 2 * (r * ld + sigma[r]);
      ci128 a = {(u128)(i128)e[0], (u128)(i128)e[1]};
      p = ci_mul(p, a);
    }
    acc->re += p.re;
    acc->im += p.im;
    return;
  }
  for (int j = 0; j < n; ++j) {
    if (used[j]) continue;
    used[j] = 1;
    sigma[i] = j;
    def_rec_ci(m, n, A, ld, i + 1, sigma, used, acc);
    used[j] = 0;
  }
}

void oracle_definition_ci128(int m, int n, const int64_t* A, int64_t ld, uint64_t* out) {
  int sigma[64], used[64] = {0};
  ci128 acc = {0, 0};
  def_rec_ci(m, n, A, ld, 0, sigma, used, &acc);
  put_i128(acc.re, out);
  put_i128(acc.im, out + 2);
}

static ci128 glynn_term_ci(int m, int n, const int64_t* A, int64_t ld, const int* delta) {
  ci128 prod = {1, 0};
  for (int j = 0; j < n; ++j) {
    i128 sr = 0, si = 0;
    for (int i = 0; i < m; ++i) {
      sr += (i128)A[2 * (i * ld + j)] * delta[i];
      si += (i128)A[2 * (i * ld + j) + 1] * delta[i];
    }
    for (int k = m; k < n; ++k) sr += delta[k];
    ci128 s = {(u128)sr, (u128)si};
    prod = ci_mul(prod, s);
  }
  return prod;
}

void oracle_glynn_ci128(int m, int n, const int64_t* A, int64_t ld, uint64_t* out) {
  int delta[64] = {0}, perm[64] = {0};
  for (int i = 0; i < n; ++i) { delta[i] = 1; perm[i] = i; }
  ci128 acc = glynn_term_ci(m, n, A, ld, delta);
  int bound = n - 1, pos = 0, sign = 1;
  while (pos != bound) {
    sign = -sign;
    delta[bound - pos] = -delta[bound - pos];
    ci128 t = glynn_term_ci(m, n, A, ld, delta);
    if (sign < 0) {
      acc.re -= t.re;
      acc.im -= t.im;
    } else {
      acc.re += t.re;
      acc.im += t.im;
    }
    pos = focus_pointer_next(perm, pos);
  }
  i128 norm = (i128)1 << bound;
  for (int i = 2; i <= n - m; ++i) norm *= i;
  put_i128((u128)((i128)acc.re / norm), out);
  put_i128((u128)((i128)acc.im / norm), out + 2);
}

void oracle_glynn_partial_ci128(int m, int n, const int64_t* A, int64_t ld, uint64_t g0, uint64_t g1,
                                uint64_t* out) {
  int delta[64] = {0};
  ci128 acc = {0, 0};
  for (uint64_t g = g0; g < g1; ++g) {
    uint64_t gray = g ^ (g >> 1);
    for (int i = 0; i < n; ++i) delta[i] = ((gray >> (n - 1 - i)) & 1u) ? -1 : 1;
    ci128 t = glynn_term_ci(m, n, A, ld, delta);
    if (g & 1u) {
      acc.re -= t.re;
      acc.im -= t.im;
    } else {
      acc.re += t.re;
      acc.im += t.im;
    }
  }
  put_i128(acc.re, out);
  put_i128(acc.im, out + 2);
}

/* Unnormalised Glynn partial sum over terms g0 <= g < g1 (same term indexing as
 * oracle_glynn_partial_ld), modulo 2^128. */
void oracle_glynn_partial_i128(int m, int n, const int64_t* A, int64_t ld, uint64_t g0, uint64_t g1, uint64_t* out) {
  int delta[64] = {0};
  u128 acc = 0;
  for (uint64_t g = g0; g < g1; ++g) {
    uint64_t gray = g ^ (g >> 1);
    for (int i = 0; i < n; ++i) delta[i] = ((gray >> (n - 1 - i)) & 1u) ? -1 : 1;
    u128 t = glynn_term_i(m, n, A, ld, delta);
    if (g & 1u) acc -= t; else acc += t;
  }
  put_i128(acc, out);
}

/* Ryser, square (Algorithm "Ryser's Algorithm for Square Matrices"), exact. */
void oracle_ryser_square_i128(int m, const int64_t* A, int64_t ld, uint64_t* out) {
  u128 acc = 0;
  uint64_t c = (uint64_t)1 << m;
  for (uint64_t k = 0; k < c; ++k) {
    u128 rowsumprod = 1;
    for (int i = 0; i < m; ++i) {
      i128 rowsum = 0;
      for (int j = 0; j < m; ++j)
        if (k & ((uint64_t)1 << j)) rowsum += A[i * ld + j];
      rowsumprod *= (u128)rowsum;
    }
    if (__builtin_popcountll(k) & 1) acc -= rowsumprod; else acc += rowsumprod;
  }
  if (m & 1) acc = (u128)0 - acc;
  put_i128(acc, out);
}

/* Ryser, rectangular (Algorithm "Ryser's Algorithm for Rectangular Matrices"), exact. */
void oracle_ryser_rect_i128(int m, int n, const int64_t* A, int64_t ld, uint64_t* out) {
  u128 acc = 0;
  int sign = 1, comb[64];
  for (int k = 0; k < m; ++k) {
    int s = m - k;
    u128 bin = binomial_u64(n - m + k, k);
    u128 permsum = 0;
    for (int t = 0; t < s; ++t) comb[t] = t;
    do {
      u128 colprod = 1;
      for (int i = 0; i < m; ++i) {
        i128 matsum = 0;
        for (int j = 0; j < s; ++j) matsum += A[i * ld + comb[j]];
        colprod *= (u128)matsum;
      }
      if (sign < 0) permsum -= colprod * bin; else permsum += colprod * bin;
    } while (next_combination(comb, s, n));
    acc += permsum;
    sign = -sign;
  }
  put_i128(acc, out);
}

/* Exact permanent by dynamic programming over column subsets: f(S) for a set S
 * of |S| = r columns is the permanent of rows 0..r-1 restricted to the columns S,
 * f(empty) = 1 and f(S) = sum_{j in S} a_{r-1, j} f(S minus j) (expansion along
 * the last row); per(A) = sum over |S| = m of f(S).  A textbook algorithm that
 * is independent of Glynn and Ryser, used to pin them on integer matrices.
 * Returns -1 if n > 28 or the table cannot be allocated. */
int oracle_subset_dp_i128(int m, int n, const int64_t* A, int64_t ld, uint64_t* out) {
  if (n > 28) return -1;
  uint64_t size = (uint64_t)1 << n;
  u128* f = (u128*)calloc(size, sizeof(u128));
  if (!f) return -1;
  f[0] = 1;
  u128 total = (m == 0) ? 1 : 0;
  for (uint64_t S = 1; S < size; ++S) {
    int r = __builtin_popcountll(S);
    if (r > m) continue;
    u128 v = 0;
    for (int j = 0; j < n; ++j)
      if (S & ((uint64_t)1 << j)) v += (u128)(i128)A[(r - 1) * ld + j] * f[S & ~((uint64_t)1 << j)];
    f[S] = v;
    if (r == m) total += v;
  }
  free(f);
  put_i128(total, out);
  return 0;
}
