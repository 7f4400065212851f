// The a-priori range check of the exact integer sums (glynn_int.cu, batched_int.cu).
//
// The Glynn and Ryser sums are 2^(n-1) (n-m)! per(A); they are exact modulo 2^128, so
// the result is exact whenever that value fits a signed int128.  From the row
// statistics of |A| (|re| + |im| for Gaussian integers):
//   lrow  = sum_i log2(r_i), r_i = sum_j |a_ij|          (per(|A|) <= prod_i r_i)
//   lbreg = sum_i log2(r_i!) / r_i                        (Bregman's bound, 0/1 entries)
// and the n - m padding rows of ones (row sum n, Bregman factor (n!)^(1/n)).
#pragma once

namespace perm {

constexpr double kInt128Bits = 126.5;  // margin below 2^127 for the bound's own rounding

// log2 of the bound on |2^(n-1) (n-m)! per(A)|
__host__ __device__ inline double glynn_sum_log2_bound(int m, int n, double lrow, double lbreg, bool binary) {
  const double ln2 = 0.69314718055994530942;
  const double lfact = lgamma((double)(n - m) + 1.0) / ln2;
  double lb = (double)(n - 1) + lfact + lrow;
  if (binary) {
    const double lpad = (double)(n - m) * lgamma((double)n + 1.0) / ln2 / (double)n;
    const double lb2 = (double)(n - 1) + lbreg + lpad;
    if (lb2 < lb) lb = lb2;
  }
  return lb;
}

// one row's contribution to lbreg
__host__ __device__ inline double bregman_log2_term(double rsum) {
  return lgamma(rsum + 1.0) / 0.69314718055994530942 / rsum;
}

// the +-2 a_ij column-sum updates need |column sum| + (n - m) below 2^61
__host__ __device__ inline bool column_sum_overflows(double csum, int m, int n) {
  return csum + (double)(n - m) > 2.0e18;
}

}  // namespace perm
