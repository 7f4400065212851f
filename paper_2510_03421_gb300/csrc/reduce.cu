// Final reductions: fixed-order sums of the per-block partials, then the
// normalisation of Eq. glynn_rectangle (division by 2^(n-1) and by (n-m)!) or of the
// Ryser formulas (none, pow2 = 0 and fact_of <= 1), and the optional a-posteriori
// error bound.  Floating-point partials are summed in double-double, integer
// partials modulo 2^128; both orders are fixed, so results are deterministic.
#include "device_common.cuh"
#include "internal.h"

namespace perm {
namespace {

typedef unsigned __int128 u128;

__global__ void finish_real_kernel(const double* rec, int nrec, int pow2, int fact_of, double err_coef, double* out,
                                   double* err, int raw, double sign) {
  __shared__ dd scratch[2 * 32];
  dd v[2] = {dd{0.0, 0.0}, dd{0.0, 0.0}};
  for (int r = threadIdx.x; r < nrec; r += blockDim.x) {
    v[0] = dd_add(v[0], dd{rec[kRealRecord * r], rec[kRealRecord * r + 1]});
    v[1] = dd_add(v[1], dd{rec[kRealRecord * r + 2], rec[kRealRecord * r + 3]});
  }
  block_sum_dd<2>(v, scratch);
  if (threadIdx.x != 0) return;
  v[0].hi *= sign;  // exact
  v[0].lo *= sign;
  if (raw) {
    out[0] = v[0].hi;
    out[1] = v[0].lo;
    if (err) err[0] = err_coef * v[1].hi;
    return;
  }
  dd s = dd_ldexp(v[0], -pow2);
  dd ab = dd_ldexp(v[1], -pow2);
  for (int k = 2; k <= fact_of; ++k) {
    s = dd_div_d(s, (double)k);
    ab = dd_div_d(ab, (double)k);
  }
  const double r = __dadd_rn(s.hi, s.lo);
  out[0] = r;
  if (err) err[0] = err_coef * ab.hi + fabs(__dsub_rn(r, s.hi) - s.lo);
}

__global__ void finish_cplx_kernel(const double* rec, int nrec, int pow2, int fact_of, double err_coef, double* out,
                                   double* err, int raw) {
  __shared__ dd scratch[3 * 32];
  dd v[3] = {dd{0.0, 0.0}, dd{0.0, 0.0}, dd{0.0, 0.0}};
  for (int r = threadIdx.x; r < nrec; r += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = dd_add(v[k], dd{rec[kCplxRecord * r + 2 * k], rec[kCplxRecord * r + 2 * k + 1]});
  }
  block_sum_dd<3>(v, scratch);
  if (threadIdx.x != 0) return;
  if (raw) {
    out[0] = v[0].hi;
    out[1] = v[0].lo;
    out[2] = v[1].hi;
    out[3] = v[1].lo;
    if (err) err[0] = err_coef * v[2].hi;
    return;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = dd_ldexp(v[k], -pow2);
  for (int f = 2; f <= fact_of; ++f)
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = dd_div_d(v[k], (double)f);
  const double re = __dadd_rn(v[0].hi, v[0].lo), im = __dadd_rn(v[1].hi, v[1].lo);
  out[0] = re;
  out[1] = im;
  if (err) err[0] = err_coef * v[2].hi + fabs(__dsub_rn(re, v[0].hi) - v[0].lo) + fabs(__dsub_rn(im, v[1].hi) - v[1].lo);
}

// Records {sum, G, Ge} of kCplxRecord doubles (sum |term| G, and Ge = sum of the
// products of (|S| + eta) when the rounding of A to fixed point was inexact, else 0):
// out = sum / (2^pow2 fact_of!) (raw: the unnormalised double-double); err = coef G,
// plus, when Ge != 0, (Ge - G) + coef (G + Ge) for the rounding of A and of the two
// bound sums themselves, plus the rounding of out.
//   diff_coef > 0: the third slot is instead the sum D of the per-term differences
//   (widened product - |term|) formed in FP64, and err = coef G + D (1 + 2^-25) +
//   diff_coef (G + D) (the two FP64 products behind each difference).
__global__ void finish_bound_kernel(const double* rec, int nrec, int pow2, int fact_of, double coef, double* out,
                                    double* err, int raw, double diff_coef) {
  __shared__ dd scratch[3 * 32];
  dd v[3] = {dd{0.0, 0.0}, dd{0.0, 0.0}, dd{0.0, 0.0}};
  for (int r = threadIdx.x; r < nrec; r += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = dd_add(v[k], dd{rec[kCplxRecord * r + 2 * k], rec[kCplxRecord * r + 2 * k + 1]});
  }
  block_sum_dd<3>(v, scratch);
  if (threadIdx.x != 0) return;
  if (!raw) {
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = dd_ldexp(v[k], -pow2);
    for (int f = 2; f <= fact_of; ++f)
#pragma unroll
      for (int k = 0; k < 3; ++k) v[k] = dd_div_d(v[k], (double)f);
  }
  const double G = v[1].hi, Ge = v[2].hi;
  double e = coef * G;
  if (diff_coef > 0.0) {
    const double D = fmax(Ge, 0.0);
    e += D * (1.0 + 0x1p-25) + diff_coef * (G + D);
  } else if (Ge != 0.0) {
    e += fmax(__dsub_rn(Ge, G), 0.0) * (1.0 + 0x1p-50) + coef * (G + Ge);
  }
  if (raw) {
    out[0] = v[0].hi;
    out[1] = v[0].lo;
    if (err) err[0] = e;
    return;
  }
  const double r = __dadd_rn(v[0].hi, v[0].lo);
  out[0] = r;
  if (err) err[0] = e + fabs(__dsub_rn(r, v[0].hi) - v[0].lo);
}

__global__ void finish_int_kernel(const unsigned long long* rec, int nrec, int pow2, int fact_of,
                                  unsigned long long* out, int raw) {
  __shared__ u128 part[256];
  u128 acc = 0;
  for (int r = threadIdx.x; r < nrec; r += blockDim.x)
    acc += ((u128)rec[kIntRecord * r + 1] << 64) | (u128)rec[kIntRecord * r];
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x != 0) return;
  u128 total = 0;
  for (int t = 0; t < (int)blockDim.x; ++t) total += part[t];
  if (!raw) {
    __int128 v = (__int128)total;
    v >>= pow2;  // exact: the sum is a multiple of 2^(n-1) whenever it did not wrap
    __int128 f = 1;
    for (int k = 2; k <= fact_of; ++k) f *= k;
    v /= f;
    total = (u128)v;
  }
  out[0] = (unsigned long long)total;
  out[1] = (unsigned long long)(total >> 64);
}

__global__ void write_double_kernel(double v, double* p) { p[0] = v; }

__global__ void write_one_kernel(int dtype, void* out) {
  if (dtype == 0) {
    static_cast<double*>(out)[0] = 1.0;
  } else if (dtype == 1) {
    static_cast<double*>(out)[0] = 1.0;
    static_cast<double*>(out)[1] = 0.0;
  } else {
    static_cast<unsigned long long*>(out)[0] = 1ull;
    static_cast<unsigned long long*>(out)[1] = 0ull;
    if (dtype == 4) {  // Gaussian integers: imaginary part 0
      static_cast<unsigned long long*>(out)[2] = 0ull;
      static_cast<unsigned long long*>(out)[3] = 0ull;
    }
  }
}

// Product of `count` block permanents (each a double or a (re, im) pair at slot k,
// 16 bytes apart) in double-double, or the zero of the dtype when count == 0.
__global__ void block_product_kernel(int dtype, const double* slots, int count, void* out) {
  double* o = static_cast<double*>(out);
  if (count == 0) {
    o[0] = 0.0;
    if (dtype == 1) o[1] = 0.0;
    return;
  }
  if (dtype == 0) {
    dd p{slots[0], 0.0};
    for (int k = 1; k < count; ++k) p = dd_mul_d(p, slots[2 * k]);
    o[0] = __dadd_rn(p.hi, p.lo);
    return;
  }
  dd pr{slots[0], 0.0}, pi{slots[1], 0.0};
  for (int k = 1; k < count; ++k) {
    const double br = slots[2 * k], bi = slots[2 * k + 1];
    const dd nr = dd_add(dd_mul_d(pr, br), dd_mul_d(pi, -bi));
    const dd ni = dd_add(dd_mul_d(pr, bi), dd_mul_d(pi, br));
    pr = nr;
    pi = ni;
  }
  o[0] = __dadd_rn(pr.hi, pr.lo);
  o[1] = __dadd_rn(pi.hi, pi.lo);
}

}  // namespace

cudaError_t launch_block_product(int dtype, const double* slots, int count, void* out, cudaStream_t s) {
  block_product_kernel<<<1, 1, 0, s>>>(dtype, slots, count, out);
  return cudaGetLastError();
}

cudaError_t launch_finish_real(const double* rec, int nrec, int pow2, int fact_of, double err_coef, double* out,
                               double* err, bool raw, cudaStream_t s, double sign) {
  finish_real_kernel<<<1, 256, 0, s>>>(rec, nrec, pow2, fact_of, err_coef, out, err, raw ? 1 : 0, sign);
  return cudaGetLastError();
}

cudaError_t launch_finish_cplx(const double* rec, int nrec, int pow2, int fact_of, double err_coef, double* out,
                               double* err, bool raw, cudaStream_t s) {
  finish_cplx_kernel<<<1, 256, 0, s>>>(rec, nrec, pow2, fact_of, err_coef, out, err, raw ? 1 : 0);
  return cudaGetLastError();
}

__global__ void negate_records_kernel(double* rec, int nrec, int stride) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += gridDim.x * blockDim.x) {
    rec[(size_t)r * stride] = -rec[(size_t)r * stride];
    rec[(size_t)r * stride + 1] = -rec[(size_t)r * stride + 1];
  }
}

cudaError_t launch_negate_records(double* rec, int nrec, int stride, cudaStream_t s) {
  negate_records_kernel<<<(nrec + 255) / 256, 256, 0, s>>>(rec, nrec, stride);
  return cudaGetLastError();
}

cudaError_t launch_finish_bound(const double* rec, int nrec, int pow2, int fact_of, double coef, double* out,
                                double* err, bool raw, cudaStream_t s, double diff_coef) {
  finish_bound_kernel<<<1, 256, 0, s>>>(rec, nrec, pow2, fact_of, coef, out, err, raw ? 1 : 0, diff_coef);
  return cudaGetLastError();
}

cudaError_t launch_finish_int(const unsigned long long* rec, int nrec, int pow2, int fact_of, unsigned long long* out,
                              bool raw, cudaStream_t s) {
  finish_int_kernel<<<1, 256, 0, s>>>(rec, nrec, pow2, fact_of, out, raw ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_write_double(double v, double* p, cudaStream_t s) {
  write_double_kernel<<<1, 1, 0, s>>>(v, p);
  return cudaGetLastError();
}

cudaError_t launch_write_one(int dtype, void* out, cudaStream_t s) {
  write_one_kernel<<<1, 1, 0, s>>>(dtype, out);
  return cudaGetLastError();
}

}  // namespace perm
