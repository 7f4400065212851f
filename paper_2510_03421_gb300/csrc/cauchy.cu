// Permanents of Cauchy matrices c_ij = 1 / (x_i - y_j) by Borchardt's theorem
// (Eq. caucy_permanent): per(C) = det(C o C) / det(C).
//
// det(C) has Cauchy's closed form prod_{i<j} (x_j - x_i)(y_i - y_j) / prod_{i,j} (x_i - y_j),
// a product with no cancellation.  det(C o C) has none: it is taken by Gaussian
// elimination with partial pivoting, and C o C is so ill-conditioned that double
// precision loses every digit from n ~ 12 on (the elimination loses roughly 7 to 9
// bits per unit of n).  Both are therefore evaluated in the multi-limb floating point
// of bigfloat.cuh, with a precision ladder: the permanent is computed at L0 limbs and
// at L0 + 1, then L0 + 3, L0 + 7, ... (at most kBigLimbs), until two successive rungs
// agree to 2^-62 relative; the higher rung is returned, rounded to double, with
// |difference| + 2^-53 |result| as its error estimate.  The result is the permanent of
// the exact Cauchy matrix of the given doubles x and y (not of C rounded to double).
//
// One block per matrix (a grid-stride loop over the batch).  The block keeps C o C in
// its own slice of global scratch (n^2 stored values of kBigWords words, resident in
// L2); per elimination step one thread picks the pivot and forms its reciprocal, the
// block forms the row multipliers and then updates the trailing submatrix, one
// element per thread.
#include <cuda_runtime.h>

#include "bigfloat.cuh"
#include "internal.h"

namespace perm {
namespace {

constexpr int kCauchyBlock = 256;

struct CauchyArgs {
  const double* x;    // count x n
  const double* y;    // count x n
  int n;
  int64_t count;
  double* out;        // count results
  double* err;        // count error estimates (or null)
  uint64_t* scratch;  // per block: `words` words
  size_t words;
  int L0;             // first rung of the precision ladder
  int* status;        // set to 1 (coinciding or non-finite points) or 2 (ladder exhausted)
};

__device__ __forceinline__ uint64_t* elem(uint64_t* M, int n, int i, int j) {
  return M + ((size_t)i * n + j) * kBigWords;
}

// per(C) of one matrix at L limbs; the result is left in `res` (thread 0 only).
__device__ void borchardt_at(const double* __restrict__ x, const double* __restrict__ y, int n, int L, uint64_t* M,
                             uint64_t* F, uint64_t* red, uint64_t* slot, Big& res) {
  const int tid = threadIdx.x;
  __shared__ int s_piv;
  __shared__ int s_sign;
  // C o C: 1 / (x_i - y_j)^2
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    Big a, b;
    big_from_double(a, x[i], L);
    big_from_double(b, y[j], L);
    big_add(a, a, b, 1, L);
    big_mul(a, a, a, L);
    big_recip(b, a, L);
    big_store(M + (size_t)idx * kBigWords, b, L);
  }
  // Cauchy's determinant: per-thread partial products, then a tree over the block
  {
    Big num, den, a, b;
    big_from_double(num, 1.0, L);
    big_from_double(den, 1.0, L);
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
      const int i = idx / n, j = idx % n;
      big_from_double(a, x[i], L);
      big_from_double(b, y[j], L);
      big_add(a, a, b, 1, L);
      big_mul(den, den, a, L);
      if (i < j) {
        big_from_double(a, x[j], L);
        big_from_double(b, x[i], L);
        big_add(a, a, b, 1, L);
        big_mul(num, num, a, L);
        big_from_double(a, y[i], L);
        big_from_double(b, y[j], L);
        big_add(a, a, b, 1, L);
        big_mul(num, num, a, L);
      }
    }
    big_store(red + (size_t)tid * kBigWords, num, L);
    big_store(red + (size_t)(blockDim.x + tid) * kBigWords, den, L);
  }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) {
      Big a, b;
      for (int part = 0; part < 2; ++part) {
        uint64_t* base = red + (size_t)part * blockDim.x * kBigWords;
        big_load(a, base + (size_t)tid * kBigWords, L);
        big_load(b, base + (size_t)(tid + s) * kBigWords, L);
        big_mul(a, a, b, L);
        big_store(base + (size_t)tid * kBigWords, a, L);
      }
    }
    __syncthreads();
  }
  // det(C o C): elimination with partial pivoting; thread 0 keeps the pivot product
  Big det;
  if (tid == 0) {
    big_from_double(det, 1.0, L);
    s_sign = 0;
  }
  for (int c = 0; c < n; ++c) {
    if (tid == 0) {
      Big best, v;
      int pr = -1;
      big_set_zero(best, L);
      for (int r = c; r < n; ++r) {
        big_load(v, elem(M, n, r, c), L);
        if (!v.z && (pr < 0 || big_cmp_abs(v, best, L) > 0)) {
          best = v;
          pr = r;
        }
      }
      s_piv = pr;
      if (pr >= 0) {
        if (pr != c) s_sign ^= 1;
        big_mul(det, det, best, L);
        big_recip(v, best, L);
        big_store(slot, v, L);
      } else {
        big_set_zero(det, L);
      }
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr < 0) break;  // singular: det(C o C) = 0
    if (pr != c) {
      for (int k = c + tid; k < n; k += blockDim.x) {
        uint64_t* p = elem(M, n, c, k);
        uint64_t* q = elem(M, n, pr, k);
        for (int w = 0; w <= L; ++w) {
          const uint64_t t = p[w];
          p[w] = q[w];
          q[w] = t;
        }
      }
      __syncthreads();
    }
    const int rest = n - c - 1;
    if (rest == 0) break;
    {
      Big inv, a;
      big_load(inv, slot, L);
      for (int r = c + 1 + tid; r < n; r += blockDim.x) {
        big_load(a, elem(M, n, r, c), L);
        big_mul(a, a, inv, L);
        big_store(F + (size_t)r * kBigWords, a, L);
      }
    }
    __syncthreads();
    for (int q = tid; q < rest * rest; q += blockDim.x) {
      const int r = c + 1 + q / rest, k = c + 1 + q % rest;
      Big f, u, a;
      big_load(f, F + (size_t)r * kBigWords, L);
      big_load(u, elem(M, n, c, k), L);
      big_mul(f, f, u, L);
      big_load(a, elem(M, n, r, k), L);
      big_add(a, a, f, 1, L);
      big_store(elem(M, n, r, k), a, L);
    }
    __syncthreads();
  }
  if (tid == 0) {
    // per = det(C o C) * prod (x_i - y_j) / prod_{i<j} (x_j - x_i)(y_i - y_j)
    Big num, den, a;
    big_load(num, red, L);
    big_load(den, red + (size_t)blockDim.x * kBigWords, L);
    big_recip(a, num, L);
    big_mul(a, a, den, L);
    big_mul(res, det, a, L);
    if (s_sign) res.s ^= 1;
  }
}

__global__ void __launch_bounds__(kCauchyBlock) cauchy_kernel(CauchyArgs a) {
  const int n = a.n;
  const int tid = threadIdx.x;
  uint64_t* M = a.scratch + (size_t)blockIdx.x * a.words;
  uint64_t* F = M + (size_t)n * n * kBigWords;
  uint64_t* red = F + (size_t)n * kBigWords;
  uint64_t* slot = red + (size_t)2 * kCauchyBlock * kBigWords;  // [0] pivot reciprocal, [1] previous rung
  __shared__ int s_bad;
  __shared__ int s_done;
  for (int64_t b = blockIdx.x; b < a.count; b += gridDim.x) {
    const double* x = a.x + b * n;
    const double* y = a.y + b * n;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    // Borchardt's quotient needs det(C) != 0: distinct x_i, distinct y_j, x_i != y_j
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
      const int i = idx / n, j = idx % n;
      const double xi = x[i], yj = y[j];
      bool bad = !isfinite(xi) || !isfinite(yj) || xi == yj;
      if (i < j) bad |= x[i] == x[j] || y[i] == y[j];
      if (bad) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) {
      if (tid == 0) {
        a.out[b] = __longlong_as_double(0x7ff8000000000000ll);
        if (a.err) a.err[b] = a.out[b];
        atomicCAS(a.status, 0, 1);
      }
      __syncthreads();
      continue;
    }
    int L = a.L0, step = 1;
    bool have_prev = false;
    for (;;) {
      Big res;
      borchardt_at(x, y, n, L, M, F, red, slot, res);
      if (tid == 0) {
        int done = 0;
        if (have_prev) {
          Big prev, d;
          big_load(prev, slot + kBigWords, L);
          big_add(d, res, prev, 1, L);
          if (d.z || (!res.z && d.e <= res.e - 62)) {
            done = 1;
            const double v = big_to_double(res, L);
            a.out[b] = v;
            if (a.err) a.err[b] = ::fabs(big_to_double(d, L)) * (1.0 + 0x1p-40) + ::fabs(v) * 0x1p-53;
          }
        }
        if (!done && L == kBigLimbs) {
          done = 1;
          a.out[b] = __longlong_as_double(0x7ff8000000000000ll);
          if (a.err) a.err[b] = a.out[b];
          atomicCAS(a.status, 0, 2);
        }
        if (!done) {
          // keep this rung, zero-padded so that the next (longer) rung reads it exactly
          for (int i = L; i < kBigLimbs; ++i) res.m[i] = 0;
          big_store(slot + kBigWords, res, kBigLimbs);
        }
        s_done = done;
      }
      __syncthreads();
      if (s_done) break;
      have_prev = true;
      L = L + step < kBigLimbs ? L + step : kBigLimbs;
      step *= 2;
    }
    __syncthreads();
  }
}

}  // namespace

size_t cauchy_scratch_words(int n) {
  return ((size_t)n * n + n + 2 * kCauchyBlock + 2) * kBigWords;
}

int cauchy_first_limbs(int n) {
  // about 9 bits lost per unit of n in the elimination, plus 96 bits of margin
  int L = (9 * n + 96 + 63) / 64;
  if (L < 2) L = 2;
  if (L > kBigLimbs) L = kBigLimbs;
  return L;
}

int cauchy_max_n() { return 64; }

cudaError_t launch_cauchy(const double* x, const double* y, int n, int64_t count, double* out, double* err,
                          uint64_t* scratch, int grid, int* status, cudaStream_t stream) {
  CauchyArgs a;
  a.x = x;
  a.y = y;
  a.n = n;
  a.count = count;
  a.out = out;
  a.err = err;
  a.scratch = scratch;
  a.words = cauchy_scratch_words(n);
  a.L0 = cauchy_first_limbs(n);
  a.status = status;
  cauchy_kernel<<<grid, kCauchyBlock, 0, stream>>>(a);
  return cudaGetLastError();
}

int cauchy_block() { return kCauchyBlock; }

}  // namespace perm
