// Permanents of Cauchy matrices c_ij = 1 / (x_i - y_j) by Borchardt's theorem
// (Eq. caucy_permanent): per(C) = det(C o C) / det(C).
//
// det(C) has Cauchy's closed form prod_{i<j} (x_j - x_i)(y_i - y_j) / prod_{i,j} (x_i - y_j),
// a product with no cancellation.  det(C o C) has none: it is taken by Gaussian
// elimination with partial pivoting, and C o C is so ill-conditioned that double
// precision loses every digit from n ~ 12 on (the elimination loses roughly 7 to 9
// bits per unit of n).  Both are therefore evaluated in the multi-limb floating point
// of bigfloat.cuh, with a precision ladder: the permanent is computed at L0 limbs and
// at L0 + 1, then L0 + 3, L0 + 7, ... (ending at kBigLimbs), until two successive rungs
// agree to 2^-62 relative; the higher rung is returned, rounded to double, with
// |difference| + 2^-53 |result| as its error estimate.  The result is the permanent of
// the exact Cauchy matrix of the given doubles x and y (not of C rounded to double).
//
// One kernel per rung, one block per matrix (a grid-stride loop over the batch; a
// matrix finished at an earlier rung is skipped).  The block keeps C o C in its own
// slice of global scratch (n^2 stored values, structure of arrays so that the trailing
// update reads coalesced, resident in L2); per elimination step one thread picks the
// pivot and the block updates the trailing submatrix, one element per thread, without
// division.
#include <cuda_runtime.h>

#include "cauchy_impl.cuh"
#include "internal.h"

namespace perm {
namespace cauchy {
namespace {

// Points of matrix b valid for Borchardt's quotient (det(C) != 0: distinct x_i,
// distinct y_j, x_i != y_j, all finite)?  Invalid matrices get NaN and are finished.
__global__ void __launch_bounds__(kBlock) cauchy_prep_kernel(CauchyArgs a) {
  __shared__ int s_bad;
  const int n = a.n;
  for (int64_t b = blockIdx.x; b < a.count; b += gridDim.x) {
    const double* x = a.x + b * n;
    const double* y = a.y + b * n;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int i = idx / n, j = idx % n;
      const double xi = x[i], yj = y[j];
      bool bad = !isfinite(xi) || !isfinite(yj) || xi == yj;
      if (i < j) bad |= x[i] == x[j] || y[i] == y[j];
      if (bad) s_bad = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_bad) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        a.out[b] = nan;
        if (a.err) a.err[b] = nan;
        atomicCAS(a.status, 0, 1);
      }
      a.state[b] = s_bad ? 2 : 0;
    }
    __syncthreads();
  }
}

cudaError_t launch_rung_l(int L, const CauchyArgs& a, int grid, cudaStream_t stream) {
  switch (L) {
    case 16: return launch_rungs_a(L, a, grid, stream);
    case 12: case 2: return launch_rungs_b(L, a, grid, stream);
    case 11: case 3: case 4: return launch_rungs_c(L, a, grid, stream);
    case 10: case 5: case 6: return launch_rungs_d(L, a, grid, stream);
    case 9: case 7: case 8: return launch_rungs_e(L, a, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

// Does the n x n real matrix A hold c_ij = 1 / (x_i - y_j) up to rounding?  Points fitted
// with x_0 = 0: y_j = -1 / a_0j, x_i = 1 / a_i0 + y_0.  Accepted when every entry is
// finite, nonzero and of the sign of a_00, |a_ij (x_i - y_j) - 1| <= tol (bounded from
// the exact split x_i - y_j = s + e and one fused multiply-add for a_ij s - 1), and the
// x_i and the y_j are distinct.  Then a_ij = c'_ij (1 + rho_ij), |rho_ij| <= tol, for the
// exact Cauchy matrix C' of the fitted points, and every term of both permanents has
// one sign, so |per(A) - per(C')| <= ((1 + tol)^n - 1) |per(C')|.
__global__ void __launch_bounds__(kBlock) cauchy_fit_kernel(const double* __restrict__ A, int n, int64_t rs,
                                                            int64_t cs, double tol, double* x, double* y, int* ok) {
  __shared__ double sx[64], sy[64];
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  if (tid == 0) s_bad = 0;
  if (tid < n) sy[tid] = __ddiv_rn(-1.0, A[tid * cs]);
  __syncthreads();
  if (tid < n) sx[tid] = __dadd_rn(__ddiv_rn(1.0, A[tid * rs]), sy[0]);
  __syncthreads();
  const bool neg = A[0] < 0.0;
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    const double a = A[i * rs + j * cs];
    bool bad = !isfinite(a) || a == 0.0 || (a < 0.0) != neg;
    if (!bad) {
      const double u = sx[i], v = -sy[j];
      const double sum = __dadd_rn(u, v);
      const double bv = __dsub_rn(sum, u);
      const double e = __dadd_rn(__dsub_rn(u, __dsub_rn(sum, bv)), __dsub_rn(v, bv));
      const double r = __fma_rn(a, sum, -1.0);
      const double bound = __dmul_rn(__dadd_rn(::fabs(r), ::fabs(__dmul_rn(a, e))), 1.0 + 0x1p-50);
      bad = !isfinite(sum) || !(bound <= tol);
    }
    if (i < j) bad |= sx[i] == sx[j] || sy[i] == sy[j];
    if (bad) s_bad = 1;
  }
  __syncthreads();
  if (tid < n) {
    x[tid] = sx[tid];
    y[tid] = sy[tid];
  }
  if (tid == 0) *ok = !s_bad;
}

// SBP coefficients of a Cauchy coefficient matrix c_ij = 1 / (x_i - y_j), i < n, j < N
// (Eq. SBGpermanent with Cauchy structure): matrix k has the points x and the y_j of the
// occupied states of occ[k] in increasing order.  A bitstring without exactly n states
// below bit N gets NaN points (so the call marks it invalid).
__global__ void cauchy_gather_kernel(const double* __restrict__ x, int n, const double* __restrict__ y, int N,
                                     const uint64_t* __restrict__ occ, int64_t count, double* xs, double* ys) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const uint64_t below = N == 64 ? ~0ull : ((1ull << N) - 1);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
    const uint64_t bits = occ[k];
    const bool ok = (bits & ~below) == 0 && __popcll(bits) == n;
    uint64_t rest = bits;
    for (int l = 0; l < n; ++l) {
      xs[k * n + l] = x[l];
      if (ok) {
        const int j = __ffsll((long long)rest) - 1;
        rest &= rest - 1;
        ys[k * n + l] = y[j];
      } else {
        ys[k * n + l] = __longlong_as_double(0x7ff8000000000000ll);
      }
    }
  }
}

}  // namespace
}  // namespace cauchy

using cauchy::CauchyArgs;
using cauchy::kBlock;
using cauchy::kWords;

size_t cauchy_scratch_words(int n) { return (size_t)kWords * ((size_t)n * n + n + 2 * kBlock); }

size_t cauchy_state_bytes(int64_t count) { return (size_t)count * (kWords * sizeof(uint64_t) + sizeof(int)); }

static int cauchy_first_limbs(int n) {
  // the elimination loses about 7.5 bits per unit of n (measured against exact
  // rationals on the paper's point ranges); 9 n + 32 bits leave the first rung more
  // than the 62 bits the agreement test needs
  int L = (9 * n + 32 + 63) / 64;
  if (L < 2) L = 2;
  return L;
}

int cauchy_max_n() { return 64; }

// The ladder: L0, L0 + 1, then steps of 2, 4, ..., with rungs above 12 limbs (not
// instantiated) raised to kBigLimbs, the last rung.
static int cauchy_ladder(int n, int* rungs) {
  int k = 0, L = cauchy_first_limbs(n), step = 1;
  while (L <= 12) {
    rungs[k++] = L;
    L += step;
    step *= 2;
  }
  rungs[k++] = kBigLimbs;
  return k;
}

// One block of kBlock threads per matrix, at most two blocks per SM at a time (the
// shorter precisions fit two per SM; 128-thread blocks, four per SM, measured slower).
int cauchy_grid(int64_t count, int sms, int* block) {
  *block = kBlock;
  if (count < 1) return 1;
  return (int)(count < 2 * (int64_t)sms ? count : 2 * (int64_t)sms);
}

cudaError_t launch_cauchy_gather(const double* x, int n, const double* y, int N, const uint64_t* occ, int64_t count,
                                 double* xs, double* ys, int sms, cudaStream_t stream) {
  int64_t grid = (count + 255) / 256;
  if (grid > 8 * (int64_t)sms) grid = 8 * (int64_t)sms;
  if (grid < 1) grid = 1;
  cauchy::cauchy_gather_kernel<<<(int)grid, 256, 0, stream>>>(x, n, y, N, occ, count, xs, ys);
  return cudaGetLastError();
}

cudaError_t launch_cauchy_fit(const double* A, int n, int64_t rs, int64_t cs, double tol, double* x, double* y,
                              int* ok, cudaStream_t stream) {
  cauchy::cauchy_fit_kernel<<<1, kBlock, 0, stream>>>(A, n, rs, cs, tol, x, y, ok);
  return cudaGetLastError();
}

cudaError_t launch_cauchy(const double* x, const double* y, int n, int64_t count, double* out, double* err,
                          uint64_t* scratch, void* state, int grid, int block, int* status, cudaStream_t stream,
                          double rel_extra) {
  CauchyArgs a;
  a.block = block;
  a.rel_extra = rel_extra;
  a.x = x;
  a.y = y;
  a.n = n;
  a.count = count;
  a.out = out;
  a.err = err;
  a.scratch = scratch;
  a.words = cauchy_scratch_words(n);
  a.prev = static_cast<uint64_t*>(state);
  a.state = reinterpret_cast<int*>(a.prev + (size_t)count * kWords);
  a.status = status;
  a.last = 0;
  cauchy::cauchy_prep_kernel<<<grid, a.block, 0, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int rungs[kBigLimbs + 1];
  const int k = cauchy_ladder(n, rungs);
  for (int i = 0; i < k; ++i) {
    a.last = i == k - 1;
    if ((e = cauchy::launch_rung_l(rungs[i], a, grid, stream)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}


}  // namespace perm
