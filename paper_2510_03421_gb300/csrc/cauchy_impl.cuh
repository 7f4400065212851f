// Templated device code of the Cauchy path, shared by the translation units that
// instantiate one or a few precisions each (cauchy_l*.cu; the long precisions take
// most of the compile time, so they are spread over files built in parallel).
#pragma once

#include <cuda_runtime.h>

#include "bigfloat.cuh"

namespace perm {
namespace cauchy {

constexpr int kBlock = 256;
constexpr int kWords = kBigLimbs + 1;  // stored value: header word + limbs

struct CauchyArgs {
  const double* x;    // count x n
  const double* y;    // count x n
  int n;
  int64_t count;
  double* out;        // count results
  double* err;        // count error estimates (or null)
  uint64_t* scratch;  // per block: `words` words
  size_t words;
  uint64_t* prev;     // per matrix: the previous rung's result, kWords words
  int* state;         // per matrix: 0 = first rung, 1 = previous rung kept, 2 = finished
  int* status;        // set to 1 (coinciding or non-finite points) or 2 (ladder exhausted)
  int last;           // this rung is the last of the ladder
  int block;          // threads per block (kBlock)
  double rel_extra;   // added to the relative error estimate (perturbation of fitted points)
};

template <int L>
__device__ __forceinline__ void point_diff(Big<L>& d, double u, double v) {
  Big<L> t;
  big_from_double(d, u);
  big_from_double(t, v);
  big_add(d, d, t, 1);
}

// per(C) of one matrix at L limbs; the result is left in `res` (thread 0 only).
// Scratch (structure of arrays): M = C o C, n^2 values; F, n values; red, 2 x block.
template <int L>
__device__ void borchardt_at(const double* __restrict__ x, const double* __restrict__ y, int n, uint64_t* M,
                             uint64_t* F, uint64_t* red, Big<L>& res) {
  const int tid = threadIdx.x;
  const size_t nn = (size_t)n * n;
  const size_t rs = 2 * (size_t)blockDim.x;
  __shared__ int s_piv, s_sign, s_pe, s_esum;
  __shared__ int s_perm[64];  // logical row r of the elimination is stored row s_perm[r]
  for (int r = tid; r < n; r += blockDim.x) s_perm[r] = r;
  // C o C: 1 / (x_i - y_j)^2
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    Big<L> d, v;
    point_diff(d, x[idx / n], y[idx % n]);
    big_mul(d, d, d);
    big_recip(v, d);
    big_store(M, nn, idx, v);
  }
  // Cauchy's determinant: per-thread partial products, then a tree over the block
  {
    Big<L> num, den, d;
    big_from_double(num, 1.0);
    big_from_double(den, 1.0);
    for (int idx = tid; idx < n * n; idx += blockDim.x) {
      const int i = idx / n, j = idx % n;
      point_diff(d, x[i], y[j]);
      big_mul(den, den, d);
      if (i < j) {
        point_diff(d, x[j], x[i]);
        big_mul(num, num, d);
        point_diff(d, y[i], y[j]);
        big_mul(num, num, d);
      }
    }
    big_store(red, rs, tid, num);
    big_store(red, rs, blockDim.x + tid, den);
  }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) {
      Big<L> u, v;
      for (int part = 0; part < 2; ++part) {
        const size_t o = (size_t)part * blockDim.x;
        big_load(u, red, rs, o + tid);
        big_load(v, red, rs, o + tid + s);
        big_mul(u, u, v);
        big_store(red, rs, o + tid, u);
      }
    }
    __syncthreads();
  }
  // det(C o C): division-free elimination with partial pivoting.  With the pivot of
  // step c written p_c = 2^e_c q_c (|q_c| in [1/2, 1)), row r > c becomes
  // q_c row_r - M[r][c] 2^-e_c row_c: every trailing row is scaled by q_c, no
  // reciprocal sits on the per-step critical path, and the magnitudes do not drift.
  // Then det(C o C) = +-2^(sum_c e_c) q_{n-1} / prod_{c <= n-2} q_c^(n-2-c).
  if (tid == 0) {
    s_sign = 0;
    s_esum = 0;
  }
  bool singular = false;
  for (int c = 0; c < n; ++c) {
    if (tid < 32) {
      // pivot: the largest |M[r][c]|, r >= c, earliest row among equals; each lane takes
      // rows c + lane + 32 i, then a shuffle reduction over the warp
      Big<L> best, v;
      int pr = -1;
      big_set_zero(best);
      for (int r = c + tid; r < n; r += 32) {
        big_load(v, M, nn, (size_t)s_perm[r] * n + c);
        if (!v.z && (pr < 0 || big_cmp_abs(v, best) > 0)) {
          best = v;
          pr = r;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const int opr = __shfl_down_sync(0xffffffffu, pr, off);
        v.e = __shfl_down_sync(0xffffffffu, best.e, off);
        v.s = __shfl_down_sync(0xffffffffu, best.s, off);
        v.z = __shfl_down_sync(0xffffffffu, best.z, off);
#pragma unroll
        for (int i = 0; i < L; ++i) v.m[i] = __shfl_down_sync(0xffffffffu, best.m[i], off);
        if (opr >= 0) {
          const int cmp = pr < 0 ? 1 : big_cmp_abs(v, best);
          if (cmp > 0 || (cmp == 0 && opr < pr)) {
            best = v;
            pr = opr;
          }
        }
      }
      if (tid == 0) {
        s_piv = pr;
        if (pr >= 0) {
          if (pr != c) {  // exchange the rows by their indices
            const int t = s_perm[c];
            s_perm[c] = s_perm[pr];
            s_perm[pr] = t;
            s_sign ^= 1;
          }
          s_pe = best.e;
          s_esum += best.e;
          best.e = 0;
          big_store(F, (size_t)n, c, best);  // q_c
        }
      }
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr < 0) {  // det(C o C) = 0
      singular = true;
      break;
    }
    const int rest = n - c - 1;
    if (rest == 0) break;
    {
      const int pe = s_pe;
      const size_t prow = (size_t)s_perm[c] * n;
      Big<L> qc, v, f, u;
      big_load(qc, F, (size_t)n, c);
      for (int q = tid; q < rest * rest; q += blockDim.x) {
        const size_t row = (size_t)s_perm[c + 1 + q / rest] * n;
        const int k = c + 1 + q % rest;
        big_load(v, M, nn, row + k);
        big_mul(v, v, qc);
        big_load(f, M, nn, row + c);
        big_load(u, M, nn, prow + k);
        u.e -= pe;
        big_mul(f, f, u);
        big_add(v, v, f, 1);
        big_store(M, nn, row + k, v);
      }
    }
    __syncthreads();
  }
  if (singular) {
    if (tid == 0) big_set_zero(res);
    return;
  }
  // prod_{c <= n-2} q_c^(n-2-c): powers by squaring in place, then a tree over c
  const int cnt = n - 1;
  for (int c = tid; c < cnt; c += blockDim.x) {
    Big<L> base, pw;
    big_load(base, F, (size_t)n, c);
    big_from_double(pw, 1.0);
    for (int k = n - 2 - c; k > 0; k >>= 1) {
      if (k & 1) big_mul(pw, pw, base);
      if (k > 1) big_mul(base, base, base);
    }
    big_store(F, (size_t)n, c, pw);
  }
  __syncthreads();
  for (int s = 32; s >= 1; s >>= 1) {
    if (tid < s && tid + s < cnt) {
      Big<L> u, v;
      big_load(u, F, (size_t)n, tid);
      big_load(v, F, (size_t)n, tid + s);
      big_mul(u, u, v);
      big_store(F, (size_t)n, tid, u);
    }
    __syncthreads();
  }
  if (tid == 0) {
    // per = det(C o C) prod (x_i - y_j) / prod_{i<j} (x_j - x_i)(y_i - y_j)
    Big<L> num, v;
    big_load(num, red, rs, 0);
    if (cnt > 0) {
      big_load(v, F, (size_t)n, 0);
      big_mul(num, num, v);
    }
    big_recip(res, num);
    big_load(v, red, rs, blockDim.x);
    big_mul(res, res, v);
    big_load(v, F, (size_t)n, n - 1);
    big_mul(res, res, v);
    res.e += s_esum;
    if (s_sign) res.s ^= 1;
  }
}

// One rung of the precision ladder over all unfinished matrices.
template <int L>
__global__ void __launch_bounds__(kBlock, L <= 8 ? 2 : 1) cauchy_rung_kernel(CauchyArgs a) {
  const int n = a.n;
  uint64_t* M = a.scratch + (size_t)blockIdx.x * a.words;
  uint64_t* F = M + (size_t)kWords * n * n;
  uint64_t* red = F + (size_t)kWords * n;
  for (int64_t b = blockIdx.x; b < a.count; b += gridDim.x) {
    const int st = a.state[b];
    if (st == 2) continue;
    Big<L> res;
    borchardt_at<L>(a.x + b * n, a.y + b * n, n, M, F, red, res);
    if (threadIdx.x == 0) {
      uint64_t* pv = a.prev + (size_t)b * kWords;
      int next = 1;
      if (st == 1) {
        Big<L> prev, d;
        big_load(prev, pv, 1, 0);  // kept zero-padded to kBigLimbs: exact at L limbs
        big_add(d, res, prev, 1);
        if (d.z || (!res.z && d.e <= res.e - 62)) {
          const double v = big_to_double(res);
          a.out[b] = v;
          if (a.err) a.err[b] = ::fabs(big_to_double(d)) * (1.0 + 0x1p-40) + ::fabs(v) * (0x1p-53 + a.rel_extra);
          next = 2;
        }
      }
      if (next != 2 && a.last) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        a.out[b] = nan;
        if (a.err) a.err[b] = nan;
        atomicCAS(a.status, 0, 2);
        next = 2;
      }
      if (next == 1) {
        pv[0] = (uint64_t)(uint32_t)res.e | ((uint64_t)res.s << 32) | ((uint64_t)res.z << 33);
        for (int i = 0; i < kBigLimbs; ++i) pv[1 + i] = i < L ? res.m[i] : 0;
      }
      a.state[b] = next;
    }
    __syncthreads();
  }
}

template <int L>
cudaError_t launch_rung(const CauchyArgs& a, int grid, cudaStream_t stream) {
  cauchy_rung_kernel<L><<<grid, a.block, 0, stream>>>(a);
  return cudaGetLastError();
}

// rung launchers of the instantiating files; each returns cudaErrorInvalidValue for an L
// it does not hold
cudaError_t launch_rungs_a(int L, const CauchyArgs& a, int grid, cudaStream_t stream);
cudaError_t launch_rungs_b(int L, const CauchyArgs& a, int grid, cudaStream_t stream);
cudaError_t launch_rungs_c(int L, const CauchyArgs& a, int grid, cudaStream_t stream);
cudaError_t launch_rungs_d(int L, const CauchyArgs& a, int grid, cudaStream_t stream);
cudaError_t launch_rungs_e(int L, const CauchyArgs& a, int grid, cudaStream_t stream);

}  // namespace cauchy
}  // namespace perm
