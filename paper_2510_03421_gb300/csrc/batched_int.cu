// Exact batched permanents of integer matrices (perm_batched with PERM_U8, PERM_I64 or
// PERM_CI64, Gaussian integers).
//
// One warp per matrix.  Glynn's formula (Eq. glynn_rectangle) over the 2^(n-1) sign
// vectors in reflected Gray-code order, the n - m padding rows of ones entering as
// virtual rows; the 32 lanes walk contiguous slices of the terms, each rebuilding its
// column sums at the slice start.  Column sums are 64-bit, products and sums wrap
// modulo 2^128, so the sum is exact whenever 2^(n-1) (n-m)! |per| < 2^127; the result
// is that sum shifted right by n - 1 and divided by 2, 3, ..., n - m in turn (each
// division exact).  An a-priori bound (row sums, Bregman's bound for 0/1 entries, the
// column sums' headroom) is checked per matrix; a matrix that fails it raises
// PERM_EOVERFLOW in the status word and still gets the value computed from the sum
// modulo 2^128.  Matrices are grouped by padded order (8, 16, 24, 32) so that the
// column loop is unrolled into registers.  Gaussian integers keep (re, im) column sums
// and a complex product of two 128-bit parts, four 128 x 64-bit products per column.
#include <cstdint>
#include <cuda_runtime.h>

#include "int_bound.cuh"
#include "internal.h"

namespace perm {
namespace {

constexpr int kIntWarps = 4;  // warps per block
constexpr int kIntMaxN = 32;

struct BatchIntArgs {
  const void* packed;
  const int64_t* offsets;
  const int32_t* M;
  const int32_t* N;
  const int32_t* list;  // matrices of this class
  int count;
  int dtype;             // 2 = uint8, 3 = int64
  unsigned long long* out;
  int* status;
};

__device__ __forceinline__ int64_t entry(const void* p, int dtype, int64_t idx) {
  return dtype == 2 ? (int64_t) static_cast<const uint8_t*>(p)[idx] : static_cast<const int64_t*>(p)[idx];
}

// (hi, lo) *= s modulo 2^128, s a signed 64-bit value
__device__ __forceinline__ void mul_s64(uint64_t& lo, uint64_t& hi, uint64_t s) {
  const uint64_t nlo = lo * s;
  const uint64_t nhi = __umul64hi(lo, s) + hi * s - ((int64_t)s < 0 ? lo : 0);
  lo = nlo;
  hi = nhi;
}

// |q| / k for a small k, q = (hi, lo) as an unsigned 128-bit value, by 32-bit limbs
__device__ __forceinline__ void div_small(uint64_t& lo, uint64_t& hi, uint32_t k) {
  uint32_t w[4] = {(uint32_t)(hi >> 32), (uint32_t)hi, (uint32_t)(lo >> 32), (uint32_t)lo};
  uint64_t rem = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint64_t cur = (rem << 32) | w[i];
    w[i] = (uint32_t)(cur / k);
    rem = cur % k;
  }
  hi = ((uint64_t)w[0] << 32) | w[1];
  lo = ((uint64_t)w[2] << 32) | w[3];
}

template <int NP>
__global__ void __launch_bounds__(32 * kIntWarps) batched_int_kernel(BatchIntArgs a) {
  __shared__ uint64_t sA[kIntWarps][NP * NP];  // the (transposed if m > n) operand, row i at i NP
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t* A = sA[w];
  const int64_t nw = (int64_t)gridDim.x * kIntWarps;
  for (int64_t k = (int64_t)blockIdx.x * kIntWarps + w; k < a.count; k += nw) {
    const int b = a.list[k];
    int m = a.M[b], n = a.N[b];
    const int ld = n;
    int64_t rs = ld, cs = 1;
    if (m > n) {
      const int t = m;
      m = n;
      n = t;
      rs = 1;
      cs = ld;
    }
    const int64_t base = a.offsets[b];
    __syncwarp();
    for (int e = lane; e < m * n; e += 32) {
      const int i = e / n, j = e % n;
      A[i * NP + j] = (uint64_t)entry(a.packed, a.dtype, base + i * rs + j * cs);
    }
    // a-priori range check: lane i takes row i, lane j column j
    double lrow = 0.0, lbreg = 0.0;
    bool zero_row = false, binary = true, col_over = false;
    if (lane < m) {
      double rsum = 0.0;
      for (int j = 0; j < n; ++j) {
        const double v = fabs((double)entry(a.packed, a.dtype, base + lane * rs + j * cs));
        binary &= v <= 1.0;
        rsum += v;
      }
      if (rsum == 0.0) {
        zero_row = true;
      } else {
        lrow = log2(rsum);
        lbreg = bregman_log2_term(rsum);
      }
    }
    if (lane < n) {
      double csum = 0.0;
      for (int i = 0; i < m; ++i) csum += fabs((double)entry(a.packed, a.dtype, base + i * rs + lane * cs));
      col_over = column_sum_overflows(csum, m, n);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      lrow += __shfl_xor_sync(0xffffffffu, lrow, off);
      lbreg += __shfl_xor_sync(0xffffffffu, lbreg, off);
    }
    zero_row = __any_sync(0xffffffffu, zero_row);
    binary = __all_sync(0xffffffffu, binary);
    col_over = __any_sync(0xffffffffu, col_over);
    __syncwarp();

    uint64_t alo = 0, ahi = 0;  // this lane's sum of terms, modulo 2^128
    if (m > 0) {
      const uint64_t terms = 1ull << (n - 1);
      const uint64_t per = (terms + 31) / 32;
      uint64_t g = (uint64_t)lane * per;
      const uint64_t g1 = g + per < terms ? g + per : terms;
      if (g < g1) {
        uint64_t S[NP];
        {
          const uint64_t gray = g ^ (g >> 1);
#pragma unroll
          for (int j = 0; j < NP; ++j) S[j] = 0;
          for (int i = 0; i < n; ++i) {
            const bool neg = (gray >> (n - 1 - i)) & 1u;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
              if (j < n) {
                const uint64_t v = i < m ? A[i * NP + j] : 1ull;
                S[j] = neg ? S[j] - v : S[j] + v;
              }
            }
          }
        }
        for (;;) {
          uint64_t plo = 1, phi = 0;
#pragma unroll
          for (int j = 0; j < NP; ++j)
            if (j < n) mul_s64(plo, phi, S[j]);
          if (g & 1) {
            const uint64_t borrow = alo < plo;
            alo -= plo;
            ahi -= phi + borrow;
          } else {
            alo += plo;
            ahi += phi + (alo < plo);
          }
          if (++g >= g1) break;
          const int bit = __ffsll((long long)g) - 1;
          const int r = n - 1 - bit;
          const bool neg = ((g ^ (g >> 1)) >> bit) & 1u;
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            if (j < n) {
              const uint64_t d = (r < m ? A[r * NP + j] : 1ull) << 1;
              S[j] = neg ? S[j] - d : S[j] + d;
            }
          }
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const uint64_t olo = __shfl_down_sync(0xffffffffu, alo, off);
      const uint64_t ohi = __shfl_down_sync(0xffffffffu, ahi, off);
      alo += olo;
      ahi += ohi + (alo < olo);
    }
    if (lane == 0) {
      uint64_t lo = alo, hi = ahi;
      if (m == 0) {
        lo = 1;
        hi = 0;
      } else {
        if (col_over || (!zero_row && glynn_sum_log2_bound(m, n, lrow, lbreg, binary) >= kInt128Bits))
          atomicCAS(a.status, 0, 3);
        // sum / 2^(n-1) / (n-m)!, exact divisions of the magnitude
        const bool negv = (int64_t)hi < 0;
        if (negv) {  // two's-complement negation
          lo = ~lo + 1;
          hi = ~hi + (lo == 0);
        }
        const int sh = n - 1;
        if (sh > 0) {
          lo = (lo >> sh) | (sh < 64 ? hi << (64 - sh) : 0);
          hi >>= sh;
        }
        for (uint32_t f = 2; f <= (uint32_t)(n - m); ++f) div_small(lo, hi, f);
        if (negv) {
          lo = ~lo + 1;
          hi = ~hi + (lo == 0);
        }
      }
      a.out[2 * (size_t)b] = lo;
      a.out[2 * (size_t)b + 1] = hi;
    }
  }
}

// (hi, lo) * s modulo 2^128 into (rhi, rlo), s a signed 64-bit value
__device__ __forceinline__ void mul_s64_to(uint64_t lo, uint64_t hi, uint64_t s, uint64_t& rlo, uint64_t& rhi) {
  rlo = lo * s;
  rhi = __umul64hi(lo, s) + hi * s - ((int64_t)s < 0 ? lo : 0);
}

// q / 2^sh / (2 .. f) of a two's-complement 128-bit value whose magnitude these divide
__device__ __forceinline__ void divide_exact(uint64_t& lo, uint64_t& hi, int sh, int f) {
  const bool negv = (int64_t)hi < 0;
  if (negv) {
    lo = ~lo + 1;
    hi = ~hi + (lo == 0);
  }
  if (sh > 0) {
    lo = (lo >> sh) | (hi << (64 - sh));
    hi >>= sh;
  }
  for (uint32_t k = 2; k <= (uint32_t)f; ++k) div_small(lo, hi, k);
  if (negv) {
    lo = ~lo + 1;
    hi = ~hi + (lo == 0);
  }
}

constexpr int kGaussWarps = 2;  // warps per block of the Gaussian-integer kernel

template <int NP>
__global__ void __launch_bounds__(32 * kGaussWarps) batched_gauss_kernel(BatchIntArgs a) {
  __shared__ uint64_t sA[kGaussWarps][2 * NP * NP];  // (re, im) of row i, column j at 2 (i NP + j)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t* A = sA[w];
  const int64_t* P = static_cast<const int64_t*>(a.packed);
  const int64_t nw = (int64_t)gridDim.x * kGaussWarps;
  for (int64_t k = (int64_t)blockIdx.x * kGaussWarps + w; k < a.count; k += nw) {
    const int b = a.list[k];
    int m = a.M[b], n = a.N[b];
    const int ld = n;
    int64_t rs = ld, cs = 1;
    if (m > n) {
      const int t = m;
      m = n;
      n = t;
      rs = 1;
      cs = ld;
    }
    const int64_t base = a.offsets[b];
    __syncwarp();
    for (int e = lane; e < m * n; e += 32) {
      const int i = e / n, j = e % n;
      const int64_t idx = base + i * rs + j * cs;
      A[2 * (i * NP + j)] = (uint64_t)P[2 * idx];
      A[2 * (i * NP + j) + 1] = (uint64_t)P[2 * idx + 1];
    }
    // a-priori range check on |re| + |im|: lane i takes row i, lane j column j
    double lrow = 0.0;
    bool zero_row = false, col_over = false;
    if (lane < m) {
      double rsum = 0.0;
      for (int j = 0; j < n; ++j) {
        const int64_t idx = base + lane * rs + j * cs;
        rsum += fabs((double)P[2 * idx]) + fabs((double)P[2 * idx + 1]);
      }
      if (rsum == 0.0) zero_row = true;
      else lrow = log2(rsum);
    }
    if (lane < n) {
      double csum = 0.0;
      for (int i = 0; i < m; ++i) {
        const int64_t idx = base + i * rs + lane * cs;
        csum += fabs((double)P[2 * idx]) + fabs((double)P[2 * idx + 1]);
      }
      col_over = column_sum_overflows(csum, m, n);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lrow += __shfl_xor_sync(0xffffffffu, lrow, off);
    zero_row = __any_sync(0xffffffffu, zero_row);
    col_over = __any_sync(0xffffffffu, col_over);
    __syncwarp();

    uint64_t rlo = 0, rhi = 0, ilo = 0, ihi = 0;  // this lane's sum, modulo 2^128 per part
    if (m > 0) {
      const uint64_t terms = 1ull << (n - 1);
      const uint64_t per = (terms + 31) / 32;
      uint64_t g = (uint64_t)lane * per;
      const uint64_t g1 = g + per < terms ? g + per : terms;
      if (g < g1) {
        uint64_t Sr[NP], Si[NP];
        {
          const uint64_t gray = g ^ (g >> 1);
#pragma unroll
          for (int j = 0; j < NP; ++j) Sr[j] = Si[j] = 0;
          for (int i = 0; i < n; ++i) {
            const bool neg = (gray >> (n - 1 - i)) & 1u;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
              if (j < n) {
                const uint64_t vr = i < m ? A[2 * (i * NP + j)] : 1ull;
                const uint64_t vi = i < m ? A[2 * (i * NP + j) + 1] : 0ull;
                Sr[j] = neg ? Sr[j] - vr : Sr[j] + vr;
                Si[j] = neg ? Si[j] - vi : Si[j] + vi;
              }
            }
          }
        }
        for (;;) {
          // (pr + i pi) = prod_j (Sr_j + i Si_j), each part modulo 2^128
          uint64_t prl = 1, prh = 0, pil = 0, pih = 0;
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            if (j < n) {
              uint64_t t1l, t1h, t2l, t2h, t3l, t3h, t4l, t4h;
              mul_s64_to(prl, prh, Sr[j], t1l, t1h);
              mul_s64_to(pil, pih, Si[j], t2l, t2h);
              mul_s64_to(prl, prh, Si[j], t3l, t3h);
              mul_s64_to(pil, pih, Sr[j], t4l, t4h);
              prl = t1l - t2l;
              prh = t1h - t2h - (t1l < t2l);
              pil = t3l + t4l;
              pih = t3h + t4h + (pil < t3l);
            }
          }
          if (g & 1) {
            rhi -= prh + (rlo < prl);
            rlo -= prl;
            ihi -= pih + (ilo < pil);
            ilo -= pil;
          } else {
            rlo += prl;
            rhi += prh + (rlo < prl);
            ilo += pil;
            ihi += pih + (ilo < pil);
          }
          if (++g >= g1) break;
          const int bit = __ffsll((long long)g) - 1;
          const int r = n - 1 - bit;
          const bool neg = ((g ^ (g >> 1)) >> bit) & 1u;
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            if (j < n) {
              const uint64_t dr = (r < m ? A[2 * (r * NP + j)] : 1ull) << 1;
              const uint64_t di = (r < m ? A[2 * (r * NP + j) + 1] : 0ull) << 1;
              Sr[j] = neg ? Sr[j] - dr : Sr[j] + dr;
              Si[j] = neg ? Si[j] - di : Si[j] + di;
            }
          }
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const uint64_t orl = __shfl_down_sync(0xffffffffu, rlo, off);
      const uint64_t orh = __shfl_down_sync(0xffffffffu, rhi, off);
      const uint64_t oil = __shfl_down_sync(0xffffffffu, ilo, off);
      const uint64_t oih = __shfl_down_sync(0xffffffffu, ihi, off);
      rlo += orl;
      rhi += orh + (rlo < orl);
      ilo += oil;
      ihi += oih + (ilo < oil);
    }
    if (lane == 0) {
      if (m == 0) {
        rlo = 1;
        rhi = ilo = ihi = 0;
      } else {
        if (col_over || (!zero_row && glynn_sum_log2_bound(m, n, lrow, 0.0, false) >= kInt128Bits))
          atomicCAS(a.status, 0, 3);
        divide_exact(rlo, rhi, n - 1, n - m);
        divide_exact(ilo, ihi, n - 1, n - m);
      }
      a.out[4 * (size_t)b] = rlo;
      a.out[4 * (size_t)b + 1] = rhi;
      a.out[4 * (size_t)b + 2] = ilo;
      a.out[4 * (size_t)b + 3] = ihi;
    }
  }
}

}  // namespace

int batched_int_class(int n) { return n <= 8 ? 8 : n <= 16 ? 16 : n <= 24 ? 24 : n <= kIntMaxN ? 32 : 0; }

int batched_int_max_n() { return kIntMaxN; }

cudaError_t launch_batched_int(const void* packed, const int64_t* offsets, const int32_t* M, const int32_t* N,
                               const int32_t* list, int count, int dtype, int npad, unsigned long long* out,
                               int* status, int sms, cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  BatchIntArgs a{packed, offsets, M, N, list, count, dtype, out, status};
  if (dtype == 4) {
    const int threads = 32 * kGaussWarps;
    int grid = (count + kGaussWarps - 1) / kGaussWarps;
    if (grid > 16 * sms) grid = 16 * sms;
    switch (npad) {
      case 8: batched_gauss_kernel<8><<<grid, threads, 0, stream>>>(a); break;
      case 16: batched_gauss_kernel<16><<<grid, threads, 0, stream>>>(a); break;
      case 24: batched_gauss_kernel<24><<<grid, threads, 0, stream>>>(a); break;
      case 32: batched_gauss_kernel<32><<<grid, threads, 0, stream>>>(a); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  const int threads = 32 * kIntWarps;
  int grid = (count + kIntWarps - 1) / kIntWarps;
  const int cap = 8 * sms;
  if (grid > cap) grid = cap;
  switch (npad) {
    case 8: batched_int_kernel<8><<<grid, threads, 0, stream>>>(a); break;
    case 16: batched_int_kernel<16><<<grid, threads, 0, stream>>>(a); break;
    case 24: batched_int_kernel<24><<<grid, threads, 0, stream>>>(a); break;
    case 32: batched_int_kernel<32><<<grid, threads, 0, stream>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace perm
