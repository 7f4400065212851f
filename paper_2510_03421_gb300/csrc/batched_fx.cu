// Batched Glynn (Eq. glynn, Eq. glynn_rectangle) on the integer pipes: the warp-item
// classes of perm_batched (matrices cut into aligned sub-ranges of 2^item_log2 terms,
// one warp each) with the arithmetic of glynn_cfx.cu (complex) and glynn_fx.cu (real).
//   * A preparation kernel (one warp per matrix, one lane per column) scales column j
//     by 2^e_j (sum_i (|re a'_ij| + |im a'_ij|) 2^e_j <= 2^61, the padding rows of ones
//     included), rounds once to int64 and writes +2q (re, im) for every row, the
//     padding rows too, into the batch workspace, and the matrix's sum of e_j.
//   * In a warp item the 32 lanes take consecutive aligned chunks of the sub-range,
//     so they flip the same row at each step and read it as one broadcast.  Column
//     sums are exact int64 in registers; the product is a complex software float
//     (two signed 64-bit mantissas with one exponent) and each lane sums its terms in
//     two 192-bit fixed-point accumulators anchored on its first term.
//   * The lanes' totals are converted to double-double and reduced by shuffles; the
//     warp that completes a matrix's last sub-range combines the partials in a fixed
//     order, as in the FP64 class kernels.
#include "device_common.cuh"
#include "fixed_common.cuh"
#include "internal.h"

namespace perm {
namespace {

// Shape of matrix b after the transpose rule per(A) = per(A^T) for m > n.
struct FxMat {
  int64_t off, rs, cs;
  int m, n;
};

__device__ __forceinline__ FxMat fxmat_of(const BatchArgs& a, int b) {
  FxMat t;
  const int mo = a.M[b], no = a.N[b];
  t.off = a.offsets[b];
  if (mo > no) {
    t.m = no;
    t.n = mo;
    t.rs = 1;
    t.cs = no;
  } else {
    t.m = mo;
    t.n = no;
    t.rs = no;
    t.cs = 1;
  }
  return t;
}

// One warp per matrix of the list; lane j handles column j (n <= 32).
__global__ void batched_cfx_prep_kernel(BatchArgs a, const int32_t* list, int count) {
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * (blockDim.x >> 5)) + (threadIdx.x >> 5));
  if (w >= count) return;
  const int b = list[w];
  const FxMat t = fxmat_of(a, b);
  const int j = lane;
  int e = 0, bad = 0;
  if (j < t.n) {
    double colabs = (double)(t.n - t.m);
    for (int i = 0; i < t.m; ++i) {
      const double* p = a.packed + 2 * (t.off + i * t.rs + j * t.cs);
      if (!isfinite(p[0]) || !isfinite(p[1])) bad = 1;
      colabs += fabs(p[0]) + fabs(p[1]);
    }
    int x = 0;
    if (colabs > 0.0) frexp(colabs, &x);
    e = 61 - x;
    long long* q = a.fx_table + a.fx_offset[b] + 2 * j;  // row i at q + 2 n i
    for (int i = 0; i < t.n; ++i) {
      long long qr, qi;
      if (i < t.m) {
        const double* p = a.packed + 2 * (t.off + i * t.rs + j * t.cs);
        qr = llrint(ldexp(p[0], e));
        qi = llrint(ldexp(p[1], e));
      } else {
        qr = llrint(ldexp(1.0, e));
        qi = 0;
      }
      q[2 * t.n * i] = 2 * qr;
      q[2 * t.n * i + 1] = 2 * qi;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_down_sync(0xffffffffu, e, o);
    bad |= __shfl_down_sync(0xffffffffu, bad, o);
  }
  if (lane == 0) a.fx_esum[b] = bad ? kFxBad : e;
}

// Sum of the Glynn terms [g, g + len) of matrix t (table q, +2q rows of 2n int64),
// unnormalised, as two 192-bit accumulators scaled by 2^e_lo.  The first K columns of
// each product are multiplied on the FP64 unit (a complex double, folded in once).
template <int N, int K>
__device__ __forceinline__ void cfx_slice(const long long* __restrict__ q, int n, int e_sum, uint64_t g, uint64_t len,
                                          u64 (&ar)[3], u64 (&ai)[3], int& e_lo) {
  long long Sr[N], Si[N];
  bool anchored = false;
  e_lo = 0;
  ar[0] = ar[1] = ar[2] = 0;
  ai[0] = ai[1] = ai[2] = 0;
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0) {
      const uint64_t gray = g ^ (g >> 1);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        Sr[j] = 0;
        Si[j] = 0;
      }
      for (int i = 0; i < n; ++i) {
        const bool minus = (gray >> (n - 1 - i)) & 1u;
        const long long* row = q + 2 * n * i;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          if (j < n) {
            const long long vr = __ldg(row + 2 * j), vi = __ldg(row + 2 * j + 1);
            Sr[j] += minus ? -vr : vr;
            Si[j] += minus ? -vi : vi;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < N; ++j) {
        Sr[j] >>= 1;
        Si[j] >>= 1;
      }
    } else {
      const int b = ctz64(g);
      const bool plus = (g >> (b + 1)) & 1u;
      const long long* row = q + 2 * n * (n - 1 - b);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        if (j < n) {
          const long long vr = __ldg(row + 2 * j), vi = __ldg(row + 2 * j + 1);
          Sr[j] += plus ? vr : -vr;
          Si[j] += plus ? vi : -vi;
        }
      }
    }
    // product (pr + i pi) 2^(E - 62), larger component in [2^61, 2^62); columns j < K
    // as a complex double dr + i di
    long long pr = 0, pi = 0;
    int E = 0;
    double dr = 1.0, di = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      if (j < K) {
        const double xr = (double)Sr[j], xi = (double)Si[j];
        if (j == 0) {
          dr = xr;
          di = xi;
        } else {
          const double nr = __fma_rn(dr, xr, -__dmul_rn(di, xi));
          const double ni = __fma_rn(dr, xi, __dmul_rn(di, xr));
          dr = nr;
          di = ni;
        }
      } else if (j < n) {
        const int l = norm_shift(Sr[j], Si[j]);
        const long long sr = Sr[j] << l, si = Si[j] << l;
        if (j == K) {
          pr = sr;
          pi = si;
          E = 62 - l;
        } else {
          cmul_step(pr, pi, E, sr, si, l);
        }
      }
    }
    if (K > 0 && (pr != 0 || pi != 0)) cfold_double(pr, pi, E, dr, di);
    if (pr != 0 || pi != 0) {
      if (g & 1u) {
        pr = -pr;
        pi = -pi;
      }
      if (!anchored) {
        e_lo = E - e_sum - kAnchorBit - 1;
        anchored = true;
      }
      int p = E - 62 - e_sum - e_lo;
      if (p > kMaxLsb) {
        shr192(ar[0], ar[1], ar[2], p - kMaxLsb);
        shr192(ai[0], ai[1], ai[2], p - kMaxLsb);
        e_lo += p - kMaxLsb;
        p = kMaxLsb;
      }
      add192(ar[0], ar[1], ar[2], pr, p);
      add192(ai[0], ai[1], ai[2], pi, p);
    }
  }
}

__device__ __forceinline__ dd normalise_fx(dd v, int n, int m) {
  v = dd_ldexp(v, -(n - 1));
  for (int k = 2; k <= n - m; ++k) v = dd_div_d(v, (double)k);
  return v;
}

__device__ __forceinline__ void write_cplx(const BatchArgs& a, int b, const FxMat& t, dd vr, dd vi, bool bad) {
  double* out = a.out + 2 * (int64_t)b;
  if (bad) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    out[0] = nan;
    out[1] = nan;
    return;
  }
  vr = normalise_fx(vr, t.n, t.m);
  vi = normalise_fx(vi, t.n, t.m);
  out[0] = __dadd_rn(vr.hi, vr.lo);
  out[1] = __dadd_rn(vi.hi, vi.lo);
}

template <int N, int K>
__global__ void __launch_bounds__(128) batched_cfx_kernel(BatchArgs a, ClassWork c) {
  const int lane = threadIdx.x & 31;
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(c.counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= c.nitems) break;
    const BatchItem it = c.items[item];
    const int b = a.order[it.first];
    const FxMat t = fxmat_of(a, b);
    if (t.m == 0) {
      if (lane == 0) {
        a.out[2 * (int64_t)b] = 1.0;
        a.out[2 * (int64_t)b + 1] = 0.0;
      }
      continue;
    }
    const int e_sum = a.fx_esum[b];
    const bool bad = e_sum == kFxBad;
    // sub-range it.count of it.parts (equal, aligned: the term count is a power of
    // two), then this lane's aligned share of it
    const uint64_t terms = 1ull << (t.n - 1);
    uint64_t g0, len0, g, len;
    split_range(0, terms, (uint64_t)it.parts, (uint64_t)it.count, &g0, &len0);
    split_range(g0, g0 + len0, 32, (uint64_t)lane, &g, &len);
    u64 ar[3], ai[3];
    int e_lo = 0;
    dd vr{0.0, 0.0}, vi{0.0, 0.0};
    if (!bad) {
      cfx_slice<N, K>(a.fx_table + a.fx_offset[b], t.n, e_sum, g, len, ar, ai, e_lo);
      vr = to_dd(ar[0], ar[1], ar[2], e_lo);
      vi = to_dd(ai[0], ai[1], ai[2], e_lo);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      vr = dd_add(vr, shfl_down_dd(vr, o));
      vi = dd_add(vi, shfl_down_dd(vi, o));
    }
    if (lane == 0) {
      if (it.parts == 1) {
        write_cplx(a, b, t, vr, vi, bad);
      } else {
        double* slot = a.partials + 4 * ((int64_t)a.part_base[b] + it.count);
        slot[0] = vr.hi;
        slot[1] = vr.lo;
        slot[2] = vi.hi;
        slot[3] = vi.lo;
        __threadfence();
        const int arrived = atomicAdd(a.done + b, 1);
        if (arrived == it.parts - 1) {  // the last sub-range of matrix b: combine in order
          __threadfence();
          const volatile double* p = a.partials + 4 * (int64_t)a.part_base[b];
          dd sr{0.0, 0.0}, si{0.0, 0.0};
          for (int k = 0; k < it.parts; ++k) {
            sr = dd_add(sr, dd{p[4 * k], p[4 * k + 1]});
            si = dd_add(si, dd{p[4 * k + 2], p[4 * k + 3]});
          }
          write_cplx(a, b, t, sr, si, bad);
        }
      }
    }
  }
}

// Real input: one warp per matrix, lane j scales column j (sum_i |a'_ij| 2^e_j <= 2^61,
// the padding rows of ones included) and writes +2q for every row (n rows of n int64).
__global__ void batched_fxr_prep_kernel(BatchArgs a, const int32_t* list, int count) {
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * (blockDim.x >> 5)) + (threadIdx.x >> 5));
  if (w >= count) return;
  const int b = list[w];
  const FxMat t = fxmat_of(a, b);
  const int j = lane;
  int e = 0, bad = 0;
  if (j < t.n) {
    double colabs = (double)(t.n - t.m);
    for (int i = 0; i < t.m; ++i) {
      const double v = a.packed[t.off + i * t.rs + j * t.cs];
      if (!isfinite(v)) bad = 1;
      colabs += fabs(v);
    }
    int x = 0;
    if (colabs > 0.0) frexp(colabs, &x);
    e = 61 - x;
    long long* q = a.fx_table + a.fx_offset[b] + j;  // row i at q + n i
    for (int i = 0; i < t.n; ++i) {
      const long long v = (i < t.m) ? llrint(ldexp(a.packed[t.off + i * t.rs + j * t.cs], e)) : llrint(ldexp(1.0, e));
      q[t.n * i] = 2 * v;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_down_sync(0xffffffffu, e, o);
    bad |= __shfl_down_sync(0xffffffffu, bad, o);
  }
  if (lane == 0) a.fx_esum[b] = bad ? kFxBad : e;
}

// Real terms [g, g + len) of an order-n matrix (table q, +2q rows of n int64) into one
// 192-bit accumulator; columns j >= n are the constant 2^31 (their scale is added to
// e_sum), the last K of the N columns are multiplied on the FP64 unit (soft_product).
template <int N, int K>
__device__ __forceinline__ void fxr_slice(const long long* __restrict__ q, int n, int e_sum, uint64_t g, uint64_t len,
                                          u64 (&acc)[3], int& e_lo) {
  long long S[N];
  bool anchored = false;
  e_lo = 0;
  acc[0] = acc[1] = acc[2] = 0;
  const int es = e_sum + 31 * (N - n);
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0) {
      const uint64_t gray = g ^ (g >> 1);
#pragma unroll
      for (int j = 0; j < N; ++j) S[j] = 0;
      for (int i = 0; i < n; ++i) {
        const bool minus = (gray >> (n - 1 - i)) & 1u;
        const long long* row = q + n * i;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          if (j < n) {
            const long long v = __ldg(row + j);
            S[j] += minus ? -v : v;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < N; ++j) S[j] = (j < n) ? (S[j] >> 1) : (1ll << 31);
    } else {
      const int b = ctz64(g);
      const bool plus = (g >> (b + 1)) & 1u;
      const long long* row = q + n * (n - 1 - b);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        if (j < n) {
          const long long v = __ldg(row + j);
          S[j] += plus ? v : -v;
        }
      }
    }
    u64 P;
    int E;
    unsigned neg;
    soft_product<N, K>(S, P, E, neg);
    if (P != 0) {
      if (!anchored) {
        e_lo = E - es - kAnchorBit;
        anchored = true;
      }
      int p = E - 63 - es - e_lo;
      if (p > kMaxLsb) {
        shr192(acc[0], acc[1], acc[2], p - kMaxLsb);
        e_lo += p - kMaxLsb;
        p = kMaxLsb;
      }
      acc_add(acc[0], acc[1], acc[2], P, p, neg ^ (unsigned)(g & 1u));
    }
  }
}

__device__ __forceinline__ void write_real(const BatchArgs& a, int b, const FxMat& t, dd v, bool bad) {
  if (bad) {
    a.out[b] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  v = normalise_fx(v, t.n, t.m);
  a.out[b] = __dadd_rn(v.hi, v.lo);
}

template <int N, int K>
__global__ void __launch_bounds__(128) batched_fxr_kernel(BatchArgs a, ClassWork c) {
  const int lane = threadIdx.x & 31;
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(c.counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= c.nitems) break;
    const BatchItem it = c.items[item];
    const int b = a.order[it.first];
    const FxMat t = fxmat_of(a, b);
    if (t.m == 0) {
      if (lane == 0) a.out[b] = 1.0;
      continue;
    }
    const int e_sum = a.fx_esum[b];
    const bool bad = e_sum == kFxBad;
    const uint64_t terms = 1ull << (t.n - 1);
    uint64_t g0, len0, g, len;
    split_range(0, terms, (uint64_t)it.parts, (uint64_t)it.count, &g0, &len0);
    split_range(g0, g0 + len0, 32, (uint64_t)lane, &g, &len);
    dd v{0.0, 0.0};
    if (!bad) {
      u64 acc[3];
      int e_lo = 0;
      fxr_slice<N, K>(a.fx_table + a.fx_offset[b], t.n, e_sum, g, len, acc, e_lo);
      v = to_dd(acc[0], acc[1], acc[2], e_lo);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = dd_add(v, shfl_down_dd(v, o));
    if (lane == 0) {
      if (it.parts == 1) {
        write_real(a, b, t, v, bad);
      } else {
        double* slot = a.partials + 4 * ((int64_t)a.part_base[b] + it.count);
        slot[0] = v.hi;
        slot[1] = v.lo;
        slot[2] = 0.0;
        slot[3] = 0.0;
        __threadfence();
        const int arrived = atomicAdd(a.done + b, 1);
        if (arrived == it.parts - 1) {
          __threadfence();
          const volatile double* p = a.partials + 4 * (int64_t)a.part_base[b];
          dd sr{0.0, 0.0};
          for (int k = 0; k < it.parts; ++k) sr = dd_add(sr, dd{p[4 * k], p[4 * k + 1]});
          write_real(a, b, t, sr, bad);
        }
      }
    }
  }
}

// Columns per product on the FP64 unit when the tuner takes the FP64 share: about
// 3/8 of the padded order (the class's smallest order, npad - 3, exceeds it).
constexpr int fp64_columns(int npad) { return (3 * npad / 8) & ~1; }

template <int N>
void* kernel_for(bool share) {
  return share ? (void*)batched_cfx_kernel<N, fp64_columns(N)> : (void*)batched_cfx_kernel<N, 0>;
}

// real: 4 columns (6 from N = 32) on the FP64 unit with the share, as the square sweep
constexpr int fp64_columns_real(int npad) { return npad >= 32 ? 6 : 4; }

template <int N>
void* kernel_for_real(bool share) {
  return share ? (void*)batched_fxr_kernel<N, fp64_columns_real(N)> : (void*)batched_fxr_kernel<N, 0>;
}

void* pick_real(int npad, bool share) {
  switch (npad) {
    case 16: return kernel_for_real<16>(share);
    case 20: return kernel_for_real<20>(share);
    case 24: return kernel_for_real<24>(share);
    case 28: return kernel_for_real<28>(share);
    case 32: return kernel_for_real<32>(share);
    default: return nullptr;
  }
}

void* pick(int npad, bool share) {
  switch (npad) {
    case 12: return kernel_for<12>(share);
    case 16: return kernel_for<16>(share);
    case 20: return kernel_for<20>(share);
    case 24: return kernel_for<24>(share);
    case 28: return kernel_for<28>(share);
    case 32: return kernel_for<32>(share);
    default: return nullptr;
  }
}

}  // namespace

bool batched_fx_has_class(int dtype, int npad) {
  return (dtype == 1 ? pick(npad, false) : pick_real(npad, false)) != nullptr;
}

int batched_fx_blocks_per_sm(int dtype, int npad, int block, bool share) {
  void* k = dtype == 1 ? pick(npad, share) : pick_real(npad, share);
  if (!k) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, 0) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_batched_fx_prep(const BatchArgs& a, int dtype, const int32_t* list, int count, cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  const int warps_per_block = 4;
  const int grid = (count + warps_per_block - 1) / warps_per_block;
  if (dtype == 1)
    batched_cfx_prep_kernel<<<grid, 32 * warps_per_block, 0, stream>>>(a, list, count);
  else
    batched_fxr_prep_kernel<<<grid, 32 * warps_per_block, 0, stream>>>(a, list, count);
  return cudaGetLastError();
}

cudaError_t launch_batched_fx(const BatchArgs& a, const ClassWork& c, int dtype, int npad, const LaunchCfg& lc,
                              bool share) {
  void* k = dtype == 1 ? pick(npad, share) : pick_real(npad, share);
  if (!k) return cudaErrorInvalidValue;
  BatchArgs args = a;
  ClassWork cw = c;
  void* params[] = {&args, &cw};
  return cudaLaunchKernel(k, dim3(lc.grid), dim3(lc.block), params, 0, lc.stream);
}

}  // namespace perm
