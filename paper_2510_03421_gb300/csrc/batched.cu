// Batched Glynn (Eq. glynn, Eq. glynn_rectangle) for many small real or complex
// matrices, one persistent kernel per size class.
//
// The host sorts the matrices into classes by padded order N (a multiple of 4) and
// builds a work list per class, longest items first:
//   * warp items (larger matrices): a matrix's 2^(n-1) terms are cut into K equal
//     sub-ranges of at most 2^item_log2 terms; one warp sums one sub-range, its 32
//     lanes taking contiguous slices (exact rebuild of the column sums at each slice
//     start and every 2^chunk_log2 terms).  The warp writes a double-double partial;
//     the warp that completes a matrix's K-th sub-range (per-matrix arrival counter,
//     no waiting) sums the K partials in a fixed order, normalises by
//     2^(n-1) (n-m)! and writes the permanent;
//   * lane items (small matrices): 32 matrices of one class, one per lane, each
//     summed whole by its lane.
// Resident warps of a class kernel take items from the class counter (atomicAdd).
// The class kernels are launched on parallel branches of one captured CUDA graph,
// so the tail of one class overlaps the others.  Update rows are read from the
// packed input (L1-resident) with fma(+-2, a, S); rows of the virtual padding are ones.
#include "device_common.cuh"
#include "internal.h"

namespace perm {
namespace {

__device__ __forceinline__ void kahan_add(double& acc, double& comp, double x) {
  const double y = __dsub_rn(x, comp);
  const double s = __dadd_rn(acc, y);
  comp = __dsub_rn(__dsub_rn(s, acc), y);
  acc = s;
}

struct Mat {
  int64_t off, rs, cs;
  int m, n;
};

// Shape of matrix b after the transpose rule per(A) = per(A^T) for m > n.
__device__ __forceinline__ Mat mat_of(const BatchArgs& a, int b) {
  Mat t;
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

// Sum of the Glynn terms [g, g + len) of one matrix (unnormalised), compensated.
template <int N, int W>
__device__ __forceinline__ void glynn_slice(const double* __restrict__ packed, const Mat& t, uint64_t g, uint64_t len,
                                            int chunk_log2, dd& out_re, dd& out_im) {
  double Sr[N], Si[N];
  double accr = 0.0, cr = 0.0, acci = 0.0, ci = 0.0;
  const uint64_t mask = (1ull << chunk_log2) - 1;
  const int m = t.m, n = t.n;
  for (uint64_t s = 0; s < len; ++s, ++g) {
    if (s == 0 || (g & mask) == 0) {
      const uint64_t gray = g ^ (g >> 1);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        Sr[j] = (j < n) ? 0.0 : 1.0;
        Si[j] = 0.0;
      }
      for (int i = 0; i < n; ++i) {
        const double sg = ((gray >> (n - 1 - i)) & 1u) ? -1.0 : 1.0;
        const double* row = packed + W * (t.off + i * t.rs);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          if (j < n) {
            const double re = (i < m) ? row[W * j * t.cs] : 1.0;
            Sr[j] = __fma_rn(sg, re, Sr[j]);
            if (W == 2) Si[j] = __fma_rn(sg, (i < m) ? row[W * j * t.cs + 1] : 0.0, Si[j]);
          }
        }
      }
    } else {
      const int b = ctz64(g);
      const int r = n - 1 - b;
      const double sg = ((g >> (b + 1)) & 1u) ? 2.0 : -2.0;
      const double* row = packed + W * (t.off + r * t.rs);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        if (j < n) {
          const double re = (r < m) ? row[W * j * t.cs] : 1.0;
          Sr[j] = __fma_rn(sg, re, Sr[j]);
          if (W == 2) Si[j] = __fma_rn(sg, (r < m) ? row[W * j * t.cs + 1] : 0.0, Si[j]);
        }
      }
    }
    double pr = Sr[0], pi = Si[0];
#pragma unroll
    for (int j = 1; j < N; ++j) {
      if (W == 2) {
        const double nr = __fma_rn(pr, Sr[j], -__dmul_rn(pi, Si[j]));
        const double ni = __fma_rn(pr, Si[j], __dmul_rn(pi, Sr[j]));
        pr = nr;
        pi = ni;
      } else {
        pr = __dmul_rn(pr, Sr[j]);
      }
    }
    if (g & 1u) {
      pr = -pr;
      pi = -pi;
    }
    kahan_add(accr, cr, pr);
    if (W == 2) kahan_add(acci, ci, pi);
  }
  out_re = two_sum(accr, -cr);
  out_im = two_sum(acci, -ci);
}

__device__ __forceinline__ dd normalise(dd v, int n, int m) {
  v = dd_ldexp(v, -(n - 1));
  for (int k = 2; k <= n - m; ++k) v = dd_div_d(v, (double)k);
  return v;
}

template <int W>
__device__ __forceinline__ void write_result(const BatchArgs& a, int b, const Mat& t, dd vr, dd vi) {
  double* out = a.out + W * (int64_t)b;
  if (t.m == 0) {
    out[0] = 1.0;
    if (W == 2) out[1] = 0.0;
    return;
  }
  vr = normalise(vr, t.n, t.m);
  out[0] = __dadd_rn(vr.hi, vr.lo);
  if (W == 2) {
    vi = normalise(vi, t.n, t.m);
    out[1] = __dadd_rn(vi.hi, vi.lo);
  }
}

template <int N, int W, bool LANE>
__global__ void __launch_bounds__(128) batched_class_kernel(BatchArgs a, ClassWork c) {
  const int lane = threadIdx.x & 31;
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(c.counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= c.nitems) break;
    const BatchItem it = c.items[item];
    if (LANE) {
      if (lane < it.count) {
        const int b = a.order[it.first + lane];
        const Mat t = mat_of(a, b);
        dd vr{0.0, 0.0}, vi{0.0, 0.0};
        if (t.m > 0) glynn_slice<N, W>(a.packed, t, 0, 1ull << (t.n - 1), a.chunk_log2, vr, vi);
        write_result<W>(a, b, t, vr, vi);
      }
    } else {
      const int b = a.order[it.first];
      const Mat t = mat_of(a, b);
      dd vr{0.0, 0.0}, vi{0.0, 0.0};
      if (t.m > 0) {
        // sub-range it.count of it.parts, then this lane's slice of it
        uint64_t g0, len0, g, len;
        split_range(0, 1ull << (t.n - 1), (uint64_t)it.parts, (uint64_t)it.count, &g0, &len0);
        split_range(g0, g0 + len0, 32, (uint64_t)lane, &g, &len);
        glynn_slice<N, W>(a.packed, t, g, len, a.chunk_log2, vr, vi);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          vr = dd_add(vr, shfl_down_dd(vr, o));
          vi = dd_add(vi, shfl_down_dd(vi, o));
        }
      }
      if (lane == 0) {
        if (it.parts == 1) {
          write_result<W>(a, b, t, vr, vi);
        } else {
          double* slot = a.partials + 4 * ((int64_t)a.part_base[b] + it.count);
          slot[0] = vr.hi;
          slot[1] = vr.lo;
          slot[2] = vi.hi;
          slot[3] = vi.lo;
          __threadfence();
          const int arrived = atomicAdd(a.done + b, 1);
          if (arrived == it.parts - 1) {  // the last sub-range of matrix b: combine
            __threadfence();
            const volatile double* p = a.partials + 4 * (int64_t)a.part_base[b];
            dd sr{0.0, 0.0}, si{0.0, 0.0};
            for (int k = 0; k < it.parts; ++k) {
              sr = dd_add(sr, dd{p[4 * k], p[4 * k + 1]});
              si = dd_add(si, dd{p[4 * k + 2], p[4 * k + 3]});
            }
            write_result<W>(a, b, t, sr, si);
          }
        }
      }
    }
  }
}

template <int W, bool LANE>
void* class_kernel(int npad) {
  switch (npad) {
    case 4: return (void*)batched_class_kernel<4, W, LANE>;
    case 8: return (void*)batched_class_kernel<8, W, LANE>;
    case 12: return (void*)batched_class_kernel<12, W, LANE>;
    case 16: return (void*)batched_class_kernel<16, W, LANE>;
    case 20: return LANE ? nullptr : (void*)batched_class_kernel<20, W, false>;
    case 24: return LANE ? nullptr : (void*)batched_class_kernel<24, W, false>;
    case 28: return LANE ? nullptr : (void*)batched_class_kernel<28, W, false>;
    case 32: return LANE ? nullptr : (void*)batched_class_kernel<32, W, false>;
    default: return nullptr;
  }
}

void* pick(int dtype, int npad, bool lane) {
  if (dtype == 1) return lane ? class_kernel<2, true>(npad) : class_kernel<2, false>(npad);
  return lane ? class_kernel<1, true>(npad) : class_kernel<1, false>(npad);
}

}  // namespace

int batched_blocks_per_sm(int dtype, int npad, bool lane, int block) {
  void* k = pick(dtype, npad, lane);
  if (!k) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, 0) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_batched_class(const BatchArgs& a, const ClassWork& c, int dtype, int npad, bool lane,
                                 const LaunchCfg& lc) {
  void* k = pick(dtype, npad, lane);
  if (!k) return cudaErrorInvalidValue;
  BatchArgs args = a;
  ClassWork cw = c;
  void* params[] = {&args, &cw};
  return cudaLaunchKernel(k, dim3(lc.grid), dim3(lc.block), params, 0, lc.stream);
}

}  // namespace perm
