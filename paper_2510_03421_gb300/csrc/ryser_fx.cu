// Ryser's formula for real input on the integer pipes (Eq. ryser_square; for m < n the
// subset-size form of Eq. ryser_rectangle): the 2^n column subsets in reflected Gray
// order, subset(g) = set bits of gray(g) = g ^ (g >> 1) (bit c <-> column c), each
// weighted by (-1)^(m-s) C(n-s, m-s) for s = |S| <= m (zero above m).
//
// Arithmetic as in glynn_fx.cu, with rows in place of columns:
//   * row i in fixed point with its own scale 2^e_i, sum_j |a_ij| 2^e_i < 2^61, each
//     a_ij rounded once to q_ij; a Gray step adds or removes one column, an exact int64
//     update of the m row sums (the table row of column j is read as a broadcast: all
//     lanes of a warp take the same step);
//   * the product of the m row sums as a software float with a 64-bit mantissa
//     (fixed_common.cuh, pairs of rows), multiplied by the exact 64-bit binomial weight;
//   * the signed terms go into a 192-bit fixed-point accumulator per thread.
// Subsets with more than m columns (weight 0) and the empty subset cost only the row
// update.  A whole sweep hands the chunks to the lanes in a size-coherent order (see
// coherent_chunk): the 32 lanes of a warp then see the same subset size at every step,
// so a warp skips the product together instead of paying for it whenever any lane
// needs one, and chunks whose subsets all exceed m columns are skipped.  The error-bound variant (ABS) takes exact magnitudes, adds up sum |term|
// and, when some entry was rounded to fixed point, the products of (|R_i| + n/2 units)
// that bound the effect of that rounding.
#include "device_common.cuh"
#include "fixed_common.cuh"
#include "internal.h"

namespace perm {

namespace {

// One block, one thread per row: row scales and the table of q (column-major).
__global__ void ryser_fx_prep_kernel(SweepArgs a, FxTable* tab) {
  const int n = a.n, m = a.m;
  const double* A = static_cast<const double*>(a.A);
  __shared__ int es[64];
  __shared__ int bad, inexact;
  if (threadIdx.x == 0) {
    bad = 0;
    inexact = 0;
  }
  __syncthreads();
  const int i = threadIdx.x;
  if (i < m) {
    double rowabs = 0.0, scaled = 0.0;
    for (int j = 0; j < n; ++j) {
      const double v = A[i * a.rs + j * a.cs];
      if (!isfinite(v)) bad = 1;
      rowabs += fabs(v);
      scaled += ldexp(fabs(v), -64);
    }
    int x = 0;
    if (rowabs > 0.0 && isfinite(rowabs)) {
      frexp(rowabs, &x);  // rowabs < 2^x
    } else if (scaled > 0.0 && isfinite(scaled)) {
      frexp(scaled, &x);
      x += 64;
    }
    const int e = 61 - x;
    es[i] = e;
    for (int j = 0; j < n; ++j) {
      const double s = ldexp(A[i * a.rs + j * a.cs], e);
      if (isfinite(s) && rint(s) != s) inexact = 1;
      tab->d[j * 64 + i] = isfinite(s) ? llrint(s) : 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int esum = 0;
    for (int k = 0; k < m; ++k) esum += es[k];
    tab->e_sum = esum;
    tab->e_max = 0;
    tab->bad = bad;
    tab->inexact = inexact;
  }
}

// Chunk of work item `item` in the size-coherent order: chunk c = gray^-1(x) where x runs
// over the (nb)-bit numbers by popcount h (h = 0, 1, ...) and, within one popcount, in
// colex order (combinatorial number system).  For g in chunk c (chunks of 2^k terms)
// the bits of gray(g) above k - 1 are those of gray(c) = x, and bit k - 1 is c_0 ^ g_{k-1}
// with c_0 = parity of x = h mod 2; so lanes holding chunks of one popcount h see the
// same subset size at every step.  cum[h] = number of items of popcount < h.
__device__ __forceinline__ uint64_t coherent_chunk(uint64_t item, int nb, const unsigned long long* cum, int* h_out) {
  int h = 0;
  while (h < nb && cum[h + 1] <= item) ++h;
  unsigned long long t = item - cum[h];
  // colex unranking: the largest p with C(p, i) <= t holds element i, for i = h .. 1
  unsigned __int128 b = 1;  // C(nb - 1, h)
  for (int q = 1; q <= h; ++q) b = b * (unsigned __int128)(nb - 1 - h + q) / (unsigned __int128)q;
  uint64_t x = 0;
  int i = h;
  for (int p = nb - 1; p >= 0 && i > 0; --p) {
    // b = C(p, i)
    if ((unsigned __int128)t >= b) {
      x |= 1ull << p;
      t -= (unsigned long long)b;
      b = p > 0 ? b * (unsigned __int128)i / (unsigned __int128)p : 0;  // C(p - 1, i - 1)
      --i;
    } else {
      b = p > 0 ? b * (unsigned __int128)(p - i) / (unsigned __int128)p : 0;  // C(p - 1, i)
    }
  }
  uint64_t c = x;  // inverse Gray code: prefix XOR from the top
  c ^= c >> 1;
  c ^= c >> 2;
  c ^= c >> 4;
  c ^= c >> 8;
  c ^= c >> 16;
  c ^= c >> 32;
  *h_out = h;
  return c;
}

template <int N, bool ABS>
__global__ void __launch_bounds__((N <= 36) ? 192 : 128, 2) ryser_fx_kernel(SweepArgs a, const FxTable* __restrict__ tab) {
  extern __shared__ long long smem_rf[];
  __shared__ dd scratch[3 * 32];
  __shared__ u64 s_wm[65];  // |weight of size s| = s_wm[s] 2^(s_we[s] - 64), normalised (0: weight 0)
  __shared__ int s_we[65];
  const int n = a.n, m = a.m;
  long long* sQ = smem_rf;  // q_ij at sQ[j * N + i]
  for (int idx = threadIdx.x; idx < n * N; idx += blockDim.x) {
    const int j = idx / N, i = idx - j * N;
    sQ[idx] = (i < m) ? tab->d[j * 64 + i] : 0;
  }
  for (int s = threadIdx.x; s <= n; s += blockDim.x) {
    if (s == 0 || s > m) {
      s_wm[s] = 0;
      s_we[s] = 0;
    } else {
      const u64 c = binom_u64(n - s, m - s);
      const int lz = __clzll((long long)c);
      s_wm[s] = c << lz;
      s_we[s] = 64 - lz;
    }
  }
  // size-coherent chunk order for whole sweeps (start_mode == 1 from the host): cum[h] =
  // sum_{h' < h} C(nb, h'), nb = n - chunk_log2 bits of chunk index
  __shared__ unsigned long long s_cum[66];
  const bool coherent = a.start_mode == 1;
  const int nb = n - a.chunk_log2;
  if (coherent && threadIdx.x == 0) {
    unsigned long long run = 0, b = 1;  // b = C(nb, h)
    for (int h = 0; h <= nb + 1 && h < 66; ++h) {
      s_cum[h] = run;
      if (h <= nb) {
        run += b;
        b = (unsigned long long)((unsigned __int128)b * (unsigned __int128)(nb - h) / (unsigned __int128)(h + 1));
      }
    }
  }
  const int e_sum = tab->e_sum + 31 * (N - m);  // padded rows hold 2^31 = 1 * 2^31
  // bound variant with inexact quantisation: a row sum of up to n rounded entries is
  // off by at most n/2 units
  const bool use_eta = ABS && tab->inexact != 0;
  const long long eta = (n + 1) / 2;
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const uint64_t L = 1ull << a.chunk_log2;
  const uint64_t c_first = a.g_begin >> a.chunk_log2;
  const uint64_t c_end = (a.g_end + L - 1) >> a.chunk_log2;
  const uint64_t rounds = (c_end - c_first + 31) / 32;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);

  int e_lo = 0;
  bool anchored = false;
  u64 a0 = 0, a1 = 0, a2 = 0;
  u64 b0 = 0, b1 = 0, b2 = 0;
  u64 c0 = 0, c1 = 0, c2 = 0;
  auto add_term = [&](u64& x0, u64& x1, u64& x2, u64 P, int E, unsigned neg) {
    if (!anchored) {
      e_lo = E - e_sum - kAnchorBit;
      anchored = true;
    }
    int p = E - 63 - e_sum - e_lo;
    if (p > kMaxLsb) {
      shr192(a0, a1, a2, p - kMaxLsb);
      if (ABS) {
        shr192(b0, b1, b2, p - kMaxLsb);
        shr192(c0, c1, c2, p - kMaxLsb);
      }
      e_lo += p - kMaxLsb;
      p = kMaxLsb;
    }
    if (p >= 0) {
      acc_add_nb(x0, x1, x2, P, p, neg);  // no divergence on the sign or the position
    } else {
      acc_add(x0, x1, x2, P, p, neg);
    }
  };
  // the weight of size s times P 2^E, renormalised
  auto weigh = [&](u64& P, int& E, int s) {
    const u64 h2 = __umul64hi(P, s_wm[s]);
    const int top = (int)(h2 >> 63);
    P = top ? h2 : (h2 << 1);
    E += s_we[s] - 1 + top;
  };
  long long R[N];
  int size = 0;
  for (uint64_t r = warp; r < rounds; r += warps) {
    uint64_t chunk = c_first + 32 * r + lane;
    bool skip = chunk >= c_end;
    if (coherent && !skip) {
      int h;
      chunk = coherent_chunk(chunk, nb, s_cum, &h);
      // every subset of the chunk has at least h columns: nothing to add above m
      skip = h > m;
    }
    uint64_t ga = chunk << a.chunk_log2, gb = ga + L;
    if (ga < a.g_begin) ga = a.g_begin;
    if (gb > a.g_end) gb = a.g_end;
    if (skip) ga = gb = a.g_end;  // idle lane
    for (uint64_t g = ga; g < gb; ++g) {
      if (g == ga) {
        const uint64_t gray = g ^ (g >> 1);
#pragma unroll
        for (int i = 0; i < N; ++i) R[i] = 0;
        for (int j = 0; j < n; ++j) {
          if (!((gray >> j) & 1u)) continue;
          const long long* col = sQ + j * N;
#pragma unroll
          for (int i = 0; i < N; ++i) R[i] += col[i];
        }
#pragma unroll
        for (int i = 0; i < N; ++i)
          if (i >= m) R[i] = 1ll << 31;
        size = __popcll(gray);
      } else {
        // column b = ctz(g) joins when bit b+1 of g is 0 (bit b of gray(g) becomes 1)
        const int b = ctz64(g);
        const long long* col = sQ + b * N;
        if ((g >> (b + 1)) & 1u) {
#pragma unroll
          for (int i = 0; i < N; ++i)
            if (i < m) R[i] -= col[i];
          --size;
        } else {
#pragma unroll
          for (int i = 0; i < N; ++i)
            if (i < m) R[i] += col[i];
          ++size;
        }
      }
      if (s_wm[size] == 0) continue;  // empty subset or more than m columns
      u64 P;
      int E;
      unsigned neg;
      soft_product<N, 0, ABS>(R, P, E, neg);  // exact magnitudes in the bound variant
      if (P != 0) {
        weigh(P, E, size);
        add_term(a0, a1, a2, P, E, neg ^ (unsigned)((m - size) & 1));
        if (ABS) add_term(b0, b1, b2, P, E, 0u);
      }
      if (use_eta) {
        u64 Pe;
        int Ee;
        soft_product_eta<N, 0>(R, m, eta, Pe, Ee);
        if (Pe != 0) {
          weigh(Pe, Ee, size);
          add_term(c0, c1, c2, Pe, Ee, 0u);
        }
      }
    }
  }

  // records {sum, sum |term|, eta-widened sum} (the last two with ABS only)
  dd v[3] = {to_dd(a0, a1, a2, e_lo), ABS ? to_dd(b0, b1, b2, e_lo) : dd{0.0, 0.0},
             use_eta ? to_dd(c0, c1, c2, e_lo) : dd{0.0, 0.0}};
  block_sum_dd<3>(v, scratch);
  if (threadIdx.x == 0) {
    double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * (ABS ? kCplxRecord : kRealRecord);
    const bool bad = tab->bad != 0;
    rec[0] = bad ? __longlong_as_double(0x7ff8000000000000ll) : v[0].hi;
    rec[1] = bad ? 0.0 : v[0].lo;
    rec[2] = v[1].hi;
    rec[3] = v[1].lo;
    if (ABS) {
      rec[4] = v[2].hi;
      rec[5] = v[2].lo;
    }
  }
}

template <int N>
void* kernel_for(bool abs) {
  return abs ? (void*)ryser_fx_kernel<N, true> : (void*)ryser_fx_kernel<N, false>;
}

void* pick(int m, bool abs) {
  switch ((m + 3) & ~3) {
    case 4: return kernel_for<4>(abs);
    case 8: return kernel_for<8>(abs);
    case 12: return kernel_for<12>(abs);
    case 16: return kernel_for<16>(abs);
    case 20: return kernel_for<20>(abs);
    case 24: return kernel_for<24>(abs);
    case 28: return kernel_for<28>(abs);
    case 32: return kernel_for<32>(abs);
    case 36: return kernel_for<36>(abs);
    case 40: return kernel_for<40>(abs);
    case 44: return kernel_for<44>(abs);
    case 48: return kernel_for<48>(abs);
    case 52: return kernel_for<52>(abs);
    case 56: return kernel_for<56>(abs);
    case 60: return kernel_for<60>(abs);
    case 64: return kernel_for<64>(abs);
    default: return nullptr;
  }
}

size_t smem_bytes(int m, int n) { return (size_t)n * (size_t)((m + 3) & ~3) * sizeof(long long); }

}  // namespace

int ryser_fx_block(int m) { return ((m + 3) & ~3) <= 36 ? 192 : 128; }

int ryser_fx_blocks_per_sm(int m, int n, int block, bool want_abs) {
  void* k = pick(m, want_abs);
  if (!k) return 0;
  const size_t smem = smem_bytes(m, n);
  if (smem > 32 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_ryser_fx(const SweepArgs& a, FxTable* tab, const LaunchCfg& c, bool want_abs) {
  if (a.m < 1 || a.m > a.n || a.n > 62) return cudaErrorInvalidValue;
  void* k = pick(a.m, want_abs);
  if (!k) return cudaErrorInvalidValue;
  ryser_fx_prep_kernel<<<1, 64, 0, c.stream>>>(a, tab);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = smem_bytes(a.m, a.n);
  if (smem > 32 * 1024) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  SweepArgs args = a;
  const FxTable* tp = tab;
  void* params[] = {&args, &tp};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), params, smem, c.stream);
}

}  // namespace perm
