// The combinatoric algorithm: the definition (Eq. rectangular_permanent_definition)
// summed over all injective maps sigma: rows -> columns, cost O(m n!/(n-m)!).
//
// The maps are split by their first d rows: prefix r (0 <= r < n!/(n-d)!) is read as
// mixed-radix digits choosing, for rows 0..d-1 in turn, the digit-th still unused
// column.  A thread takes prefixes in a grid-stride loop; a prefix whose product is
// zero is skipped, and below it a depth-first search visits the remaining rows with
// a bitmask of the columns still free and of the row's nonzero entries, so zero
// entries prune whole subtrees.  The search evaluates each subtree bottom-up
// (value(row k) = sum over free columns c of a_kc * value(row k+1)), so rounding
// grows with the depth of the tree, not with the number of leaves.  Prefix values are
// combined in a Kahan sum (real, complex) or modulo 2^128 (integer; Gaussian integers
// per part).
//
// The last rows: below a node with r rows left, the subtree's value depends only on
// the set of free columns.  For n <= 16 (not for Gaussian integers) the block first
// tabulates, for every column triple S (colex rank x + C(y,2) + C(z,3), x < y < z),
// the permanent of the last three rows on S -- the sum of the six leaf products the
// search would form -- from m = 5, for every column quadruple, the permanent of the
// last four rows on it, formed from the triples' table the way the search combines a
// row with the rows below (sum over c in S of a_{m-4,c} T3[S - c]), and, for real
// input from m = 6, the same for the last five rows on every quintuple.  The search
// stops where the tables take over: with six free columns (a square) each nonzero
// free column of the sixth-last row times the five-row entry of the other five, found
// from their colex ranks; otherwise with five rows left, each free column times the
// four-row entries of the rest (one entry for a square).  The tables remove the five
// or six deepest levels of the tree, which hold all but a 120th (720th) of its nodes.
#include <type_traits>

#include "device_common.cuh"
#include "internal.h"

namespace perm {
namespace {

typedef unsigned __int128 u128;

struct RealF {
  typedef double T;
  __device__ static T zero() { return 0.0; }
  __device__ static T one() { return 1.0; }
  __device__ static T load(const void* A, int64_t e) { return static_cast<const double*>(A)[e]; }
  __device__ static bool is_zero(T x) { return x == 0.0; }
  __device__ static T mul(T a, T b) { return __dmul_rn(a, b); }
  __device__ static T fma(T a, T b, T c) { return __fma_rn(a, b, c); }
  __device__ static T add(T a, T b) { return __dadd_rn(a, b); }
};

struct CplxF {
  typedef double2 T;
  __device__ static T zero() { return make_double2(0.0, 0.0); }
  __device__ static T one() { return make_double2(1.0, 0.0); }
  __device__ static T load(const void* A, int64_t e) {
    const double* p = static_cast<const double*>(A) + 2 * e;
    return make_double2(p[0], p[1]);
  }
  __device__ static bool is_zero(T x) { return x.x == 0.0 && x.y == 0.0; }
  __device__ static T mul(T a, T b) {
    return make_double2(__fma_rn(a.x, b.x, -__dmul_rn(a.y, b.y)), __fma_rn(a.x, b.y, __dmul_rn(a.y, b.x)));
  }
  __device__ static T fma(T a, T b, T c) {
    T p = mul(a, b);
    return make_double2(__dadd_rn(p.x, c.x), __dadd_rn(p.y, c.y));
  }
  __device__ static T add(T a, T b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
};

template <typename E>
struct IntF {
  typedef u128 T;
  __device__ static T zero() { return 0; }
  __device__ static T one() { return 1; }
  __device__ static T load(const void* A, int64_t e) { return (u128)(__int128)(long long)static_cast<const E*>(A)[e]; }
  __device__ static bool is_zero(T x) { return x == 0; }
  __device__ static T mul(T a, T b) { return a * b; }
  __device__ static T fma(T a, T b, T c) { return a * b + c; }
  __device__ static T add(T a, T b) { return a + b; }
};

// Gaussian integers: both parts modulo 2^128
struct GaussT {
  u128 re, im;
};

struct GaussF {
  typedef GaussT T;
  __device__ static T zero() { return T{0, 0}; }
  __device__ static T one() { return T{1, 0}; }
  __device__ static T load(const void* A, int64_t e) {
    const long long* p = static_cast<const long long*>(A) + 2 * e;
    return T{(u128)(__int128)p[0], (u128)(__int128)p[1]};
  }
  __device__ static bool is_zero(T x) { return x.re == 0 && x.im == 0; }
  __device__ static T mul(T a, T b) { return T{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
  __device__ static T fma(T a, T b, T c) {
    const T p = mul(a, b);
    return T{p.re + c.re, p.im + c.im};
  }
  __device__ static T add(T a, T b) { return T{a.re + b.re, a.im + b.im}; }
};

constexpr int kMaxN = 64;

// Compensated accumulation of prefix values.
__device__ __forceinline__ void kahan(double& acc, double& comp, double x) {
  const double y = __dsub_rn(x, comp);
  const double s = __dadd_rn(acc, y);
  comp = __dsub_rn(__dsub_rn(s, acc), y);
  acc = s;
}

constexpr int kTailN = 16;  // column count up to which the tail tables are built

// C(c, k) for small c, k by the product formula (after step i, r = C(c, i + 1); exact),
// without recursion so that the kernel's stack size stays statically known
__host__ __device__ constexpr int binom_small(int c, int k) {
  long long r = 1;
  for (int i = 0; i < k; ++i) r = r * (c - i) / (i + 1);
  return c < k ? 0 : (int)r;
}

template <class F>
__global__ void __launch_bounds__(256) combinatoric_kernel(SweepArgs a, int depth, uint64_t prefixes, int tail) {
  typedef typename F::T T;
  extern __shared__ unsigned char smem_c[];
  __shared__ unsigned long long rowmask[kMaxN];
  __shared__ int sB[6][kTailN + 1];  // sB[k][c] = C(c, k): colex ranks of column sets
  const int n = a.n, m = a.m;
  T* sA = reinterpret_cast<T*>(smem_c);  // sA[i * n + j]
  T* sT3 = sA + m * n;              // last three rows on triple rank x + C(y,2) + C(z,3)
  T* sT4 = sT3 + binom_small(n, 3); // last four rows on quadruple rank ... + C(w,4)
  T* sT5 = sT4 + binom_small(n, 4); // last five rows on quintuple rank (tail == 2)
  const bool tail4 = tail && m >= 5;
  const bool tail5 = tail == 2 && m >= 6;
  for (int idx = threadIdx.x; idx < m * n; idx += blockDim.x) {
    const int i = idx / n, j = idx - i * n;
    sA[idx] = F::load(a.A, i * a.rs + j * a.cs);
  }
  for (int idx = threadIdx.x; idx < 6 * (kTailN + 1); idx += blockDim.x) {
    const int k = idx / (kTailN + 1), c = idx - k * (kTailN + 1);
    sB[k][c] = binom_small(c, k);
  }
  __syncthreads();
  if (tail) {
    const T* r0 = sA + (m - 3) * n;
    const T* r1 = sA + (m - 2) * n;
    const T* r2 = sA + (m - 1) * n;
    for (int idx = threadIdx.x; idx < sB[3][n]; idx += blockDim.x) {
      // colex unranking: z the largest column with C(z,3) <= idx, then y, then x
      int rem = idx, z = 2, y = 1;
      while (z + 1 < n && sB[3][z + 1] <= rem) ++z;
      rem -= sB[3][z];
      while (y + 1 < z && sB[2][y + 1] <= rem) ++y;
      const int x = rem - sB[2][y];
      // the six orderings of (x, y, z) over rows r0, r1, r2
      T v = F::mul(r0[x], F::add(F::mul(r1[y], r2[z]), F::mul(r1[z], r2[y])));
      v = F::fma(r0[y], F::add(F::mul(r1[x], r2[z]), F::mul(r1[z], r2[x])), v);
      v = F::fma(r0[z], F::add(F::mul(r1[x], r2[y]), F::mul(r1[y], r2[x])), v);
      sT3[idx] = v;
    }
    __syncthreads();
    if (tail4) {
      const T* r = sA + (m - 4) * n;
      for (int idx = threadIdx.x; idx < sB[4][n]; idx += blockDim.x) {
        int rem = idx, w = 3, z = 2, y = 1;
        while (w + 1 < n && sB[4][w + 1] <= rem) ++w;
        rem -= sB[4][w];
        while (z + 1 < w && sB[3][z + 1] <= rem) ++z;
        rem -= sB[3][z];
        while (y + 1 < z && sB[2][y + 1] <= rem) ++y;
        const int x = rem - sB[2][y];
        // row m-4 on each column c of the quadruple, the last three rows on the rest
        T v = F::mul(r[x], sT3[y + sB[2][z] + sB[3][w]]);
        v = F::fma(r[y], sT3[x + sB[2][z] + sB[3][w]], v);
        v = F::fma(r[z], sT3[x + sB[2][y] + sB[3][w]], v);
        v = F::fma(r[w], sT3[x + sB[2][y] + sB[3][z]], v);
        sT4[idx] = v;
      }
      __syncthreads();
    }
    if (tail5) {
      const T* r = sA + (m - 5) * n;
      for (int idx = threadIdx.x; idx < sB[5][n]; idx += blockDim.x) {
        int c[5];
        int rem = idx, top = n;
#pragma unroll
        for (int j = 5; j >= 1; --j) {  // colex unranking, largest element first
          int p = j - 1;
          while (p + 1 < top && sB[j][p + 1] <= rem) ++p;
          rem -= sB[j][p];
          c[j - 1] = p;
          top = p;
        }
        // row m-5 on each column of the quintuple, the last four rows on the rest
        T v = F::zero();
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          int rank = 0, j = 1;
#pragma unroll
          for (int q = 0; q < 5; ++q)
            if (q != i) rank += sB[j++][c[q]];
          v = (i == 0) ? F::mul(r[c[0]], sT4[rank]) : F::fma(r[c[i]], sT4[rank], v);
        }
        sT5[idx] = v;
      }
      __syncthreads();
    }
  }
  const unsigned long long allcols = (n == 64) ? ~0ull : ((1ull << n) - 1);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    unsigned long long mk = 0;
    for (int j = 0; j < n; ++j)
      if (!F::is_zero(sA[i * n + j])) mk |= 1ull << j;
    rowmask[i] = mk;
  }
  __syncthreads();

  // per-thread accumulators: Kahan pairs for floating point, u128 for integers
  T acc = F::zero();
  double kr = 0.0, kcr = 0.0, ki = 0.0, kci = 0.0;
  // depth-first state (local memory)
  unsigned long long cand[kMaxN];
  int col[kMaxN];
  T val[kMaxN + 1];

  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < prefixes; r += stride) {
    // unrank the prefix (in 32-bit arithmetic when every prefix index fits: 64-bit
    // division by a run-time radix costs several times more)
    uint64_t rem = r;
    unsigned rem32 = (unsigned)r;
    const bool narrow = prefixes <= 0xffffffffull;
    unsigned long long used = 0;
    T pre = F::one();
    bool zero = false;
    for (int k = 0; k < depth; ++k) {
      const int radix = n - k;
      int digit;
      if (narrow) {
        digit = (int)(rem32 % (unsigned)radix);
        rem32 /= (unsigned)radix;
      } else {
        digit = (int)(rem % (uint64_t)radix);
        rem /= (uint64_t)radix;
      }
      unsigned long long freecols = ~used & ((n == 64) ? ~0ull : ((1ull << n) - 1));
      for (int t = 0; t < digit; ++t) freecols &= freecols - 1;
      const int c = __ffsll((long long)freecols) - 1;
      used |= 1ull << c;
      const T v = sA[k * n + c];
      if (F::is_zero(v)) zero = true;
      pre = F::mul(pre, v);
    }
    if (zero) continue;
    T sub;
    if (depth == m) {
      sub = F::one();
    } else {
      // value of rows depth..m-1 over the free columns, bottom-up
      int k = depth;
      cand[k] = rowmask[k] & ~used;
      val[k] = F::zero();
      // sums of the table entries over the triples / quadruples of the column set fm
      auto triples = [&](unsigned long long fm) {
        T s = F::zero();
        unsigned long long xm = fm;
        while (xm) {
          const int x = __ffsll((long long)xm) - 1;
          xm &= xm - 1;
          unsigned long long ym = xm;
          while (ym) {
            const int y = __ffsll((long long)ym) - 1;
            ym &= ym - 1;
            const int rxy = x + sB[2][y];
            unsigned long long zm = ym;
            while (zm) {
              const int z = __ffsll((long long)zm) - 1;
              zm &= zm - 1;
              s = F::add(s, sT3[rxy + sB[3][z]]);
            }
          }
        }
        return s;
      };
      auto quadruples = [&](unsigned long long fm) {
        T s = F::zero();
        unsigned long long xm = fm;
        while (xm) {
          const int x = __ffsll((long long)xm) - 1;
          xm &= xm - 1;
          unsigned long long ym = xm;
          while (ym) {
            const int y = __ffsll((long long)ym) - 1;
            ym &= ym - 1;
            const int rxy = x + sB[2][y];
            unsigned long long zm = ym;
            while (zm) {
              const int z = __ffsll((long long)zm) - 1;
              zm &= zm - 1;
              const int rxyz = rxy + sB[3][z];
              unsigned long long wm = zm;
              while (wm) {
                const int w = __ffsll((long long)wm) - 1;
                wm &= wm - 1;
                s = F::add(s, sT4[rxyz + sB[4][w]]);
              }
            }
          }
        }
        return s;
      };
      while (true) {
        if (tail5 && k == m - 6 && __popcll(allcols & ~used) == 6) {
          // six rows left with six free columns (a square): each nonzero free column
          // c_i of row k times the table entry of the other five, by their colex rank
          const unsigned long long fm = allcols & ~used;
          const unsigned long long xm = rowmask[k] & fm;
          unsigned long long r = fm;
          int c[6];
#pragma unroll
          for (int q = 0; q < 6; ++q) {
            c[q] = __ffsll((long long)r) - 1;
            r &= r - 1;
          }
          T s = F::zero();
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            if (!((xm >> c[i]) & 1ull)) continue;
            int rank = 0, j = 1;
#pragma unroll
            for (int q = 0; q < 6; ++q)
              if (q != i) rank += sB[j++][c[q]];
            s = F::fma(sA[k * n + c[i]], sT5[rank], s);
          }
          val[k] = s;
          cand[k] = 0;
        } else if (tail4 && k == m - 5) {
          // five rows left: each nonzero free column x of row k times the quadruple sum
          // over the rest, without descending
          const unsigned long long fm = allcols & ~used;
          unsigned long long xm = rowmask[k] & fm;
          T s = F::zero();
          if (__popcll(fm) == 5) {
            // five free columns c0 < .. < c4 (a square): the rest of c_i is one quadruple,
            // colex rank sum_j C(d_j, j + 1) over the other four in increasing order
            unsigned long long r = fm;
            int c[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
              c[q] = __ffsll((long long)r) - 1;
              r &= r - 1;
            }
#pragma unroll
            for (int i = 0; i < 5; ++i) {
              if (!((xm >> c[i]) & 1ull)) continue;
              int rank = 0, j = 1;
#pragma unroll
              for (int q = 0; q < 5; ++q)
                if (q != i) rank += sB[j++][c[q]];
              s = F::fma(sA[k * n + c[i]], sT4[rank], s);
            }
          } else {
            while (xm) {
              const int x = __ffsll((long long)xm) - 1;
              xm &= xm - 1;
              s = F::fma(sA[k * n + x], quadruples(fm & ~(1ull << x)), s);
            }
          }
          val[k] = s;
          cand[k] = 0;
        } else if (tail4 && k == m - 4) {
          val[k] = quadruples(allcols & ~used);
          cand[k] = 0;
        } else if (tail && k == m - 4) {
          const unsigned long long fm = allcols & ~used;
          unsigned long long xm = rowmask[k] & fm;
          T s = F::zero();
          while (xm) {
            const int x = __ffsll((long long)xm) - 1;
            xm &= xm - 1;
            s = F::fma(sA[k * n + x], triples(fm & ~(1ull << x)), s);
          }
          val[k] = s;
          cand[k] = 0;
        } else if (tail && k == m - 3) {
          // three rows left: the triples of free columns, from the table
          val[k] = triples(allcols & ~used);
          cand[k] = 0;
        } else if (k == m - 1) {
          T s = F::zero();
          unsigned long long cm = cand[k];
          while (cm) {
            const int c = __ffsll((long long)cm) - 1;
            cm &= cm - 1;
            s = F::add(s, sA[k * n + c]);
          }
          val[k] = s;
          cand[k] = 0;
        }
        if (cand[k] == 0) {
          if (k == depth) break;
          --k;  // return val[k+1] to the parent
          used &= ~(1ull << col[k]);
          val[k] = F::fma(sA[k * n + col[k]], val[k + 1], val[k]);
          continue;
        }
        const int c = __ffsll((long long)cand[k]) - 1;
        cand[k] &= cand[k] - 1;
        col[k] = c;
        used |= 1ull << c;
        ++k;
        cand[k] = rowmask[k] & ~used;
        val[k] = F::zero();
      }
      sub = val[depth];
    }
    const T contrib = F::mul(pre, sub);
    if constexpr (std::is_same_v<T, double>) {
      kahan(kr, kcr, contrib);
    } else if constexpr (std::is_same_v<T, double2>) {
      kahan(kr, kcr, contrib.x);
      kahan(ki, kci, contrib.y);
    } else {
      acc = F::add(acc, contrib);
    }
  }

  // block reduction into one record per block
  if constexpr (std::is_same_v<T, GaussT>) {
    // real parts at record blockIdx.x, imaginary parts at gridDim.x + blockIdx.x
    __shared__ u128 part[2][128];
    part[0][threadIdx.x] = acc.re;
    part[1][threadIdx.x] = acc.im;
    __syncthreads();
    if (threadIdx.x == 0) {
      u128 tr = 0, ti = 0;
      for (int i = 0; i < (int)blockDim.x; ++i) {
        tr += part[0][i];
        ti += part[1][i];
      }
      unsigned long long* rec = static_cast<unsigned long long*>(a.partials);
      rec[(size_t)blockIdx.x * kIntRecord] = (unsigned long long)tr;
      rec[(size_t)blockIdx.x * kIntRecord + 1] = (unsigned long long)(tr >> 64);
      rec[(size_t)(gridDim.x + blockIdx.x) * kIntRecord] = (unsigned long long)ti;
      rec[(size_t)(gridDim.x + blockIdx.x) * kIntRecord + 1] = (unsigned long long)(ti >> 64);
    }
  } else if constexpr (std::is_same_v<T, u128>) {
    __shared__ u128 part[128];
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      u128 t = 0;
      for (int i = 0; i < (int)blockDim.x; ++i) t += part[i];
      unsigned long long* rec = static_cast<unsigned long long*>(a.partials) + (size_t)blockIdx.x * kIntRecord;
      rec[0] = (unsigned long long)t;
      rec[1] = (unsigned long long)(t >> 64);
    }
  } else {
    __shared__ dd scratch[3 * 32];
    dd v[3] = {two_sum(kr, -kcr), two_sum(ki, -kci), dd{0.0, 0.0}};
    block_sum_dd<3>(v, scratch);
    if (threadIdx.x == 0) {
      if constexpr (std::is_same_v<T, double>) {
        double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * kRealRecord;
        rec[0] = v[0].hi;
        rec[1] = v[0].lo;
        rec[2] = 0.0;
        rec[3] = 0.0;
      } else {
        double* rec = static_cast<double*>(a.partials) + (size_t)blockIdx.x * kCplxRecord;
        rec[0] = v[0].hi;
        rec[1] = v[0].lo;
        rec[2] = v[1].hi;
        rec[3] = v[1].lo;
        rec[4] = 0.0;
        rec[5] = 0.0;
      }
    }
  }
}

void* pick(int dtype) {
  switch (dtype) {
    case 0: return (void*)combinatoric_kernel<RealF>;
    case 1: return (void*)combinatoric_kernel<CplxF>;
    case 2: return (void*)combinatoric_kernel<IntF<unsigned char>>;
    case 3: return (void*)combinatoric_kernel<IntF<long long>>;
    case 4: return (void*)combinatoric_kernel<GaussF>;
    default: return nullptr;
  }
}

size_t elem_bytes(int dtype) { return dtype == 0 ? 8 : dtype == 4 ? 32 : 16; }

// the tables of the last rows: n <= 16, at least four rows, not Gaussian integers
// (room for C(16,3) triples and C(16,4) quadruples)
bool use_tail(int m, int n, int dtype) { return n <= kTailN && m >= 4 && dtype != 4; }

// the table of the last five rows as well: real input (8-byte entries, 54 KB of tables
// in all at n = 16, shared by the 8 warps of a 256-thread block; 16-byte entries would
// leave one block per SM) with m >= 6
bool use_tail5(int m, int n, int dtype) { return use_tail(m, n, dtype) && m >= 6 && dtype == 0; }

size_t smem_bytes(int m, int n, int dtype) {
  size_t cells = (size_t)m * n;
  if (use_tail(m, n, dtype)) cells += (size_t)(binom_small(n, 3) + binom_small(n, 4));
  if (use_tail5(m, n, dtype)) cells += (size_t)binom_small(n, 5);
  return cells * elem_bytes(dtype);
}

}  // namespace

// threads per block: 256 for real input with the five-row table (one copy of the tables
// for 8 warps), else 128 (the integer and Gaussian reductions hold 128 partials)
int combinatoric_block(int m, int n, int dtype) { return use_tail5(m, n, dtype) ? 256 : 128; }

// rows below the search taken from the tables (five, four with only the four-row table,
// none without tables): the prefix depth stays above them, so that every prefix still
// has a level of the search below it
int combinatoric_table_rows(int m, int n, int dtype) {
  return use_tail5(m, n, dtype) ? 6 : (use_tail(m, n, dtype) && m >= 5) ? 5 : use_tail(m, n, dtype) ? 4 : 0;
}

int combinatoric_blocks_per_sm(int m, int n, int dtype, int block) {
  void* k = pick(dtype);
  if (!k) return 0;
  size_t smem = smem_bytes(m, n, dtype);
  if (smem > 32 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, smem) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_combinatoric(const SweepArgs& a, int dtype, int depth, uint64_t prefixes, const LaunchCfg& c) {
  void* k = pick(dtype);
  if (!k) return cudaErrorInvalidValue;
  size_t smem = smem_bytes(a.m, a.n, dtype);
  if (smem > 32 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  SweepArgs args = a;
  int d = depth;
  uint64_t p = prefixes;
  int t = use_tail5(a.m, a.n, dtype) ? 2 : use_tail(a.m, a.n, dtype) ? 1 : 0;
  void* params[] = {&args, &d, &p, &t};
  return cudaLaunchKernel(k, dim3(c.grid), dim3(c.block), params, smem, c.stream);
}

}  // namespace perm
