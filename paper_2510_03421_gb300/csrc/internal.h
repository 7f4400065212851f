// Host-side interfaces between the C ABI (capi.cu) and the kernel files.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace perm {

// One Gray-code sweep over the terms [g_begin, g_end) of one matrix.
struct SweepArgs {
  const void* A;      // device pointer to the matrix
  int m, n;           // m <= n <= 64 (after the transpose rule)
  int64_t rs, cs;     // element (i, j) of the m x n operand is A[i * rs + j * cs]
  uint64_t g_begin;   // first term
  uint64_t g_end;     // one past the last term
  int chunk_log2;     // column sums are rebuilt exactly at every multiple of 2^chunk_log2
  int start_mode;     // 1 = per-thread rebuild, 2 = warp DMMA contraction
  int want_abs = 0;   // integer-pipe sweeps: also accumulate sum |term| (runtime flag)
  void* partials;     // per-block records (layout per kernel family, see below)
  int fp64_cols = 0;  // complex integer-pipe sweep: the last fp64_cols columns of each
                      // product on the FP64 unit (0 = none)
};

struct LaunchCfg {
  int grid;
  int block;
  cudaStream_t stream;
};

// Per-block record of the real FP64 sweeps: {sum.hi, sum.lo, abssum.hi, abssum.lo}.
constexpr int kRealRecord = 4;
// Per-block record of the complex sweeps: {re.hi, re.lo, im.hi, im.lo, abs.hi, abs.lo}.
constexpr int kCplxRecord = 6;
// Per-block record of the integer sweeps: int128 as {low u64, high u64}.
constexpr int kIntRecord = 2;

// --- Glynn, real FP64 arithmetic (glynn_f64.cu)
cudaError_t launch_glynn_f64(const SweepArgs& a, const LaunchCfg& c, bool want_abs);
int glynn_f64_blocks_per_sm(int n, int block, bool want_abs);

// --- Glynn, real FP64 with chunk-start column sums on the FP64 tensor cores (glynn_dmma.cu)
cudaError_t launch_glynn_dmma(const SweepArgs& a, const LaunchCfg& c, bool want_abs);
int glynn_dmma_blocks_per_sm(int n, int block, bool want_abs);
int glynn_dmma_max_n();

// --- Glynn, real input on the integer pipes (glynn_fx.cu)
// Quantised +-2q table (row i, column j at d[i * 64 + j]) and the exponents the
// preparation kernel derives on the device.
struct FxTable {
  long long d[64 * 64];
  int e_max;    // sum_j x_j with sum_i |a'_ij| < 2^x_j
  int e_sum;    // sum_j e_j (column j scaled by 2^e_j)
  int bad;      // a non-finite entry was seen
  int inexact;  // some entry was rounded when scaled to fixed point
};
// mixed: the last glynn_fx_mixed_columns(n) columns' product runs on the FP64 unit
cudaError_t launch_fx_prep(const SweepArgs& a, FxTable* tab, cudaStream_t stream);
// pair: the lane-pair kernel (glynn_fxp_kernel; mixed, no error bound, its own block)
cudaError_t launch_glynn_fx(const SweepArgs& a, FxTable* tab, const LaunchCfg& c, bool want_abs, bool mixed,
                            bool pair = false);
int glynn_fx_blocks_per_sm(int n, int block, bool mixed, bool pair = false);
int glynn_fx_mixed_columns(int n);
int glynn_fx_block(int n);  // threads per block of the square kernel (its launch bound)
bool glynn_fx_pair_available(int n);
int glynn_fx_pair_block();               // threads per block of the lane-pair kernel
int glynn_fx_pair_mixed_columns(int n);  // columns on the FP64 unit, both halves together
// grouped rectangular walk (1 <= m < n; glynn_fxg.cu): g ranges over [0, 2^(m-1)),
// n - m + 1 terms each
cudaError_t launch_glynn_fxg(const SweepArgs& a, FxTable* tab, const LaunchCfg& c, bool want_abs);
int glynn_fxg_blocks_per_sm(int m, int n, int block);

// rectangular walk with the padding summed in closed form (1 <= m <= glynn_esym_max_m(),
// m < n; glynn_esym.cu): g ranges over [0, 2^(m-1)); records of kCplxRecord doubles
// {sum, sum e_m(|c|), quantisation term} (unnormalised), reduced by launch_esym_finish
struct EsymTable {
  long long d[64 * 64];  // +2 q_ij at d[i * 64 + j] (rows i < m)
  int e[64];             // column j is held as q_ij = a_ij 2^e[j]
  int bad;               // a non-finite entry was seen
  int inexact;           // some a_ij 2^e[j] was not an integer (rounded)
  int eta;               // bound on a column sum's quantisation error, in units
  int pad;
};
cudaError_t launch_glynn_esym(const SweepArgs& a, EsymTable* tab, const LaunchCfg& c, bool want_abs);
int glynn_esym_blocks_per_sm(int m, int n, int block, bool want_abs);
int glynn_esym_max_m();
int glynn_esym_block();
// out = sum / 2^(m-1); err = coef * G + F + the rounding of out (err may be null)
cudaError_t launch_esym_finish(const double* rec, int nrec, int m, double coef, double* out, double* err,
                               cudaStream_t s);

// complex rectangles with the padding summed in closed form (glynn_cesym.cu): same
// index range and records as the complex sweeps (kCplxRecord, no error term)
struct CesymTable {
  long long d[2 * 64 * 64];  // (re, im) of +2 q_ij at d[2 (i * 64 + j)]
  int e[64];
  int bad;
  int pad;
};
cudaError_t launch_glynn_cesym(const SweepArgs& a, CesymTable* tab, const LaunchCfg& c);
int glynn_cesym_blocks_per_sm(int m, int n, int block);
int glynn_cesym_max_m();
int glynn_cesym_block();

// --- Glynn, complex input on the integer pipes (glynn_cfx.cu); n <= glynn_cfx_max_n()
struct CfxTable {
  long long d[2 * 64 * 64];  // (re, im) of +2q for row i, column j at 2 (i * 64 + j)
  int e_sum;
  int bad;
};
// grouped: the rectangular walk over the 2^(m-1) real-row sign vectors (1 <= m < n)
cudaError_t launch_glynn_cfx(const SweepArgs& a, CfxTable* tab, const LaunchCfg& c, bool grouped);
int glynn_cfx_blocks_per_sm(int m, int n, int block, bool grouped);
int glynn_cfx_max_n();

// --- Glynn, complex FP64 (glynn_c128.cu); n <= glynn_c128_max_n()
cudaError_t launch_glynn_c128(const SweepArgs& a, const LaunchCfg& c, bool want_abs);
int glynn_c128_blocks_per_sm(int n, int block, bool want_abs);
int glynn_c128_max_n();

// --- Glynn, exact integer (glynn_int.cu); dtype 2 = uint8, 3 = int64
// grouped: the rectangular walk over the 2^(m-1) real-row sign vectors (1 <= m < n)
cudaError_t launch_glynn_int(const SweepArgs& a, int dtype, const LaunchCfg& c, bool grouped);
int glynn_int_blocks_per_sm(int n, int dtype, int block, bool grouped);
// Gaussian integers (dtype 4, n <= glynn_gaussian_max_n()): records as two int128 arrays
// (real parts at [0, grid), imaginary parts at [grid, 2 grid))
cudaError_t launch_glynn_gaussian(const SweepArgs& a, const LaunchCfg& c);
int glynn_gaussian_blocks_per_sm(int n, int block);
int glynn_gaussian_max_n();
// a-priori int128 range check; writes 3 (PERM_EOVERFLOW) to *status if exactness is not
// assured (glynn: for the Glynn / Ryser sums, else for the plain sum of products)
cudaError_t launch_int_bound(const void* A, int dtype, int m, int n, int64_t rs, int64_t cs, int* status,
                             cudaStream_t s, bool glynn = true);

// --- Ryser over the 2^n column subsets in Gray-code order (ryser_f64.cu)
// w[s] = (-1)^(m-s) C(n-s, m-s) for s <= m, else 0 (used when m < n)
struct SizeWeights {
  double w[65];
};
cudaError_t launch_ryser_f64(const SweepArgs& a, const SizeWeights& weights, const LaunchCfg& c, bool want_abs);
// Ryser on the integer pipes (ryser_fx.cu), real input, 1 <= m <= n <= 62: g over the
// 2^n Gray-ordered subsets, weights (-1)^(m-s) C(n-s, m-s); kRealRecord records
cudaError_t launch_ryser_fx(const SweepArgs& a, FxTable* tab, const LaunchCfg& c, bool want_abs);
int ryser_fx_blocks_per_sm(int m, int n, int block, bool want_abs);
int ryser_fx_block(int m);
// c[s] = number of nonempty subsets of size < s (c[1] = 0): start of size s in the
// global index of the by-size Ryser enumeration
struct SizeCounts {
  unsigned long long c[66];
};
// rectangular Ryser by subset size in colex order (ryser_colex.cu), real FP64
cudaError_t launch_ryser_colex(const SweepArgs& a, const SizeWeights& w, const SizeCounts& cum, const LaunchCfg& c);
int ryser_colex_blocks_per_sm(int m, int n, int block);
// exact weights for the integer Ryser sweep, as two's-complement int128 halves
struct IntWeights {
  unsigned long long lo[65];
  unsigned long long hi[65];
};
// complex (dtype 1, m <= 40) and integer (dtype 2 / 3) Ryser sweeps (ryser_ext.cu)
cudaError_t launch_ryser_ext(const SweepArgs& a, int dtype, const SizeWeights& fw, const IntWeights& iw,
                             const LaunchCfg& c);
int ryser_ext_blocks_per_sm(int m, int n, int dtype, int block);
int ryser_f64_blocks_per_sm(int m, int n, int block, bool weighted, bool want_abs);

// --- combinatoric algorithm (combinatoric.cu); dtype as perm_dtype
cudaError_t launch_combinatoric(const SweepArgs& a, int dtype, int depth, uint64_t prefixes, const LaunchCfg& c);
int combinatoric_block(int m, int n, int dtype);  // threads per block of the combinatoric kernel
int combinatoric_table_rows(int m, int n, int dtype);  // rows from the first table level down
int combinatoric_blocks_per_sm(int m, int n, int dtype, int block);

// --- batched Glynn (batched.cu)
struct BatchItem {
  int first;  // position in `order` of the (first) matrix
  int count;  // lane items: number of matrices (<= 32); warp items: sub-range index
  int parts;  // warp items: number of sub-ranges of the matrix (1 = whole)
  int pad;
};
struct ClassWork {
  const BatchItem* items;  // this class's items, longest first
  int nitems;
  int* counter;            // next item (zeroed before the launch)
};
struct BatchArgs {
  const double* packed;     // elements of all matrices (complex: (re, im) pairs)
  const int64_t* offsets;   // element offset of matrix b
  const int32_t* M;         // rows of matrix b (row-major, leading dimension N[b])
  const int32_t* N;         // columns of matrix b
  const int32_t* order;     // matrices in item order
  const int32_t* part_base; // first partial slot of matrix b (split matrices)
  double* partials;         // 4 doubles per slot
  int* done;                // sub-ranges finished per matrix (zeroed before the launch)
  double* out;              // results (complex: (re, im) pairs)
  int chunk_log2;
  // integer-pipe classes (batched_fx.cu): quantised +2q tables, n rows of n (real) or 2n
  // (complex, (re, im)) int64 per matrix at fx_table + fx_offset[b], and the sum of the
  // column exponents
  long long* fx_table;
  const int64_t* fx_offset;
  int* fx_esum;
};
constexpr int kFxBad = -2147483647 - 1;  // fx_esum of a matrix with a non-finite entry
cudaError_t launch_batched_class(const BatchArgs& a, const ClassWork& c, int dtype, int npad, bool lane,
                                 const LaunchCfg& lc);
int batched_blocks_per_sm(int dtype, int npad, bool lane, int block);
// warp-item classes on the integer pipes (batched_fx.cu), dtype 0 (real) or 1 (complex);
// share: part of each product's columns on the FP64 unit (a tuner choice)
bool batched_fx_has_class(int dtype, int npad);
int batched_fx_blocks_per_sm(int dtype, int npad, int block, bool share);
cudaError_t launch_batched_fx_prep(const BatchArgs& a, int dtype, const int32_t* list, int count, cudaStream_t stream);
cudaError_t launch_batched_fx(const BatchArgs& a, const ClassWork& c, int dtype, int npad, const LaunchCfg& lc,
                              bool share);
}  // namespace perm
struct perm_handle_s;
namespace perm {
// SBP coefficients (sbp.cu): out[k] = per(C[:, occupied columns of occ[k]]); device
// pointers; real input on the integer pipes unless fp64; scratch: >= 33 KiB of device
// memory for the quantised table; returns 0, 1 (unsupported n) or 2 (CUDA error)
int sbp_run(perm_handle_s* h, const double* dC, int64_t ld, int n, int N, int dtype, const uint64_t* docc,
            int64_t count, double* dout, cudaStream_t stream, int chunk_log2, int sms, bool fp64, void* scratch);
// Cauchy permanents by Borchardt's theorem (cauchy.cu): out[b] = per(1 / (x_i - y_j)) of
// matrix b (x, y: count x n, device); err (or null) gets an error estimate per matrix;
// scratch: grid * cauchy_scratch_words(n) words of device memory; state:
// cauchy_state_bytes(count) bytes (8-byte aligned, no initial contents needed);
// status: sticky code (1 = coinciding or non-finite points, 2 = precision ladder
// exhausted; result NaN)
size_t cauchy_scratch_words(int n);
size_t cauchy_state_bytes(int64_t count);
int cauchy_max_n();
int cauchy_grid(int64_t count, int sms, int* block);  // blocks (and threads per block) of a launch
cudaError_t launch_cauchy(const double* x, const double* y, int n, int64_t count, double* out, double* err,
                          uint64_t* scratch, void* state, int grid, int block, int* status, cudaStream_t stream,
                          double rel_extra = 0.0);
// the points of count Cauchy matrices from occupation bitstrings: xs[k n + l] = x[l],
// ys[k n + l] = y[l-th occupied state of occ[k]] (NaN if occ[k] does not hold n states < N)
cudaError_t launch_cauchy_gather(const double* x, int n, const double* y, int N, const uint64_t* occ, int64_t count,
                                 double* xs, double* ys, int sms, cudaStream_t stream);
// fit points x, y (n each, device) to a real n x n matrix (n <= 64); *ok = 1 if every
// entry is 1 / (x_i - y_j) within relative tol, all of one sign (see cauchy.cu)
cudaError_t launch_cauchy_fit(const double* A, int n, int64_t rs, int64_t cs, double tol, double* x, double* y,
                              int* ok, cudaStream_t stream);
// host orchestration of perm_batched (batched_host.cu)
int batched_run(perm_handle_s* h, const void* packed, const int64_t* offsets, const int32_t* M, const int32_t* N,
                int64_t count, int dtype, void* out, cudaStream_t stream, const void* opts);
void batched_release(perm_handle_s* h);
// exact batched permanents of integer matrices (batched_int.cu; host side in
// batched_host.cu): out gets an int128 {low, high} per matrix (Gaussian integers: two,
// real then imaginary); status: 3 if some matrix failed the a-priori range check
int batched_int_run(perm_handle_s* h, const void* packed, const int64_t* offsets, const int32_t* M, const int32_t* N,
                    int64_t count, int dtype, void* out, int* status, cudaStream_t s);
int batched_int_class(int n);  // padded order 8, 16, 24 or 32 (0 above)
int batched_int_max_n();
cudaError_t launch_batched_int(const void* packed, const int64_t* offsets, const int32_t* M, const int32_t* N,
                               const int32_t* list, int count, int dtype, int npad, unsigned long long* out,
                               int* status, int sms, cudaStream_t stream);

// --- final reductions (reduce.cu)
// Sum `nrec` real records in a fixed order, scale by 2^-pow2 / fact (fact = (n-m)!,
// given as the integer whose factorial divides), write result (and error bound).
// If `raw` is set, write the unnormalised double-double sum to out[0..1] instead.
cudaError_t launch_finish_real(const double* rec, int nrec, int pow2, int fact_of, double err_coef, double* out,
                               double* err, bool raw, cudaStream_t s, double sign = 1.0);

// records {sum, sum |term|, sum of the eta-widened products} (kCplxRecord doubles, the
// integer-pipe sweeps with an error bound): see reduce.cu
cudaError_t launch_finish_bound(const double* rec, int nrec, int pow2, int fact_of, double coef, double* out,
                                double* err, bool raw, cudaStream_t s, double diff_coef = 0.0);
// negate the leading double-double of each record (stride doubles apart)
cudaError_t launch_negate_records(double* rec, int nrec, int stride, cudaStream_t s);
cudaError_t launch_finish_cplx(const double* rec, int nrec, int pow2, int fact_of, double err_coef, double* out,
                               double* err, bool raw, cudaStream_t s);
cudaError_t launch_finish_int(const unsigned long long* rec, int nrec, int pow2, int fact_of, unsigned long long* out,
                              bool raw, cudaStream_t s);

// Write one double (e.g. -1 for "no error bound") to device memory.
cudaError_t launch_write_double(double v, double* p, cudaStream_t s);

// Write a constant result (used for m == 0, per = 1) for a dtype code.
cudaError_t launch_write_one(int dtype, void* out, cudaStream_t s);
// out = product of `count` block permanents at slots (16 bytes apart; dtype 0 real,
// 1 complex), in double-double; count == 0 writes zero
cudaError_t launch_block_product(int dtype, const double* slots, int count, void* out, cudaStream_t s);

}  // namespace perm
