/*
 * perm.h -- C ABI of the GB300 permanent library (libperm.so).
 *
 * The permanent of an m x n matrix A (m <= n) is
 *     per(A) = sum over m-permutations sigma of {1..n} of prod_i a_{i sigma(i)}
 * (Eq. permanent_definition and Eq. rectangular_permanent_definition of the paper;
 * for m > n the library evaluates per(A^T), as that definition prescribes, and
 * per of a 0 x n matrix is 1).
 *
 * Common argument conventions for the per-matrix entry points
 * ------------------------------------------------------------
 *   h        handle from perm_create (owns device workspace; one host thread at a time).
 *            The workspace is shared by all calls on the handle: calls issued on
 *            different streams through one handle must be ordered by the caller (one
 *            stream per handle, or one handle per stream, avoids the question).
 *   A        pointer to the matrix, row-major, element (i, j) at A[i * ld + j].
 *            May be device memory or host memory (pageable or pinned); host input
 *            is copied to the handle's workspace on `stream` before the launch.
 *            The caller keeps ownership.
 *   m, n     0 <= m, n <= 64 after the transpose rule (max(m, n) <= 64).
 *   ld       leading dimension in elements, ld >= n (ld >= m is not needed).
 *   dtype    perm_dtype below.  Real input is double, complex input is interleaved
 *            (re, im) doubles (ld counted in complex elements), PERM_U8 input is
 *            one unsigned byte per entry (0/1 matrices, any value 0..255 allowed),
 *            PERM_I64 input is int64.
 *   out      pointer (device or host) receiving the result:
 *              PERM_F64  -> 1 double
 *              PERM_C128 -> 2 doubles (re, im)
 *              PERM_U8 / PERM_I64 -> 16-byte two's-complement int128 {low u64, high u64}
 *            Device output is written asynchronously on `stream`; host output is
 *            written before the call returns (the call synchronises `stream`).
 *   stream   cudaStream_t (NULL = legacy default stream).
 *   opts     optional tuning / accuracy options (NULL = defaults).
 *
 * Errors: every entry point returns a perm_status.  Argument errors are reported
 * synchronously before any work is queued.  No entry point throws, traps, aborts
 * or prints.
 */
#ifndef PERM_H_
#define PERM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PERM_F64 = 0,  /* double */
  PERM_C128 = 1, /* complex double, interleaved (re, im) */
  PERM_U8 = 2,   /* uint8 entries (0/1 biadjacency matrices), exact integer result */
  PERM_I64 = 3,  /* int64 entries, exact integer result */
  PERM_CI64 = 4  /* Gaussian integers: interleaved (re, im) int64 pairs, exact result as two
                    int128 (real part, then imaginary part; 32 bytes); perm_glynn,
                    perm_glynn_partial, perm_auto (which takes Glynn) and perm_batched
                    with n <= 32, perm_ryser with m <= 32, perm_combinatoric */
} perm_dtype;

typedef enum {
  PERM_OK = 0,
  PERM_EINVAL = 1,    /* null pointer, ld < n, unknown dtype / algorithm / option */
  PERM_ETOOBIG = 2,   /* max(m, n) > 64, or the term count exceeds opts->max_terms */
  PERM_EOVERFLOW = 3, /* integer input whose a-priori bound may not fit in int128 */
  PERM_ECUDA = 4,     /* a CUDA runtime call failed */
  PERM_ENOMEM = 5,    /* workspace allocation failed */
  PERM_EUNSUPPORTED = 6 /* combination of dtype / algorithm / option not provided */
} perm_status;

/* Arithmetic of the Glynn sweeps (real and complex input; Ryser is FP64 or exact).
 * The integer-pipe choices (FIXED, MIXED) keep exact 64-bit fixed-point column sums
 * and sum the terms in 192-bit fixed point; for m < n they walk the real rows only,
 * with the padding rows of ones grouped by their number of -1 signs (integer
 * products), 2^(m-1) (n-m+1) terms instead of 2^(n-1). */
typedef enum {
  PERM_ARITH_AUTO = 0,  /* real: MIXED for n >= 10; complex: FIXED for n >= 10 unless an
                           error bound is asked for; FP64 below 10 or with DMMA chunk starts */
  PERM_ARITH_FP64 = 1,  /* FP64 column sums updated by +-2 a_rj, FP64 products, Kahan sums */
  PERM_ARITH_FIXED = 2, /* products in a 64-bit-mantissa software float on the integer pipes */
  PERM_ARITH_MIXED = 3  /* real Glynn: as FIXED, with the product of a few columns per term on
                           the FP64 unit beside the integer pipes (relative error 2^-53 per
                           such factor); other sweeps treat it as FIXED */
} perm_arith;

/* How the column sums at the start of each chunk of the Gray-code sweep are formed. */
typedef enum {
  PERM_START_AUTO = 0,
  PERM_START_SCALAR = 1, /* each thread sums its own rows */
  PERM_START_DMMA = 2    /* one +-1 x A contraction per warp on the FP64 tensor cores */
} perm_start;

typedef struct {
  int32_t chunk_log2;   /* terms between exact re-anchoring of the column sums (0 = planner) */
  int32_t block;        /* threads per block (0 = planner).  The real square sweep on the
                           integer pipes from n = 37 (mixed arithmetic, no error bound)
                           runs a lane pair per term in 256-thread blocks; a block of at
                           most 128 threads selects the one-lane kernel there */
  int32_t grid;         /* blocks (0 = planner: a multiple of the SM count) */
  int32_t arith;        /* perm_arith */
  int32_t start;        /* perm_start */
  int32_t exhaustive;   /* perm_auto only: time every candidate instead of the cost model */
  uint64_t max_terms;   /* refuse sweeps longer than this (0 = 2^44 terms) */
  double* err;          /* optional pointer (device or host, like out) receiving an a-posteriori
                           bound on |result - per(A)| (floating dtypes; complex: bound on modulus) */
} perm_opts;

typedef struct perm_handle_s* perm_handle;

/* Create a handle on CUDA device `device` (workspace is allocated lazily, never
 * during stream capture).  Returns PERM_ECUDA if the device is unusable. */
int perm_create(perm_handle* h, int device);

/* Free the handle and its workspace.  Synchronises the device first. */
int perm_destroy(perm_handle h);

/* Glynn's formula, Eq. glynn, with the rectangular extension of Eq. glynn_filled_matrix /
 * Eq. glynn_rectangle for m < n (n - m virtual rows of ones, result divided by (n-m)!).
 * The 2^(n-1) sign vectors are visited in reflected Gray-code order.  All dtypes. */
int perm_glynn(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, void* out,
               void* stream, const perm_opts* opts);

/* Ryser's inclusion-exclusion formula: Eq. ryser_square over all 2^n column subsets
 * (Gray-code order) for m = n, Eq. ryser_rectangle over the column subsets of sizes
 * 1..m with weights (-1)^(m-s) C(n-s, m-s) for m < n.  All dtypes. */
int perm_ryser(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, void* out,
               void* stream, const perm_opts* opts);

/* The combinatoric algorithm: the definition (Eq. rectangular_permanent_definition)
 * summed over all m-permutations with shared prefix products; zero entries prune
 * whole subtrees.  For n <= 16 (not PERM_CI64) the last three to five rows come from
 * per-block tables of their permanents on every column subset, so the search stops
 * that many levels early.  Cost O(m n!/(n-m)!) on dense input (the tables divide it by
 * up to 6!); opts->max_terms (default 2^44) caps the dense count n!/(n-m)!; all dtypes. */
int perm_combinatoric(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, void* out,
                      void* stream, const perm_opts* opts);

/* Algorithm selection in place of the paper's tuned hyperplanes (Algorithm "Optimized
 * Algorithm Selection"): a cost model trained on this library's own timings picks the
 * algorithm and kernel configuration; opts->exhaustive times every candidate instead.
 * Structure is used first (not with opts->exhaustive): a real or complex matrix with an
 * empty row gives 0, one whose nonzero pattern splits into independent blocks is the
 * product of the blocks' permanents, and a dense real square matrix of order >= 24
 * whose entries are 1/(x_i - y_j) within 2^-48 relative, all of one sign, is evaluated
 * by Borchardt's theorem on the fitted points (perm_cauchy), the error bound widened
 * by n 2^-48 (1 + n 2^-48) |per| for the fit.
 * Cost of that structure pass: the matrix is copied to the host and `stream` is
 * synchronised before the sweep is launched (at most 64 KiB of copy, microseconds;
 * but the call does not return before the stream's earlier work has finished, so it
 * cannot be captured in a CUDA graph).  Ryser candidates take real input only; the
 * FP64 configurations among the candidates are offered for square matrices only. */
int perm_auto(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, void* out,
              void* stream, const perm_opts* opts);

/* Many permanents in one call.  Matrix b (0 <= b < count) has shape M[b] x N[b],
 * row-major with leading dimension N[b], starting at element offsets[b] of `packed`
 * (elements of `dtype`).  packed, offsets, M, N and out may each be device or host
 * memory; out receives `count` results laid out as for the single-matrix calls.
 * The call buckets the matrices by size and runs them in one persistent launch per
 * bucket, captured once into a CUDA graph and replayed for the same size signature;
 * max(M[b], N[b]) <= 32.  Real and complex matrices of order >= 13 taken one per warp
 * run on the integer pipes unless opts->arith is PERM_ARITH_FP64; opts->exhaustive tunes the launch settings (and whether part of
 * each product goes to the FP64 unit: forced on by PERM_ARITH_MIXED, off by
 * PERM_ARITH_FIXED) on a sample and keeps them for batches of the same sizes.
 * Integer matrices (PERM_U8, PERM_I64, PERM_CI64; max(M[b], N[b]) <= 32) are computed
 * exactly, one warp per matrix (Glynn, int128 modulo 2^128 per part, results laid out
 * as for perm_glynn); a matrix whose a-priori bound reaches 2^126.5 raises
 * PERM_EOVERFLOW, returned by the call when out is host memory, else kept for
 * perm_device_status; no graph, no tuner. */
int perm_batched(perm_handle h, const void* packed, const int64_t* offsets, const int32_t* M, const int32_t* N,
                 int64_t count, int dtype, void* out, void* stream, const perm_opts* opts);

/* Coefficients of a symmetric product of bosons (Eq. SBP): for each occupation
 * bitstring occ[k] (bit j set = state j occupied, exactly n states occupied, all
 * below bit N), out[k] = c_m = per(C P) (Eq. SBGpermanent), the permanent of the
 * n x n matrix formed by the occupied columns of C in increasing order.  C is n x N,
 * row-major with leading dimension ld >= N (elements of `dtype`, PERM_F64 or
 * PERM_C128); n <= 32, N <= 64.  The columns are gathered inside the kernel; no
 * submatrix is materialised.  C, occ and out may each be device or host memory; out
 * receives `count` results (double, or (re, im) pairs).  A bitstring with the wrong
 * number of occupied states gets NaN.  Real input runs on the integer pipes (exact
 * fixed-point column sums, 64-bit-mantissa products, 192-bit sums; a column with a
 * non-finite entry makes the bitstrings that occupy it NaN) unless opts->arith is
 * PERM_ARITH_FP64; complex input, and real input with PERM_ARITH_FP64, use FP64 with
 * compensated sums, opts->chunk_log2 setting the rebuild interval of the column sums
 * (default 14).
 * Errors: PERM_EINVAL (shapes, null pointers), PERM_ETOOBIG (n > 32 or N > 64),
 * PERM_EUNSUPPORTED (integer dtypes). */
int perm_sbp(perm_handle h, const void* C, int64_t n, int64_t N, int64_t ld, int dtype, const uint64_t* occ,
             int64_t count, void* out, void* stream, const perm_opts* opts);

/* Permanents of square Cauchy matrices c_ij = 1 / (x_i - y_j) by Borchardt's theorem
 * (Eq. caucy_permanent): per(C) = det(C o C) / det(C), with det(C) from Cauchy's product
 * formula and det(C o C) by Gaussian elimination with partial pivoting, both in a
 * multi-limb binary floating point (up to 1024-bit mantissas, 32-bit exponents).
 * C o C is very ill-conditioned (an elimination in double loses every digit from
 * n ~ 12 on), so the call climbs a precision ladder: the permanent is computed at
 * about 9 n + 32 bits and at successively longer precisions until two rungs agree to
 * 2^-62 relative, and the longer one is returned rounded to double.  The value is the
 * permanent of the exact Cauchy matrix of the given doubles (not of C rounded to
 * double).
 *   x, y     points of matrix b (0 <= b < count) at x[b n .. b n + n), y[b n .. b n + n)
 *   n        order, 1 <= n <= 64
 *   out      count doubles
 *   opts     only opts->err is read: if set, count doubles receiving an error estimate
 *            per matrix, |difference of the last two rungs| + 2^-53 |result| (an
 *            estimate from the ladder, not a proven bound)
 * x, y, out and opts->err may each be device or host memory; with any of them in host
 * memory the call synchronises `stream` before returning.  A matrix with a
 * non-finite or coinciding point (x_i = x_k, y_j = y_l or x_i = y_j, where det(C) = 0 or
 * an entry is infinite) gets NaN and status PERM_EINVAL; one whose ladder ends without
 * agreement (per(C) = 0 is the known case) gets NaN and PERM_ETOOBIG.  These statuses
 * are returned by the call when out or err is in host memory, else kept for
 * perm_device_status.  One block of 256 threads per matrix; the handle keeps about
 * 2.6 KiB x (n^2 + n + 514) of scratch per concurrently running block.
 * Errors: PERM_EINVAL (null pointers, n < 1, count < 0), PERM_ETOOBIG (n > 64),
 * PERM_ENOMEM. */
int perm_cauchy(perm_handle h, const double* x, const double* y, int64_t n, int64_t count, double* out,
                void* stream, const perm_opts* opts);

/* SBP coefficients (Eq. SBGpermanent) of a Cauchy coefficient matrix c_ij = 1/(x_i - y_j),
 * i < n, j < N -- the form of the pairing wavefunctions the paper names as the source of
 * Cauchy permanents: out[k] = per of the n x n Cauchy matrix of the points x and the y_j
 * of the occupied states of occ[k] in increasing order (bit j set = state j occupied),
 * by Borchardt's theorem as in perm_cauchy (opts->err as there).  x (n doubles), y (N),
 * occ (count uint64) and out (count) may each be device or host memory.  A bitstring
 * without exactly n occupied states below bit N gets NaN and status PERM_EINVAL, as
 * coinciding points do (see perm_cauchy).  Errors: PERM_EINVAL (null pointers, n < 1,
 * N < n, count < 0), PERM_ETOOBIG (n or N > 64), PERM_ENOMEM. */
int perm_cauchy_sbp(perm_handle h, const double* x, int64_t n, const double* y, int64_t N, const uint64_t* occ,
                    int64_t count, double* out, void* stream, const perm_opts* opts);

/* Unnormalised partial Glynn sum over the terms g_begin <= g < g_end of Eq. glynn_rectangle:
 *     sum_g (-1)^g prod_j ( sum_{i<m} delta_i(g) a_ij + sum_{i>=m} delta_i(g) ),
 * where delta_i(g) = -1 if bit (n-1-i) of gray(g) = g ^ (g >> 1) is set, else +1,
 * 0 <= g_begin <= g_end <= 2^(n-1) (m <= n required; no transpose).
 * `partial` receives, for PERM_F64, a double-double (hi, lo); for PERM_C128,
 * (re_hi, re_lo, im_hi, im_lo); for integer dtypes the int128 sum modulo 2^128.
 * Ranges are the unit of resumption and of sharding across devices. */
int perm_glynn_partial(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype,
                       uint64_t g_begin, uint64_t g_end, void* partial, void* stream, const perm_opts* opts);

/* Partial Ryser sum over the column subsets g_begin <= g < g_end in reflected Gray-code
 * order (subset(g) = set bits of gray(g) = g ^ (g >> 1), bit c <-> column c), each
 * weighted as in the sum that perm_ryser evaluates: (-1)^(m-|S|) C(n-|S|, m-|S|)
 * prod_i sum_{j in S} a_ij (Eq. ryser_rectangle; for m = n, Eq. ryser_square).  The
 * sum over [0, 2^n) is per(A).  PERM_F64 only; m <= n required (no transpose);
 * `partial` receives a double-double (hi, lo). */
int perm_ryser_partial(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype,
                       uint64_t g_begin, uint64_t g_end, void* partial, void* stream, const perm_opts* opts);

/* Real (PERM_F64) Glynn sweep for callers that cannot allocate device memory, such
 * as runtimes that hand out every buffer from a pool reserved up front or plugin
 * hosts that forbid cudaMalloc.  The paper has no counterpart; this is a deployment
 * variant of perm_glynn.
 *   A, out   device (or managed) pointers on the current device; host pointers and
 *            another device's memory are rejected with PERM_EINVAL before anything is
 *            launched.  Layout as for perm_glynn; out gets 1 double.
 *   grid     blocks of the sweep, 0 = chosen by the library; at most 2048, larger
 *            values return PERM_ETOOBIG.
 * The call allocates nothing: its scratch (2048 records of 32 bytes, 64 KiB) is a
 * fixed array in device memory that the library declares, present on every GPU
 * that loads the library until the process exits.  The first call on a device looks
 * up that array's device address; make that first call before any stream capture.
 * The address is kept for the life of the process: after cudaDeviceReset on a device
 * (which discards the array with the context) do not call this function again.
 * Every call shares the array, so calls whose kernels overlap on a GPU (for
 * example on two streams) race and must be serialised by the caller.  No part of the
 * scratch needs to start at zero.  No error bound is produced.  PERM_ECUDA if the
 * sweep's launch configuration cannot be set up on this device. */
int perm_glynn_noalloc(const void* A, int64_t m, int64_t n, int64_t ld, void* out, void* stream, int32_t grid);

/* Device-detected status since the last call of this function on handle h:
 * PERM_EOVERFLOW if an integer call whose result went to device memory could not
 * be guaranteed exact (its a-priori bound reached 2^126.5; the value written is
 * still the sum modulo 2^128); PERM_EINVAL or PERM_ETOOBIG if a perm_cauchy matrix
 * got NaN (see there); else PERM_OK (one of the codes raised, if several were).  Synchronises `stream`, then clears
 * the status.  Integer calls with a host `out` report PERM_EOVERFLOW directly. */
int perm_device_status(perm_handle h, void* stream, int* status);

/* Human-readable text of a perm_status (static storage). */
const char* perm_status_string(int status);

/* Library version as major * 10000 + minor * 100 + patch. */
int perm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PERM_H_ */
