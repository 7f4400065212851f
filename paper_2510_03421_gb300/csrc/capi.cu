// C ABI of libperm: argument checks, the transpose rule, host/device staging,
// the launch planner and the dispatch to the kernel families (perm_auto and the cost
// model: capi_auto.cu).
#include <algorithm>
#include <new>

#include "capi_internal.h"

namespace perm {

size_t elem_size(int dtype) {
  switch (dtype) {
    case PERM_F64: return 8;
    case PERM_C128: return 16;
    case PERM_U8: return 1;
    case PERM_I64: return 8;
    case PERM_CI64: return 16;
    default: return 0;
  }
}

size_t out_size(int dtype) { return dtype == PERM_F64 ? 8 : dtype == PERM_CI64 ? 32 : 16; }

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Grow the device workspace (never while `stream` is being captured into a graph).
int ensure_ws(perm_handle h, size_t bytes, cudaStream_t stream) {
  if (h->ws_bytes >= bytes) return PERM_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  if (h->ws) {
    if (cudaDeviceSynchronize() != cudaSuccess) return PERM_ECUDA;
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  size_t want = bytes < kWsDefault ? kWsDefault : bytes;
  if (cudaMalloc(&h->ws, want) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  h->ws_bytes = want;
  // staging area and the device status word start at zero
  if (cudaMemset(h->ws, 0, kStageA + kStageOut * 16) != cudaSuccess) return PERM_ECUDA;
  return PERM_OK;
}

// Validate, apply per(A) = per(A^T) for m > n, stage host operands.
int prepare(Call& c, perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, void* out,
            void* stream, const perm_opts* opts, bool allow_transpose) {
  if (!h || !out) return PERM_EINVAL;
  size_t es = elem_size(dtype);
  if (es == 0) return PERM_EINVAL;
  if (m < 0 || n < 0 || ld < n) return PERM_EINVAL;
  if (m > 64 || n > 64) return PERM_ETOOBIG;
  if (m > 0 && n > 0 && !A) return PERM_EINVAL;
  c.h = h;
  c.stream = static_cast<cudaStream_t>(stream);
  c.dtype = dtype;
  c.o = opts ? *opts : perm_opts{};
  if (c.o.arith < 0 || c.o.arith > 3 || c.o.start < 0 || c.o.start > 2 || c.o.chunk_log2 < 0 ||
      c.o.chunk_log2 > 62 || c.o.block < 0 || c.o.block > 1024 || (c.o.block % 32) != 0 || c.o.grid < 0)
    return PERM_EINVAL;
  if (m > n) {
    if (!allow_transpose) return PERM_EINVAL;
    c.m = (int)n;
    c.n = (int)m;
    c.rs = 1;
    c.cs = ld;
  } else {
    c.m = (int)m;
    c.n = (int)n;
    c.rs = ld;
    c.cs = 1;
  }
  if (cudaSetDevice(h->device) != cudaSuccess) return PERM_ECUDA;
  int rc = ensure_ws(h, kWsDefault, c.stream);
  if (rc) return rc;
  char* ws = static_cast<char*>(h->ws);
  // operand
  c.dA = A;
  if (m > 0 && n > 0 && !on_device(A)) {
    if (cudaMemcpy2DAsync(ws, (size_t)n * es, A, (size_t)ld * es, (size_t)n * es, (size_t)m, cudaMemcpyHostToDevice,
                          c.stream) != cudaSuccess)
      return PERM_ECUDA;
    c.dA = ws;
    if (m > n) {
      c.rs = 1;
      c.cs = n;
    } else {
      c.rs = n;
      c.cs = 1;
    }
  }
  // result
  c.hOut = nullptr;
  c.dOut = out;
  if (!on_device(out)) {
    c.hOut = out;
    c.dOut = ws + kStageA;
  }
  c.hErr = nullptr;
  c.dErr = c.o.err;
  if (c.o.err && !on_device(c.o.err)) {
    c.hErr = c.o.err;
    c.dErr = reinterpret_cast<double*>(ws + kStageA + 64);
  }
  return PERM_OK;
}

int finish(Call& c, size_t out_bytes) {
  if (cudaGetLastError() != cudaSuccess) return PERM_ECUDA;
  if (c.hOut || c.hErr) {
    if (c.hOut && cudaMemcpyAsync(c.hOut, c.dOut, out_bytes, cudaMemcpyDeviceToHost, c.stream) != cudaSuccess)
      return PERM_ECUDA;
    if (c.hErr && cudaMemcpyAsync(c.hErr, c.dErr, sizeof(double), cudaMemcpyDeviceToHost, c.stream) != cudaSuccess)
      return PERM_ECUDA;
    int dev_status = 0;
    if (c.dtype == PERM_U8 || c.dtype == PERM_I64 || c.dtype == PERM_CI64) {
      // host result: the integer range check is reported synchronously
      int* sw = reinterpret_cast<int*>(static_cast<char*>(c.h->ws) + kStageA + 132);
      if (cudaMemcpyAsync(&dev_status, sw, sizeof(int), cudaMemcpyDeviceToHost, c.stream) != cudaSuccess)
        return PERM_ECUDA;
      if (cudaStreamSynchronize(c.stream) != cudaSuccess) return PERM_ECUDA;
      if (dev_status) return dev_status;
    }
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return PERM_ECUDA;
  }
  return PERM_OK;
}

// sticky device status (calls with device output; read by perm_device_status)
int* status_word(perm_handle h) { return reinterpret_cast<int*>(static_cast<char*>(h->ws) + kStageA + 128); }
// status of the current call when its result goes to host memory (cleared per call)
int* call_status_word(perm_handle h) { return reinterpret_cast<int*>(static_cast<char*>(h->ws) + kStageA + 132); }

// workspace layout: [staged operand | result/err/status | fixed-point table | partial records]
constexpr size_t kFxTableOffset = kStageA + kStageOut * 16;
constexpr size_t kCfxTableOffset = kFxTableOffset + ((sizeof(FxTable) + 255) / 256) * 256;
constexpr size_t kPartialsOffset = kCfxTableOffset + ((sizeof(CfxTable) + 255) / 256) * 256;
CfxTable* cfx_table(perm_handle h) {
  return reinterpret_cast<CfxTable*>(static_cast<char*>(h->ws) + kCfxTableOffset);
}
FxTable* fx_table(perm_handle h) { return reinterpret_cast<FxTable*>(static_cast<char*>(h->ws) + kFxTableOffset); }
char* partials_base(perm_handle h) { return static_cast<char*>(h->ws) + kPartialsOffset; }
size_t partials_capacity(perm_handle h) { return h->ws_bytes - kPartialsOffset; }

// Grid for a sweep of `terms` terms: a multiple of the SM count at full
// occupancy, shrunk so that every thread has at least `min_per_thread` terms.
LaunchCfg plan_grid(perm_handle h, const perm_opts& o, int block, int bps, uint64_t terms, uint64_t min_per_thread,
                    size_t record_bytes) {
  LaunchCfg lc;
  lc.block = o.block ? o.block : block;
  int grid = o.grid ? o.grid : h->sms * (bps > 0 ? bps : 1);
  uint64_t want = (terms + (uint64_t)lc.block * min_per_thread - 1) / ((uint64_t)lc.block * min_per_thread);
  if (!o.grid && want < (uint64_t)grid) grid = (int)(want > 0 ? want : 1);
  size_t cap = partials_capacity(h) / record_bytes;
  if ((size_t)grid > cap) grid = (int)cap;
  lc.grid = grid;
  lc.stream = nullptr;
  return lc;
}

SweepArgs sweep_args(const Call& c, uint64_t g0, uint64_t g1, int default_chunk);

// Real Glynn with the chunk-start column sums formed by a +-1 x A' contraction on the
// FP64 tensor cores (glynn_dmma.cu).
int glynn_dmma(Call& c, bool raw, uint64_t g0, uint64_t g1) {
  if (c.n > glynn_dmma_max_n()) return PERM_EUNSUPPORTED;
  const bool want_abs = c.dErr != nullptr;
  const int block = c.o.block ? c.o.block : 256;
  int bps = glynn_dmma_blocks_per_sm(c.n, block, want_abs);
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, g1 - g0, 32, (want_abs ? kCplxRecord : kRealRecord) * sizeof(double));
  lc.stream = c.stream;
  SweepArgs a = sweep_args(c, g0, g1, 14);
  if (!c.o.chunk_log2) {
    // chunks of 2^k terms, at least four rounds of 32 chunks per resident warp; with an
    // error bound at most 2^8 (the drift part of the bound grows with the chunk)
    const uint64_t warps = (uint64_t)lc.grid * (lc.block / 32);
    int k = want_abs ? 8 : 16;
    while (k > 2 && ((g1 - g0) >> k) < 128 * warps) --k;
    a.chunk_log2 = k;
  }
  if (launch_glynn_dmma(a, lc, want_abs) != cudaSuccess) return PERM_ECUDA;
  // as for the FP64 sweep: products and the Kahan sum against sum |term|, the column
  // sums' errors through the per-term widened products
  const double u = 1.1102230246251565e-16;
  const double coef = u * ((double)c.n + 4.0);
  const cudaError_t f =
      want_abs ? launch_finish_bound(static_cast<const double*>(a.partials), lc.grid, c.n - 1, c.n - c.m, coef,
                                     static_cast<double*>(c.dOut), c.dErr, raw, c.stream, 2.0 * u * (c.n + 1))
               : launch_finish_real(static_cast<const double*>(a.partials), lc.grid, c.n - 1, c.n - c.m, coef,
                                    static_cast<double*>(c.dOut), nullptr, raw, c.stream);
  if (f != cudaSuccess) return PERM_ECUDA;
  return PERM_OK;
}

int glynn_fp64(Call& c, bool raw, uint64_t g0, uint64_t g1) {
  if (c.o.start == PERM_START_DMMA) return glynn_dmma(c, raw, g0, g1);
  const bool want_abs = c.dErr != nullptr;
  const int block = 256;
  int bps = glynn_f64_blocks_per_sm(c.n, c.o.block ? c.o.block : block, want_abs);
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, g1 - g0, 16, (want_abs ? kCplxRecord : kRealRecord) * sizeof(double));
  lc.stream = c.stream;
  SweepArgs a;
  a.A = c.dA;
  a.m = c.m;
  a.n = c.n;
  a.rs = c.rs;
  a.cs = c.cs;
  a.g_begin = g0;
  a.g_end = g1;
  // with an error bound: column sums rebuilt every 2^8 terms (the drift term of the
  // bound grows with the chunk length; the rebuild costs n^2 / 2^8 per term)
  a.chunk_log2 = c.o.chunk_log2 ? c.o.chunk_log2 : (want_abs ? 8 : 14);
  a.start_mode = c.o.start ? c.o.start : PERM_START_SCALAR;
  a.partials = partials_base(c.h);
  if (launch_glynn_f64(a, lc, want_abs) != cudaSuccess) return PERM_ECUDA;
  // error bound: products (n-1 roundings) and the Kahan sum (2) against sum |term|; the
  // column sums' own errors (rebuild and drift, bounded by the columns' absolute sums)
  // through the per-term widened products; their FP64 evaluation (2 (n-1) u)
  const double u = 1.1102230246251565e-16;
  const double coef = u * ((double)c.n + 4.0);
  const cudaError_t f =
      want_abs ? launch_finish_bound(static_cast<const double*>(a.partials), lc.grid, c.n - 1, c.n - c.m, coef,
                                     static_cast<double*>(c.dOut), c.dErr, raw, c.stream, 2.0 * u * (c.n + 1))
               : launch_finish_real(static_cast<const double*>(a.partials), lc.grid, c.n - 1, c.n - c.m, coef,
                                    static_cast<double*>(c.dOut), nullptr, raw, c.stream);
  if (f != cudaSuccess) return PERM_ECUDA;
  return PERM_OK;
}


// Rectangular real Glynn with the padding rows summed in closed form (glynn_esym.cu):
// per(A) = 2^-(m-1) sum_d (prod d) e_m(c(d)).  Taken for m <= 32 when n - m >= 3 (or
// m <= 8): there the padded walk cancels far more (10^3 .. 10^16 times |per| on
// uniform entries) and e_m costs m n software multiply-adds per sign vector against
// (n - m + 1) n for the padded products.
bool use_esym(const Call& c) {
  return c.m < c.n && c.m <= glynn_esym_max_m() && (c.n - c.m >= 3 || c.m <= 8);
}

int glynn_esym_run(Call& c) {
  const bool want_abs = c.dErr != nullptr;
  const int block = glynn_esym_block();
  if (c.o.block > block) return PERM_EINVAL;
  const int nb = c.o.block ? c.o.block : block;
  const uint64_t g1 = 1ull << (c.m - 1);
  const int bps = glynn_esym_blocks_per_sm(c.m, c.n, nb, want_abs);
  if (bps <= 0) return PERM_ECUDA;
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, g1, 1, kCplxRecord * sizeof(double));
  lc.stream = c.stream;
  SweepArgs a = sweep_args(c, 0, g1, 0);
  if (!c.o.chunk_log2) {
    // chunks of 2^k sign vectors, four rounds of 32 chunks per resident warp if there are enough
    const uint64_t warps = (uint64_t)lc.grid * (lc.block / 32);
    int k = 12;
    while (k > 0 && (g1 >> k) < 128 * warps) --k;
    a.chunk_log2 = k;
  }
  static_assert(sizeof(EsymTable) <= kPartialsOffset - kFxTableOffset, "e_m table slot");
  EsymTable* tab = reinterpret_cast<EsymTable*>(fx_table(c.h));
  if (launch_glynn_esym(a, tab, lc, want_abs) != cudaSuccess) return PERM_ECUDA;
  // each product of the recurrence truncates by < 2^-60, each sum by < 2^-60 of the
  // larger operand: relative to e_m(|c|), m + n roundings; 4 more for the
  // accumulator window, the double-double reduction and the sums of the bound itself
  const double coef = std::ldexp((double)(c.m + c.n) + 4.0, -60);
  if (launch_esym_finish(static_cast<const double*>(a.partials), lc.grid, c.m, coef, static_cast<double*>(c.dOut),
                         c.dErr, c.stream) != cudaSuccess)
    return PERM_ECUDA;
  return PERM_OK;
}

// Real Glynn on the integer pipes: exact fixed-point column sums, 64-bit-mantissa
// products, 192-bit accumulation (glynn_fx.cu).
int glynn_fixed(Call& c, bool raw, uint64_t g0, uint64_t g1, bool mixed) {
  const bool want_abs = c.dErr != nullptr;
  if (!raw && use_esym(c)) return glynn_esym_run(c);
  // a whole rectangular permanent: the grouped walk over the real rows' sign vectors
  const bool grouped = !raw && c.m < c.n;
  // the lane-pair sweep (24 warps per SM) for a mixed square sweep without a bound,
  // unless a block of at most the one-lane kernel's size is asked for; otherwise 6
  // warps, two blocks per SM at up to 168 registers (from N = 40: 4 warps)
  const bool pair = !grouped && mixed && !want_abs && glynn_fx_pair_available(c.n) &&
                    (c.o.block == 0 || c.o.block > glynn_fx_block(c.n));
  const int block = grouped ? 192 : pair ? glynn_fx_pair_block() : glynn_fx_block(c.n);
  if (c.o.block > block || (pair && c.o.block && c.o.block != block)) return PERM_EINVAL;
  if (grouped) {
    g0 = 0;
    g1 = 1ull << (c.m - 1);
  }
  const int bps = grouped ? glynn_fxg_blocks_per_sm(c.m, c.n, c.o.block ? c.o.block : block)
                          : glynn_fx_blocks_per_sm(c.n, c.o.block ? c.o.block : block, mixed, pair);
  const uint64_t work = grouped ? (g1 - g0) * (uint64_t)(c.n - c.m + 1) : g1 - g0;
  // with an error bound both sweeps write {sum, sum |term|, eta-widened sum}
  const bool three = want_abs;
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, work, 16, (three ? kCplxRecord : kRealRecord) * sizeof(double));
  lc.stream = c.stream;
  SweepArgs a = sweep_args(c, g0, g1, 12);
  if (!c.o.chunk_log2) {
    // aligned chunks of 2^k steps, at least 32 rounds of 32 chunks per resident warp
    const uint64_t warps = (uint64_t)lc.grid * (lc.block / 32);
    const uint64_t per_step = grouped ? (uint64_t)(c.n - c.m + 1) : 1;
    int k = 12;
    while (k > (grouped ? 0 : 2) && ((g1 - g0) >> k) * per_step < 1024 * warps) --k;
    a.chunk_log2 = k;
  }
  // the 192-bit accumulator holds 2^40 maximal terms per chunk (2^6 per grouped step)
  if (a.chunk_log2 > (grouped ? 34 : 40)) return PERM_ETOOBIG;
  const cudaError_t e = grouped ? launch_glynn_fxg(a, fx_table(c.h), lc, want_abs)
                                : launch_glynn_fx(a, fx_table(c.h), lc, want_abs, mixed, pair);
  if (e != cudaSuccess) return PERM_ECUDA;
  // relative error of a term against |term|: n/2 pair products of < 2^-59 each (the
  // running mantissa keeps >= 60 bits), the binomial weight of a grouped term (< 2^-62);
  // the mixed variant's K columns: K conversions and K - 1 multiplications in FP64.
  // The bound variants take exact magnitudes and bound the rounding of A to fixed
  // point by their eta-widened products (zero when every entry was exact)
  const int K = (mixed && !grouped) ? (pair ? glynn_fx_pair_mixed_columns(c.n) : glynn_fx_mixed_columns(c.n)) : 0;
  const double coef = std::ldexp((double)(c.n - K) + 5.0, -60) + std::ldexp(2.0 * K, -53);
  const cudaError_t f = three ? launch_finish_bound(static_cast<const double*>(a.partials), lc.grid, c.n - 1, c.n - c.m,
                                                    coef, static_cast<double*>(c.dOut), c.dErr, raw, c.stream)
                              : launch_finish_real(static_cast<const double*>(a.partials), lc.grid, c.n - 1, c.n - c.m,
                                                   coef, static_cast<double*>(c.dOut), c.dErr, raw, c.stream);
  if (f != cudaSuccess) return PERM_ECUDA;
  return PERM_OK;
}

// Complex Glynn on the integer pipes: FIXED or MIXED asked for, or AUTO from n = 10;
// not when an error bound is asked for (the complex integer-pipe sweep states none).
bool cplx_glynn_on_integer_pipes(const Call& c) {
  return c.n <= glynn_cfx_max_n() && !c.dErr &&
         (c.o.arith == PERM_ARITH_FIXED || c.o.arith == PERM_ARITH_MIXED ||
          (c.o.arith == PERM_ARITH_AUTO && c.n >= 10));
}

bool real_glynn_on_integer_pipes(const Call& c) {
  return c.o.arith == PERM_ARITH_FIXED || c.o.arith == PERM_ARITH_MIXED ||
         (c.o.arith == PERM_ARITH_AUTO && c.o.start != PERM_START_DMMA && c.n >= 10);
}

// Real Glynn: the integer-pipe sweep by default (faster on GB300 and at least as
// accurate), mixed with the FP64 unit unless FIXED is asked for; the FP64 sweep when
// asked for or when the tensor-core chunk starts are.
int glynn_real(Call& c, bool raw, uint64_t g0, uint64_t g1) {
  if (c.o.arith == PERM_ARITH_FIXED) return glynn_fixed(c, raw, g0, g1, false);
  if (real_glynn_on_integer_pipes(c)) return glynn_fixed(c, raw, g0, g1, true);
  return glynn_fp64(c, raw, g0, g1);
}

SweepArgs sweep_args(const Call& c, uint64_t g0, uint64_t g1, int default_chunk) {
  SweepArgs a;
  a.A = c.dA;
  a.m = c.m;
  a.n = c.n;
  a.rs = c.rs;
  a.cs = c.cs;
  a.g_begin = g0;
  a.g_end = g1;
  a.chunk_log2 = c.o.chunk_log2 ? c.o.chunk_log2 : default_chunk;
  a.start_mode = c.o.start ? c.o.start : PERM_START_SCALAR;
  a.want_abs = 0;
  a.partials = partials_base(c.h);
  return a;
}

// Complex rectangle with the padding summed in closed form (glynn_cesym.cu), for every
// m <= 32: on complex Gaussian rectangles the padded walk cancels 10^6-fold already
// at n - m = 1.
int glynn_cesym_run(Call& c) {
  const int block = glynn_cesym_block();
  if (c.o.block > block) return PERM_EINVAL;
  const int nb = c.o.block ? c.o.block : block;
  const uint64_t g1 = 1ull << (c.m - 1);
  const int bps = glynn_cesym_blocks_per_sm(c.m, c.n, nb);
  if (bps <= 0) return PERM_ECUDA;
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, g1, 1, kCplxRecord * sizeof(double));
  lc.stream = c.stream;
  SweepArgs a = sweep_args(c, 0, g1, 0);
  if (!c.o.chunk_log2) {
    const uint64_t warps = (uint64_t)lc.grid * (lc.block / 32);
    int k = 12;
    while (k > 0 && (g1 >> k) < 128 * warps) --k;
    a.chunk_log2 = k;
  }
  static_assert(sizeof(CesymTable) <= kPartialsOffset - kFxTableOffset, "complex e_m table slot");
  CesymTable* tab = reinterpret_cast<CesymTable*>(fx_table(c.h));
  if (launch_glynn_cesym(a, tab, lc) != cudaSuccess) return PERM_ECUDA;
  if (c.dErr && launch_write_double(-1.0, c.dErr, c.stream) != cudaSuccess) return PERM_ECUDA;
  if (launch_finish_cplx(static_cast<const double*>(a.partials), lc.grid, c.m - 1, 0, 0.0,
                         static_cast<double*>(c.dOut), nullptr, false, c.stream) != cudaSuccess)
    return PERM_ECUDA;
  return PERM_OK;
}

// Complex Glynn on the integer pipes (glynn_cfx.cu).
int glynn_cfixed(Call& c, bool raw, uint64_t g0, uint64_t g1) {
  if (c.o.block > 128) return PERM_EINVAL;
  if (!raw && c.m < c.n && c.m <= glynn_cesym_max_m()) return glynn_cesym_run(c);
  const int block = c.n <= 40 ? 128 : 64;  // shared memory: 32 n^2 + 16 n per thread bytes
  // a whole rectangular permanent: the grouped walk over the real rows' sign vectors
  const bool grouped = !raw && c.m < c.n;
  if (grouped) {
    g0 = 0;
    g1 = 1ull << (c.m - 1);
  }
  int bps = glynn_cfx_blocks_per_sm(c.m, c.n, c.o.block ? c.o.block : block, grouped);
  const uint64_t per_step = grouped ? (uint64_t)(c.n - c.m + 1) : 1;
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, (g1 - g0) * per_step, 16, kCplxRecord * sizeof(double));
  lc.stream = c.stream;
  SweepArgs a = sweep_args(c, g0, g1, 12);
  if (!c.o.chunk_log2) {
    const uint64_t warps = (uint64_t)lc.grid * (lc.block / 32);
    int k = 12;
    while (k > (grouped ? 0 : 2) && ((g1 - g0) >> k) * per_step < 1024 * warps) --k;
    a.chunk_log2 = k;
  }
  // MIXED: about 3/8 of the columns of each product on the FP64 unit.  Not the default:
  // +10% / +6% at n = 26 / 32 on uniform entries, -7% on the 32x32 Gaussian workload.
  if (!grouped && c.o.arith == PERM_ARITH_MIXED && c.n >= 20) a.fp64_cols = (3 * c.n) / 8;
  // 2^40 maximal terms per 192-bit accumulator (2^6 per grouped step)
  if (a.chunk_log2 > (grouped ? 34 : 40)) return PERM_ETOOBIG;
  if (launch_glynn_cfx(a, cfx_table(c.h), lc, grouped) != cudaSuccess) return PERM_ECUDA;
  if (c.dErr && launch_write_double(-1.0, c.dErr, c.stream) != cudaSuccess) return PERM_ECUDA;
  if (launch_finish_cplx(static_cast<const double*>(a.partials), lc.grid, c.n - 1, c.n - c.m, 0.0,
                         static_cast<double*>(c.dOut), nullptr, raw, c.stream) != cudaSuccess)
    return PERM_ECUDA;
  return PERM_OK;
}

int glynn_cplx(Call& c, bool raw, uint64_t g0, uint64_t g1) {
  if (cplx_glynn_on_integer_pipes(c)) return glynn_cfixed(c, raw, g0, g1);
  if (c.n > glynn_c128_max_n()) return PERM_ETOOBIG;
  if (c.o.block > 128) return PERM_EINVAL;
  const bool want_abs = c.dErr != nullptr;
  const int block = 128;
  int bps = glynn_c128_blocks_per_sm(c.n, c.o.block ? c.o.block : block, want_abs);
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, g1 - g0, 16, kCplxRecord * sizeof(double));
  lc.stream = c.stream;
  SweepArgs a = sweep_args(c, g0, g1, want_abs ? 8 : 14);  // shorter chunks bound the drift tighter
  if (launch_glynn_c128(a, lc, want_abs) != cudaSuccess) return PERM_ECUDA;
  // the bound variant accumulates each term's full bound (rounding of the products and
  // the widened difference for the column sums' errors); its own FP64 sum of positive
  // terms is inflated by 2^-20
  const double coef = 1.0 + 0x1p-20;
  if (launch_finish_cplx(static_cast<const double*>(a.partials), lc.grid, c.n - 1, c.n - c.m, coef,
                         static_cast<double*>(c.dOut), c.dErr, raw, c.stream) != cudaSuccess)
    return PERM_ECUDA;
  return PERM_OK;
}

int glynn_integer(Call& c, bool raw, uint64_t g0, uint64_t g1) {
  const int block = 256;
  // a whole rectangular permanent: the grouped walk over the real rows' sign vectors
  const bool grouped = !raw && c.m < c.n;
  if (grouped) {
    g0 = 0;
    g1 = 1ull << (c.m - 1);
  }
  int bps = glynn_int_blocks_per_sm(c.n, c.dtype, c.o.block ? c.o.block : block, grouped);
  const uint64_t work = grouped ? (g1 - g0) * (uint64_t)(c.n - c.m + 1) : g1 - g0;
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, work, 16, kIntRecord * sizeof(unsigned long long));
  lc.stream = c.stream;
  SweepArgs a = sweep_args(c, g0, g1, 62);
  int* st = c.hOut ? call_status_word(c.h) : status_word(c.h);
  if (c.hOut && cudaMemsetAsync(st, 0, sizeof(int), c.stream) != cudaSuccess) return PERM_ECUDA;
  if (!raw && launch_int_bound(c.dA, c.dtype, c.m, c.n, c.rs, c.cs, st, c.stream) != cudaSuccess) return PERM_ECUDA;
  if (launch_glynn_int(a, c.dtype, lc, grouped) != cudaSuccess) return PERM_ECUDA;
  if (c.dErr && cudaMemsetAsync(c.dErr, 0, sizeof(double), c.stream) != cudaSuccess) return PERM_ECUDA;
  if (launch_finish_int(static_cast<const unsigned long long*>(a.partials), lc.grid, c.n - 1, c.n - c.m,
                        static_cast<unsigned long long*>(c.dOut), raw, c.stream) != cudaSuccess)
    return PERM_ECUDA;
  return PERM_OK;
}

// Glynn for Gaussian integers, exact modulo 2^128 per component (glynn_int.cu).
int glynn_gaussian(Call& c, bool raw, uint64_t g0, uint64_t g1) {
  if (c.n > glynn_gaussian_max_n()) return PERM_ETOOBIG;
  const int block = 128;
  if (c.o.block > block) return PERM_EINVAL;
  int bps = glynn_gaussian_blocks_per_sm(c.n, c.o.block ? c.o.block : block);
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, g1 - g0, 16, 2 * kIntRecord * sizeof(unsigned long long));
  lc.stream = c.stream;
  SweepArgs a = sweep_args(c, g0, g1, 62);
  int* st = c.hOut ? call_status_word(c.h) : status_word(c.h);
  if (c.hOut && cudaMemsetAsync(st, 0, sizeof(int), c.stream) != cudaSuccess) return PERM_ECUDA;
  if (!raw && launch_int_bound(c.dA, c.dtype, c.m, c.n, c.rs, c.cs, st, c.stream) != cudaSuccess) return PERM_ECUDA;
  if (launch_glynn_gaussian(a, lc) != cudaSuccess) return PERM_ECUDA;
  if (c.dErr && cudaMemsetAsync(c.dErr, 0, sizeof(double), c.stream) != cudaSuccess) return PERM_ECUDA;
  const unsigned long long* rec = static_cast<const unsigned long long*>(a.partials);
  unsigned long long* out = static_cast<unsigned long long*>(c.dOut);
  if (launch_finish_int(rec, lc.grid, c.n - 1, c.n - c.m, out, raw, c.stream) != cudaSuccess ||
      launch_finish_int(rec + kIntRecord * lc.grid, lc.grid, c.n - 1, c.n - c.m, out + 2, raw, c.stream) !=
          cudaSuccess)
    return PERM_ECUDA;
  return PERM_OK;
}

double binomial_d(int a, int b) {
  if (b < 0 || b > a) return 0.0;
  unsigned __int128 r = 1;
  for (int i = 1; i <= b; ++i) r = r * (unsigned __int128)(a - b + i) / (unsigned __int128)i;
  return (double)r;
}

// Ryser over the 2^n column subsets (square: Eq. ryser_square; m < n: the subset-size
// weights of Eq. ryser_rectangle).
// Rectangular Ryser visiting only the subsets of size <= m, by size in colex order.
int ryser_by_size(Call& c, unsigned long long total) {
  if (total > (c.o.max_terms ? c.o.max_terms : (1ull << 44))) return PERM_ETOOBIG;
  const int block = 256;
  int bps = ryser_colex_blocks_per_sm(c.m, c.n, c.o.block ? c.o.block : block);
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, total, 16, kRealRecord * sizeof(double));
  lc.stream = c.stream;
  SweepArgs a = sweep_args(c, 0, total, 14);
  SizeWeights w;
  SizeCounts cum;
  unsigned long long run = 0;
  for (int s = 0; s <= 64; ++s) {
    w.w[s] = 0.0;
    if (s <= c.m) w.w[s] = (((c.m - s) & 1) ? -1.0 : 1.0) * binomial_d(c.n - s, c.m - s);
  }
  for (int s = 0; s < 66; ++s) cum.c[s] = 0;
  for (int s = 1; s <= c.m + 1 && s < 66; ++s) {
    cum.c[s] = run;
    if (s <= c.m) {
      unsigned __int128 b = 1;  // exact C(n, s)
      for (int i = 1; i <= s; ++i) b = b * (unsigned __int128)(c.n - s + i) / (unsigned __int128)i;
      run += (unsigned long long)b;
    }
  }
  if (run != total) return PERM_ETOOBIG;
  if (launch_ryser_colex(a, w, cum, lc) != cudaSuccess) return PERM_ECUDA;
  if (c.dErr && launch_write_double(-1.0, c.dErr, c.stream) != cudaSuccess) return PERM_ECUDA;
  if (launch_finish_real(static_cast<const double*>(a.partials), lc.grid, 0, 0, 0.0, static_cast<double*>(c.dOut),
                         nullptr, false, c.stream) != cudaSuccess)
    return PERM_ECUDA;
  return PERM_OK;
}

// Real Ryser over the 2^n Gray-ordered subsets on the integer pipes (ryser_fx.cu):
// exact fixed-point row sums, 64-bit-mantissa products, 192-bit accumulation.
int ryser_fixed(Call& c) {
  if (c.n > 62) return PERM_ETOOBIG;
  const uint64_t terms = 1ull << c.n;
  if (terms > (c.o.max_terms ? c.o.max_terms : (1ull << 44))) return PERM_ETOOBIG;
  const bool want_abs = c.dErr != nullptr;
  const int block = ryser_fx_block(c.m);
  if (c.o.block > block) return PERM_EINVAL;
  const int bps = ryser_fx_blocks_per_sm(c.m, c.n, c.o.block ? c.o.block : block, want_abs);
  if (bps <= 0) return PERM_ECUDA;
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, terms, 16, (want_abs ? kCplxRecord : kRealRecord) * sizeof(double));
  lc.stream = c.stream;
  SweepArgs a = sweep_args(c, 0, terms, 12);
  if (!c.o.chunk_log2) {
    const uint64_t warps = (uint64_t)lc.grid * (lc.block / 32);
    int k = 12;
    while (k > 2 && (terms >> k) < 1024 * warps) --k;
    a.chunk_log2 = k;
  }
  // 2^40 maximal terms per 192-bit accumulator
  if (a.chunk_log2 > 40) return PERM_ETOOBIG;
  // rectangles: chunks in the size-coherent order when there are enough of them
  // (start_mode 1; a square needs every subset, so order buys it nothing)
  a.start_mode = (c.m < c.n && c.n - a.chunk_log2 >= 6) ? 1 : 0;
  if (launch_ryser_fx(a, fx_table(c.h), lc, want_abs) != cudaSuccess) return PERM_ECUDA;
  // per term: m/2 pair products (< 2^-59 each), the binomial weight (< 2^-62), and the
  // accumulation; the rounding of A to fixed point is bounded by the eta-widened sum
  const double coef = std::ldexp((double)c.m + 6.0, -60);
  const cudaError_t f = want_abs ? launch_finish_bound(static_cast<const double*>(a.partials), lc.grid, 0, 0, coef,
                                                       static_cast<double*>(c.dOut), c.dErr, false, c.stream)
                                 : launch_finish_real(static_cast<const double*>(a.partials), lc.grid, 0, 0, coef,
                                                      static_cast<double*>(c.dOut), nullptr, false, c.stream);
  if (f != cudaSuccess) return PERM_ECUDA;
  return PERM_OK;
}

bool real_ryser_on_integer_pipes(const Call& c) {
  return c.o.arith == PERM_ARITH_FIXED || c.o.arith == PERM_ARITH_MIXED || (c.o.arith == PERM_ARITH_AUTO && c.n >= 10);
}

int ryser_real(Call& c, bool raw, uint64_t g0, uint64_t g1) {
  if (!raw && c.m < c.n) {
    // by size when the subsets of size <= m are few compared with all 2^n
    long double by_size = 0.0L;
    for (int s = 1; s <= c.m; ++s) by_size += (long double)binomial_d(c.n, s);
    if (by_size * 3.0L < std::ldexp(1.0L, c.n) && by_size < 1.8e19L) return ryser_by_size(c, (unsigned long long)by_size);
  }
  if (!raw && real_ryser_on_integer_pipes(c)) return ryser_fixed(c);
  if (c.n > 62) return PERM_ETOOBIG;
  const uint64_t terms = raw ? g1 - g0 : (1ull << c.n);
  if (!raw) g1 = terms;
  if (terms > (c.o.max_terms ? c.o.max_terms : (1ull << 44))) return PERM_ETOOBIG;
  const bool want_abs = c.dErr != nullptr;
  const bool weighted = c.m < c.n;
  const int block = 256;
  int bps = ryser_f64_blocks_per_sm(c.m, c.n, c.o.block ? c.o.block : block, weighted, want_abs);
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, terms, 16, (want_abs ? kCplxRecord : kRealRecord) * sizeof(double));
  lc.stream = c.stream;
  SweepArgs a = sweep_args(c, g0, g1, want_abs ? 8 : 14);  // shorter chunks bound the drift tighter
  SizeWeights w;
  for (int s = 0; s <= 64; ++s) {
    w.w[s] = 0.0;
    if (s <= c.n && s <= c.m) w.w[s] = (((c.m - s) & 1) ? -1.0 : 1.0) * binomial_d(c.n - s, c.m - s);
  }
  if (launch_ryser_f64(a, w, lc, want_abs) != cudaSuccess) return PERM_ECUDA;
  // m - 1 product roundings, the weight, the Kahan sum against sum |term|; the row
  // sums' own errors through the widened products (2 (m + 1) u for their evaluation)
  const double u = 1.1102230246251565e-16;
  const double coef = u * ((double)c.m + 5.0);
  const double sign = (!weighted && (c.n & 1)) ? -1.0 : 1.0;
  cudaError_t f;
  if (want_abs) {
    // the sign (-1)^n of the unweighted square sum is applied to the partial records
    f = sign < 0 ? launch_negate_records(static_cast<double*>(a.partials), lc.grid, kCplxRecord, c.stream) : cudaSuccess;
    if (f == cudaSuccess)
      f = launch_finish_bound(static_cast<const double*>(a.partials), lc.grid, 0, 0, coef, static_cast<double*>(c.dOut),
                              c.dErr, raw, c.stream, 2.0 * u * (c.m + 1));
  } else {
    f = launch_finish_real(static_cast<const double*>(a.partials), lc.grid, 0, 0, coef, static_cast<double*>(c.dOut),
                           nullptr, raw, c.stream, sign);
  }
  if (f != cudaSuccess) return PERM_ECUDA;
  return PERM_OK;
}

// Ryser for complex and integer input (ryser_ext.cu): all weights carry the sign.
int ryser_other(Call& c) {
  if (c.n > 62) return PERM_ETOOBIG;
  const uint64_t terms = 1ull << c.n;
  if (terms > (c.o.max_terms ? c.o.max_terms : (1ull << 44))) return PERM_ETOOBIG;
  if (c.dtype == PERM_C128 && c.m > 40) return PERM_EUNSUPPORTED;
  if (c.dtype == PERM_CI64 && c.m > 32) return PERM_ETOOBIG;
  const int block = c.dtype == PERM_C128 ? 128 : 256;
  if (c.o.block > block) return PERM_EINVAL;
  int bps = ryser_ext_blocks_per_sm(c.m, c.n, c.dtype, c.o.block ? c.o.block : block);
  const size_t rec = c.dtype == PERM_C128 ? kCplxRecord * 8 : (c.dtype == PERM_CI64 ? 2 : 1) * kIntRecord * 8;
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, terms, 16, rec);
  lc.stream = c.stream;
  SweepArgs a = sweep_args(c, 0, terms, 14);
  SizeWeights fw;
  IntWeights iw;
  for (int s = 0; s <= 64; ++s) {
    fw.w[s] = 0.0;
    iw.lo[s] = iw.hi[s] = 0;
    if (s <= c.m) {
      unsigned __int128 b = 1;
      for (int i = 1; i <= c.m - s; ++i) b = b * (unsigned __int128)(c.n - s - (c.m - s) + i) / (unsigned __int128)i;
      const bool neg = ((c.m - s) & 1) != 0;
      fw.w[s] = (neg ? -1.0 : 1.0) * (double)b;
      const unsigned __int128 v = neg ? (unsigned __int128)0 - b : b;
      iw.lo[s] = (unsigned long long)v;
      iw.hi[s] = (unsigned long long)(v >> 64);
    }
  }
  if (c.dtype != PERM_C128) {
    int* st = c.hOut ? call_status_word(c.h) : status_word(c.h);
    if (c.hOut && cudaMemsetAsync(st, 0, sizeof(int), c.stream) != cudaSuccess) return PERM_ECUDA;
    if (launch_int_bound(c.dA, c.dtype, c.m, c.n, c.rs, c.cs, st, c.stream) != cudaSuccess) return PERM_ECUDA;
  }
  if (launch_ryser_ext(a, c.dtype, fw, iw, lc) != cudaSuccess) return PERM_ECUDA;
  cudaError_t e;
  if (c.dtype == PERM_C128) {
    const double u = 1.1102230246251565e-16;
    e = launch_finish_cplx(static_cast<const double*>(a.partials), lc.grid, 0, 0, u, static_cast<double*>(c.dOut),
                           nullptr, false, c.stream);
    if (e == cudaSuccess && c.dErr) e = launch_write_double(-1.0, c.dErr, c.stream);
  } else {
    const unsigned long long* recs = static_cast<const unsigned long long*>(a.partials);
    unsigned long long* out = static_cast<unsigned long long*>(c.dOut);
    e = launch_finish_int(recs, lc.grid, 0, 0, out, false, c.stream);
    if (e == cudaSuccess && c.dtype == PERM_CI64)  // imaginary parts after the real ones
      e = launch_finish_int(recs + kIntRecord * lc.grid, lc.grid, 0, 0, out + 2, false, c.stream);
    if (e == cudaSuccess && c.dErr) e = cudaMemsetAsync(c.dErr, 0, sizeof(double), c.stream);
  }
  return e == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

// The combinatoric algorithm over all injective maps (combinatoric.cu).
int combinatoric_run(Call& c) {
  // dense count of injective maps n!/(n-m)! (sparse inputs are pruned, so this bounds the work)
  long double leaves = 1.0L;
  for (int k = 0; k < c.m; ++k) leaves *= (long double)(c.n - k);
  const uint64_t cap = c.o.max_terms ? c.o.max_terms : (1ull << 44);
  if (leaves > (long double)cap) return PERM_ETOOBIG;
  const int block = combinatoric_block(c.m, c.n, c.dtype);
  if (c.o.block > block) return PERM_EINVAL;
  int bps = combinatoric_blocks_per_sm(c.m, c.n, c.dtype, c.o.block ? c.o.block : block);
  const size_t rec = (c.dtype == PERM_F64)    ? kRealRecord * 8
                     : (c.dtype == PERM_C128) ? kCplxRecord * 8
                                              : (c.dtype == PERM_CI64 ? 2 : 1) * kIntRecord * 8;
  LaunchCfg lc = plan_grid(c.h, c.o, block, bps, ~0ull >> 1, 1, rec);
  lc.stream = c.stream;
  const uint64_t threads = (uint64_t)lc.grid * lc.block;
  int depth = 0;
  uint64_t prefixes = 1;
  // at most down to the level above the first table level (below it a prefix would be
  // one table step, and unranking it would cost more than the step)
  const int max_depth = std::max(c.m - combinatoric_table_rows(c.m, c.n, c.dtype) - 1, 0);
  const int depth_cap = combinatoric_table_rows(c.m, c.n, c.dtype) ? max_depth : c.m;
  while (depth < depth_cap && prefixes < 8 * threads) {
    prefixes *= (uint64_t)(c.n - depth);
    ++depth;
  }
  if (!c.o.grid && prefixes < threads) lc.grid = (int)((prefixes + lc.block - 1) / lc.block);
  SweepArgs a = sweep_args(c, 0, 0, 0);
  const bool integer = c.dtype == PERM_U8 || c.dtype == PERM_I64 || c.dtype == PERM_CI64;
  if (integer) {  // the sum of products is exact while per(|A|) < 2^126.5
    int* st = c.hOut ? call_status_word(c.h) : status_word(c.h);
    if (c.hOut && cudaMemsetAsync(st, 0, sizeof(int), c.stream) != cudaSuccess) return PERM_ECUDA;
    if (launch_int_bound(c.dA, c.dtype, c.m, c.n, c.rs, c.cs, st, c.stream, false) != cudaSuccess) return PERM_ECUDA;
  }
  if (launch_combinatoric(a, c.dtype, depth, prefixes, lc) != cudaSuccess) return PERM_ECUDA;
  if (c.dErr && launch_write_double(-1.0, c.dErr, c.stream) != cudaSuccess) return PERM_ECUDA;
  cudaError_t e;
  if (c.dtype == PERM_F64)
    e = launch_finish_real(static_cast<const double*>(a.partials), lc.grid, 0, 0, 0.0, static_cast<double*>(c.dOut),
                           nullptr, false, c.stream);
  else if (c.dtype == PERM_C128)
    e = launch_finish_cplx(static_cast<const double*>(a.partials), lc.grid, 0, 0, 0.0, static_cast<double*>(c.dOut),
                           nullptr, false, c.stream);
  else {
    const unsigned long long* recs = static_cast<const unsigned long long*>(a.partials);
    unsigned long long* out = static_cast<unsigned long long*>(c.dOut);
    e = launch_finish_int(recs, lc.grid, 0, 0, out, false, c.stream);
    if (e == cudaSuccess && c.dtype == PERM_CI64)  // imaginary parts after the real ones
      e = launch_finish_int(recs + kIntRecord * lc.grid, lc.grid, 0, 0, out + 2, false, c.stream);
  }
  return e == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

uint64_t max_terms(const perm_opts& o) { return o.max_terms ? o.max_terms : kDefaultMaxTerms; }

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Grow the staging / scratch buffer of perm_sbp and perm_cauchy (not during capture).
int ensure_sws(perm_handle h, size_t need) {
  if (need <= h->sws_bytes) return PERM_OK;
  if (h->sws) {
    if (cudaDeviceSynchronize() != cudaSuccess) return PERM_ECUDA;
    cudaFree(h->sws);
    h->sws = nullptr;
    h->sws_bytes = 0;
  }
  if (cudaMalloc(&h->sws, need) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  h->sws_bytes = need;
  return PERM_OK;
}

}  // namespace perm

using namespace perm;

extern "C" {

int perm_version(void) { return 100; }

const char* perm_status_string(int s) {
  switch (s) {
    case PERM_OK: return "ok";
    case PERM_EINVAL: return "invalid argument";
    case PERM_ETOOBIG: return "problem too large (max(m, n) > 64 or more terms than max_terms)";
    case PERM_EOVERFLOW: return "integer result may not fit in int128";
    case PERM_ECUDA: return "CUDA runtime error";
    case PERM_ENOMEM: return "workspace allocation failed";
    case PERM_EUNSUPPORTED: return "unsupported combination of dtype, algorithm and options";
    default: return "unknown status";
  }
}

int perm_create(perm_handle* out, int device) {
  if (!out) return PERM_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return PERM_ECUDA;
  perm_handle h = new (std::nothrow) perm_handle_s;
  if (!h) return PERM_ENOMEM;
  h->device = device;
  if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete h;
    return PERM_ECUDA;
  }
  int rc = ensure_ws(h, kWsDefault, nullptr);
  if (rc) {
    delete h;
    return rc;
  }

  *out = h;
  return PERM_OK;
}

int perm_destroy(perm_handle h) {
  if (!h) return PERM_EINVAL;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  if (h->ws) cudaFree(h->ws);
  if (h->sws) cudaFree(h->sws);
  batched_release(h);
  delete h;
  return PERM_OK;
}

int perm_device_status(perm_handle h, void* stream, int* status) {
  if (!h || !status) return PERM_EINVAL;
  if (cudaSetDevice(h->device) != cudaSuccess) return PERM_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int v = 0;
  if (cudaMemcpyAsync(&v, status_word(h), sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PERM_ECUDA;
  if (cudaMemsetAsync(status_word(h), 0, sizeof(int), s) != cudaSuccess) return PERM_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PERM_ECUDA;
  *status = v;
  return PERM_OK;
}

int perm_glynn(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, void* out, void* stream,
               const perm_opts* opts) {
  Call c;
  int rc = prepare(c, h, A, m, n, ld, dtype, out, stream, opts, true);
  if (rc) return rc;
  if (c.m == 0) {
    if (launch_write_one(dtype, c.dOut, c.stream) != cudaSuccess) return PERM_ECUDA;
    if (c.dErr && cudaMemsetAsync(c.dErr, 0, sizeof(double), c.stream) != cudaSuccess) return PERM_ECUDA;
    return finish(c, out_size(dtype));
  }
  const uint64_t terms = 1ull << (c.n - 1);
  // the integer-pipe walk of a real rectangle visits 2^(m-1) (n-m+1) grouped terms
  const bool grouped = c.m < c.n && ((dtype == PERM_F64 && real_glynn_on_integer_pipes(c)) ||
                                     (dtype == PERM_C128 && cplx_glynn_on_integer_pipes(c)) ||
                                     dtype == PERM_U8 || dtype == PERM_I64);
  const uint64_t visited = grouped ? (1ull << (c.m - 1)) * (uint64_t)(c.n - c.m + 1) : terms;
  if (visited > max_terms(c.o)) return PERM_ETOOBIG;
  switch (dtype) {
    case PERM_F64: rc = glynn_real(c, false, 0, terms); break;
    case PERM_C128: rc = glynn_cplx(c, false, 0, terms); break;
    case PERM_CI64: rc = glynn_gaussian(c, false, 0, terms); break;
    default: rc = glynn_integer(c, false, 0, terms); break;
  }
  if (rc) return rc;
  return finish(c, out_size(dtype));
}

int perm_glynn_partial(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, uint64_t g_begin,
                       uint64_t g_end, void* partial, void* stream, const perm_opts* opts) {
  Call c;
  if (m > n || m < 1) return PERM_EINVAL;
  int rc = prepare(c, h, A, m, n, ld, dtype, partial, stream, opts, false);
  if (rc) return rc;
  const uint64_t terms = 1ull << (c.n - 1);
  if (g_begin > g_end || g_end > terms) return PERM_EINVAL;
  if (g_end - g_begin > max_terms(c.o)) return PERM_ETOOBIG;
  size_t bytes = 0;
  switch (dtype) {
    case PERM_F64:
      rc = glynn_real(c, true, g_begin, g_end);
      bytes = 16;
      break;
    case PERM_C128:
      rc = glynn_cplx(c, true, g_begin, g_end);
      bytes = 32;
      break;
    case PERM_CI64:
      rc = glynn_gaussian(c, true, g_begin, g_end);
      bytes = 32;
      break;
    default:
      rc = glynn_integer(c, true, g_begin, g_end);
      bytes = 16;
      break;
  }
  if (rc) return rc;
  return finish(c, bytes);
}

int perm_ryser_partial(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, uint64_t g_begin,
                       uint64_t g_end, void* partial, void* stream, const perm_opts* opts) {
  Call c;
  if (m > n || m < 1) return PERM_EINVAL;
  if (dtype != PERM_F64) return PERM_EUNSUPPORTED;
  int rc = prepare(c, h, A, m, n, ld, dtype, partial, stream, opts, false);
  if (rc) return rc;
  if (c.n > 62) return PERM_ETOOBIG;
  if (g_begin > g_end || g_end > (1ull << c.n)) return PERM_EINVAL;
  rc = ryser_real(c, true, g_begin, g_end);
  if (rc) return rc;
  return finish(c, 16);
}

int perm_ryser(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, void* out, void* stream,
               const perm_opts* opts) {
  Call c;
  int rc = prepare(c, h, A, m, n, ld, dtype, out, stream, opts, true);
  if (rc) return rc;
  if (c.m == 0) {
    if (launch_write_one(dtype, c.dOut, c.stream) != cudaSuccess) return PERM_ECUDA;
    if (c.dErr && cudaMemsetAsync(c.dErr, 0, sizeof(double), c.stream) != cudaSuccess) return PERM_ECUDA;
    return finish(c, out_size(dtype));
  }
  switch (dtype) {
    case PERM_F64: rc = ryser_real(c); break;
    default: rc = ryser_other(c); break;
  }
  if (rc) return rc;
  return finish(c, out_size(dtype));
}

int perm_combinatoric(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, void* out,
                      void* stream, const perm_opts* opts) {
  Call c;
  int rc = prepare(c, h, A, m, n, ld, dtype, out, stream, opts, true);
  if (rc) return rc;
  if (c.m == 0) {
    if (launch_write_one(dtype, c.dOut, c.stream) != cudaSuccess) return PERM_ECUDA;
    if (c.dErr && cudaMemsetAsync(c.dErr, 0, sizeof(double), c.stream) != cudaSuccess) return PERM_ECUDA;
    return finish(c, out_size(dtype));
  }
  rc = combinatoric_run(c);
  if (rc) return rc;
  return finish(c, out_size(dtype));
}

int perm_batched(perm_handle h, const void* packed, const int64_t* offsets, const int32_t* M, const int32_t* N,
                 int64_t count, int dtype, void* out, void* stream, const perm_opts* opts) {
  if (!h) return PERM_EINVAL;
  if (cudaSetDevice(h->device) != cudaSuccess) return PERM_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == PERM_U8 || dtype == PERM_I64 || dtype == PERM_CI64) {
    // exact integer batches: one warp per matrix; the range check reports like the
    // single-matrix calls (returned for host output, kept for perm_device_status else)
    if (count < 0 || (count > 0 && (!packed || !offsets || !M || !N || !out))) return PERM_EINVAL;
    if (count == 0) return PERM_OK;
    int rc = ensure_ws(h, kWsDefault, s);
    if (rc) return rc;
    const bool host_out = !on_device(out);
    int* st = host_out ? call_status_word(h) : status_word(h);
    if (host_out && cudaMemsetAsync(st, 0, sizeof(int), s) != cudaSuccess) return PERM_ECUDA;
    rc = batched_int_run(h, packed, offsets, M, N, count, dtype, out, st, s);
    if (rc || !host_out) return rc;
    int dev_status = 0;
    if (cudaMemcpyAsync(&dev_status, st, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return PERM_ECUDA;
    return dev_status;
  }
  return batched_run(h, packed, offsets, M, N, count, dtype, out, s, opts);
}

int perm_sbp(perm_handle h, const void* C, int64_t n, int64_t N, int64_t ld, int dtype, const uint64_t* occ,
             int64_t count, void* out, void* stream, const perm_opts* opts) {
  if (!h) return PERM_EINVAL;
  if (dtype == PERM_U8 || dtype == PERM_I64 || dtype == PERM_CI64) return PERM_EUNSUPPORTED;
  if (dtype != PERM_F64 && dtype != PERM_C128) return PERM_EINVAL;
  if (count < 0 || n < 1 || N < n || ld < N) return PERM_EINVAL;
  if (count > 0 && (!C || !occ || !out)) return PERM_EINVAL;
  if (n > 32 || N > 64) return PERM_ETOOBIG;
  const int chunk = (opts && opts->chunk_log2) ? opts->chunk_log2 : 14;
  if (chunk < 1 || chunk > 62) return PERM_EINVAL;
  if (count == 0) return PERM_OK;
  if (cudaSetDevice(h->device) != cudaSuccess) return PERM_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc0 = PERM_OK;
  const size_t W = dtype == PERM_C128 ? 2 : 1;
  const size_t c_bytes = 8 * W * (size_t)((n - 1) * ld + N);
  const bool hC = !on_device(C), hOcc = !on_device(occ), hOut = !on_device(out);
  const size_t need = (hC ? align_up(c_bytes) : 0) + (hOcc ? align_up(8 * (size_t)count) : 0) +
                      (hOut ? align_up(8 * W * (size_t)count) : 0);
  if ((rc0 = ensure_sws(h, need)) != PERM_OK) return rc0;
  char* base = static_cast<char*>(h->sws);
  const double* dC = static_cast<const double*>(C);
  const uint64_t* dOcc = occ;
  double* dOut = static_cast<double*>(out);
  if (hC) {
    if (cudaMemcpyAsync(base, C, c_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return PERM_ECUDA;
    dC = reinterpret_cast<const double*>(base);
    base += align_up(c_bytes);
  }
  if (hOcc) {
    if (cudaMemcpyAsync(base, occ, 8 * (size_t)count, cudaMemcpyHostToDevice, s) != cudaSuccess) return PERM_ECUDA;
    dOcc = reinterpret_cast<const uint64_t*>(base);
    base += align_up(8 * (size_t)count);
  }
  if (hOut) dOut = reinterpret_cast<double*>(base);
  if (opts && (opts->arith < 0 || opts->arith > 3)) return PERM_EINVAL;
  const bool fp64 = opts && opts->arith == PERM_ARITH_FP64;
  if ((rc0 = ensure_ws(h, kWsDefault, s)) != PERM_OK) return rc0;
  const int rc = sbp_run(h, dC, ld, (int)n, (int)N, dtype, dOcc, count, dOut, s, chunk, h->sms, fp64,
                         partials_base(h));
  if (rc == 1) return PERM_ETOOBIG;
  if (rc) return PERM_ECUDA;
  if (hOut) {
    if (cudaMemcpyAsync(out, dOut, 8 * W * (size_t)count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return PERM_ECUDA;
  }
  if (hC || hOcc || hOut) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return PERM_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

int perm_cauchy(perm_handle h, const double* x, const double* y, int64_t n, int64_t count, double* out,
                void* stream, const perm_opts* opts) {
  if (!h) return PERM_EINVAL;
  if (count < 0 || n < 1) return PERM_EINVAL;
  if (count > 0 && (!x || !y || !out)) return PERM_EINVAL;
  if (n > cauchy_max_n()) return PERM_ETOOBIG;
  if (count == 0) return PERM_OK;
  if (cudaSetDevice(h->device) != cudaSuccess) return PERM_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* err = opts ? opts->err : nullptr;
  const size_t pts = 8 * (size_t)(n * count);
  const bool hx = !on_device(x), hy = !on_device(y), hOut = !on_device(out), hErr = err && !on_device(err);
  int block = 0;
  const int grid = cauchy_grid(count, h->sms, &block);
  const size_t scratch = align_up(8 * cauchy_scratch_words((int)n) * (size_t)grid);
  const size_t state = align_up(cauchy_state_bytes(count));
  const size_t need = scratch + state + (hx ? align_up(pts) : 0) + (hy ? align_up(pts) : 0) +
                      (hOut ? align_up(8 * (size_t)count) : 0) + (hErr ? align_up(8 * (size_t)count) : 0);
  int rc = ensure_sws(h, need);
  if (rc) return rc;
  if ((rc = ensure_ws(h, kWsDefault, s)) != PERM_OK) return rc;
  char* base = static_cast<char*>(h->sws);
  uint64_t* dScratch = reinterpret_cast<uint64_t*>(base);
  base += scratch;
  void* dState = base;
  base += state;
  const double* dx = x;
  const double* dy = y;
  double* dOut = out;
  double* dErr = err;
  if (hx) {
    if (cudaMemcpyAsync(base, x, pts, cudaMemcpyHostToDevice, s) != cudaSuccess) return PERM_ECUDA;
    dx = reinterpret_cast<const double*>(base);
    base += align_up(pts);
  }
  if (hy) {
    if (cudaMemcpyAsync(base, y, pts, cudaMemcpyHostToDevice, s) != cudaSuccess) return PERM_ECUDA;
    dy = reinterpret_cast<const double*>(base);
    base += align_up(pts);
  }
  if (hOut) {
    dOut = reinterpret_cast<double*>(base);
    base += align_up(8 * (size_t)count);
  }
  if (hErr) dErr = reinterpret_cast<double*>(base);
  const bool host_result = hOut || hErr;
  int* st = host_result ? call_status_word(h) : status_word(h);
  if (host_result && cudaMemsetAsync(st, 0, sizeof(int), s) != cudaSuccess) return PERM_ECUDA;
  if (launch_cauchy(dx, dy, (int)n, count, dOut, dErr, dScratch, dState, grid, block, st, s) != cudaSuccess)
    return PERM_ECUDA;
  if (hOut && cudaMemcpyAsync(out, dOut, 8 * (size_t)count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PERM_ECUDA;
  if (hErr && cudaMemcpyAsync(err, dErr, 8 * (size_t)count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PERM_ECUDA;
  if (host_result) {
    int dev_status = 0;
    if (cudaMemcpyAsync(&dev_status, st, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PERM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PERM_ECUDA;
    if (dev_status) return dev_status;
  } else if (hx || hy) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return PERM_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

int perm_cauchy_sbp(perm_handle h, const double* x, int64_t n, const double* y, int64_t N, const uint64_t* occ,
                    int64_t count, double* out, void* stream, const perm_opts* opts) {
  if (!h) return PERM_EINVAL;
  if (count < 0 || n < 1 || N < n) return PERM_EINVAL;
  if (count > 0 && (!x || !y || !occ || !out)) return PERM_EINVAL;
  if (n > cauchy_max_n() || N > 64) return PERM_ETOOBIG;
  if (count == 0) return PERM_OK;
  if (cudaSetDevice(h->device) != cudaSuccess) return PERM_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* err = opts ? opts->err : nullptr;
  const bool hx = !on_device(x), hy = !on_device(y), hOcc = !on_device(occ), hOut = !on_device(out),
             hErr = err && !on_device(err);
  int block = 0;
  const int grid = cauchy_grid(count, h->sms, &block);
  const size_t scratch = align_up(8 * cauchy_scratch_words((int)n) * (size_t)grid);
  const size_t state = align_up(cauchy_state_bytes(count));
  const size_t pts = align_up(8 * (size_t)n * (size_t)count);
  const size_t need = scratch + state + 2 * pts + (hx ? align_up(8 * (size_t)n) : 0) +
                      (hy ? align_up(8 * (size_t)N) : 0) + (hOcc ? align_up(8 * (size_t)count) : 0) +
                      (hOut ? align_up(8 * (size_t)count) : 0) + (hErr ? align_up(8 * (size_t)count) : 0);
  int rc = ensure_sws(h, need);
  if (rc) return rc;
  if ((rc = ensure_ws(h, kWsDefault, s)) != PERM_OK) return rc;
  char* base = static_cast<char*>(h->sws);
  uint64_t* dScratch = reinterpret_cast<uint64_t*>(base);
  base += scratch;
  void* dState = base;
  base += state;
  double* xs = reinterpret_cast<double*>(base);
  base += pts;
  double* ys = reinterpret_cast<double*>(base);
  base += pts;
  const double* dx = x;
  const double* dy = y;
  const uint64_t* dOcc = occ;
  double* dOut = out;
  double* dErr = err;
  if (hx) {
    if (cudaMemcpyAsync(base, x, 8 * (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess) return PERM_ECUDA;
    dx = reinterpret_cast<const double*>(base);
    base += align_up(8 * (size_t)n);
  }
  if (hy) {
    if (cudaMemcpyAsync(base, y, 8 * (size_t)N, cudaMemcpyHostToDevice, s) != cudaSuccess) return PERM_ECUDA;
    dy = reinterpret_cast<const double*>(base);
    base += align_up(8 * (size_t)N);
  }
  if (hOcc) {
    if (cudaMemcpyAsync(base, occ, 8 * (size_t)count, cudaMemcpyHostToDevice, s) != cudaSuccess) return PERM_ECUDA;
    dOcc = reinterpret_cast<const uint64_t*>(base);
    base += align_up(8 * (size_t)count);
  }
  if (hOut) {
    dOut = reinterpret_cast<double*>(base);
    base += align_up(8 * (size_t)count);
  }
  if (hErr) dErr = reinterpret_cast<double*>(base);
  const bool host_result = hOut || hErr;
  int* st = host_result ? call_status_word(h) : status_word(h);
  if (host_result && cudaMemsetAsync(st, 0, sizeof(int), s) != cudaSuccess) return PERM_ECUDA;
  if (launch_cauchy_gather(dx, (int)n, dy, (int)N, dOcc, count, xs, ys, h->sms, s) != cudaSuccess ||
      launch_cauchy(xs, ys, (int)n, count, dOut, dErr, dScratch, dState, grid, block, st, s) != cudaSuccess)
    return PERM_ECUDA;
  if (hOut && cudaMemcpyAsync(out, dOut, 8 * (size_t)count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PERM_ECUDA;
  if (hErr && cudaMemcpyAsync(err, dErr, 8 * (size_t)count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PERM_ECUDA;
  if (host_result) {
    int dev_status = 0;
    if (cudaMemcpyAsync(&dev_status, st, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PERM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PERM_ECUDA;
    if (dev_status) return dev_status;
  } else if (hx || hy || hOcc) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return PERM_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

}  // extern "C"
