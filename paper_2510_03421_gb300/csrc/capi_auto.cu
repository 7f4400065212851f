// perm_auto and its cost model: the features, the candidates and their feasibility,
// the model's inference on the host, the structure used first (empty rows, independent
// blocks of the nonzero pattern, Cauchy matrices given as dense doubles) and the
// exports perm_auto, perm_auto_features, perm_set_cost_model, perm_auto_choice.
#include "capi_internal.h"

namespace perm {
namespace {

// ---------------------------------------------------------------- learned dispatch
double log2_perm_nodes(int m, int n, double density) {
  // log2 of sum_{k=1..m} n!/(n-k)! density^k: nodes of the pruned search tree
  double total = 0.0, term = 1.0;
  for (int k = 1; k <= m; ++k) {
    term *= (double)(n - k + 1) * density;
    total += term;
  }
  return total > 1.0 ? std::log2(total) : 0.0;
}

void features(int m, int n, double density, int dtype, float* f) {
  const double mm = m, nn = n > 0 ? n : 1;
  f[0] = (float)(mm / 64.0);
  f[1] = (float)(nn / 64.0);
  f[2] = (float)(mm / nn);
  f[3] = (float)density;
  f[4] = (float)(((double)(n - 1) + std::log2(nn)) / 64.0);             // Glynn: 2^(n-1) terms of n columns
  f[5] = (float)(((double)n + std::log2(mm > 0 ? mm : 1.0)) / 64.0);    // Ryser: 2^n subsets of m rows
  f[6] = (float)(log2_perm_nodes(m, n, 1.0) / 64.0);                   // combinatoric, dense
  f[7] = (float)(log2_perm_nodes(m, n, density) / 64.0);               // combinatoric, pruned
  f[8] = dtype == PERM_F64 ? 1.f : 0.f;
  f[9] = dtype == PERM_C128 ? 1.f : 0.f;
  f[10] = (dtype == PERM_U8 || dtype == PERM_I64) ? 1.f : 0.f;
  f[11] = (float)((nn - mm) / 64.0);
}

// Which candidates exist for the dtype and stay under the work cap.
void feasible(int m, int n, double density, int dtype, uint64_t cap, bool* ok) {
  const double lcap = std::log2((double)cap);
  ok[PERM_CAND_COMBINATORIC] = log2_perm_nodes(m, n, density) <= lcap;
  ok[PERM_CAND_RYSER] = dtype == PERM_F64 && n <= 62 && (double)n <= lcap;
  ok[PERM_CAND_GLYNN] = (double)(n - 1) <= lcap && (dtype != PERM_C128 || n <= glynn_c128_max_n());
  // rectangles: the grouped walk, 2^(m-1) (n-m+1) terms
  const double lfixed = m < n ? (double)(m - 1) + std::log2((double)(n - m + 1)) : (double)(n - 1);
  ok[PERM_CAND_GLYNN_FIXED] = dtype == PERM_F64 && lfixed <= lcap;
  ok[PERM_CAND_RYSER_FP64] = ok[PERM_CAND_RYSER];
  // the FP64 configurations evaluate the padded sum of a rectangle: squares only
  ok[PERM_CAND_GLYNN_DMMA] = dtype == PERM_F64 && m == n && n <= glynn_dmma_max_n() && (double)(n - 1) <= lcap;
  ok[PERM_CAND_GLYNN_INT] = ok[PERM_CAND_GLYNN_FIXED];
  ok[PERM_CAND_GLYNN_SHORT] = (dtype == PERM_F64 && ok[PERM_CAND_GLYNN_FIXED]) ||
                              (dtype == PERM_C128 && m == n && ok[PERM_CAND_GLYNN]);
}

// Host-side inference of the installed model.
void model_predict(const perm_handle h, const float* x, float* y) {
  const int in = h->model_in, hid = h->model_hid, out = h->model_out;
  const float* W1 = h->model.data();
  const float* b1 = W1 + (size_t)in * hid;
  const float* W2 = b1 + hid;
  const float* b2 = W2 + (size_t)hid * hid;
  const float* W3 = b2 + hid;
  const float* b3 = W3 + (size_t)hid * out;
  std::vector<float> a1(hid), a2(hid);
  for (int o = 0; o < hid; ++o) {
    float z = b1[o];
    for (int i = 0; i < in; ++i) z = std::fma(x[i], W1[(size_t)i * hid + o], z);
    a1[o] = z > 0.f ? z : 0.f;
  }
  for (int o = 0; o < hid; ++o) {
    float z = b2[o];
    for (int i = 0; i < hid; ++i) z = std::fma(a1[i], W2[(size_t)i * hid + o], z);
    a2[o] = z > 0.f ? z : 0.f;
  }
  for (int o = 0; o < out; ++o) {
    float z = b3[o];
    for (int i = 0; i < hid; ++i) z = std::fma(a2[i], W3[(size_t)i * out + o], z);
    y[o] = z;
  }
}

// Fraction of nonzero entries of the operand (reads a host copy).
int density_of(const Call& c, double* d) {
  const size_t es = elem_size(c.dtype);
  const size_t count = (size_t)c.m * c.n;
  if (count == 0) {
    *d = 1.0;
    return PERM_OK;
  }
  std::vector<unsigned char> host(count * es);
  // the operand is m x n with strides (rs, cs); copy element by element rows of the
  // underlying buffer: the m x n block spans at most (m-1) rs + (n-1) cs + 1 elements
  const int64_t span = (int64_t)(c.m - 1) * c.rs + (int64_t)(c.n - 1) * c.cs + 1;
  std::vector<unsigned char> raw((size_t)span * es);
  if (cudaMemcpyAsync(raw.data(), c.dA, raw.size(), cudaMemcpyDefault, c.stream) != cudaSuccess ||
      cudaStreamSynchronize(c.stream) != cudaSuccess)
    return PERM_ECUDA;
  size_t nnz = 0;
  for (int i = 0; i < c.m; ++i)
    for (int j = 0; j < c.n; ++j) {
      const unsigned char* e = raw.data() + (size_t)(i * c.rs + j * c.cs) * es;
      bool nz = false;
      for (size_t b = 0; b < es; ++b) nz |= (e[b] != 0);
      if (c.dtype == PERM_F64 || c.dtype == PERM_C128) {  // -0.0 is zero
        double v[2] = {0.0, 0.0};
        std::memcpy(v, e, es);
        nz = (v[0] != 0.0) || (v[1] != 0.0);
      }
      nnz += nz ? 1 : 0;
    }
  *d = (double)nnz / (double)count;
  return PERM_OK;
}

// The m x n operand as a contiguous host array (elements of c.dtype).
int host_matrix(const Call& c, std::vector<unsigned char>& out) {
  const size_t es = elem_size(c.dtype);
  out.assign((size_t)c.m * c.n * es, 0);
  if (c.m == 0 || c.n == 0) return PERM_OK;
  const int64_t span = (int64_t)(c.m - 1) * c.rs + (int64_t)(c.n - 1) * c.cs + 1;
  std::vector<unsigned char> raw((size_t)span * es);
  if (cudaMemcpyAsync(raw.data(), c.dA, raw.size(), cudaMemcpyDefault, c.stream) != cudaSuccess ||
      cudaStreamSynchronize(c.stream) != cudaSuccess)
    return PERM_ECUDA;
  for (int i = 0; i < c.m; ++i)
    for (int j = 0; j < c.n; ++j)
      std::memcpy(out.data() + ((size_t)i * c.n + j) * es, raw.data() + (size_t)(i * c.rs + j * c.cs) * es, es);
  return PERM_OK;
}

bool nonzero(const unsigned char* e, int dtype) {
  if (dtype == PERM_F64 || dtype == PERM_C128) {
    double v[2] = {0.0, 0.0};
    std::memcpy(v, e, elem_size(dtype));
    return v[0] != 0.0 || v[1] != 0.0;
  }
  bool nz = false;
  for (size_t b = 0; b < elem_size(dtype); ++b) nz |= e[b] != 0;
  return nz;
}

// Structure of the nonzero pattern: the connected components of the bipartite graph
// rows <-> columns.  A term of the permanent maps every row into its own component,
// so per(A) is the product of the components' permanents, and it is zero when a row
// is empty or a component has more rows than columns.
struct Blocks {
  bool zero = false;
  std::vector<std::vector<int>> rows, cols;  // components that contain rows
};

Blocks find_blocks(const std::vector<unsigned char>& host, int m, int n, int dtype) {
  Blocks B;
  const size_t es = elem_size(dtype);
  std::vector<int> parent(m + n);
  for (int v = 0; v < m + n; ++v) parent[v] = v;
  auto find = [&](int v) {
    while (parent[v] != v) v = parent[v] = parent[parent[v]];
    return v;
  };
  for (int i = 0; i < m; ++i) {
    bool any = false;
    for (int j = 0; j < n; ++j)
      if (nonzero(host.data() + ((size_t)i * n + j) * es, dtype)) {
        any = true;
        const int a = find(i), b = find(m + j);
        if (a != b) parent[a] = b;
      }
    if (!any) {
      B.zero = true;
      return B;
    }
  }
  std::vector<int> id(m + n, -1);
  for (int i = 0; i < m; ++i) {
    const int r = find(i);
    if (id[r] < 0) {
      id[r] = (int)B.rows.size();
      B.rows.emplace_back();
      B.cols.emplace_back();
    }
    B.rows[id[r]].push_back(i);
  }
  for (int j = 0; j < n; ++j) {
    const int r = find(m + j);
    if (id[r] >= 0) B.cols[id[r]].push_back(j);
  }
  for (size_t k = 0; k < B.rows.size(); ++k)
    if (B.rows[k].size() > B.cols[k].size()) B.zero = true;
  return B;
}

// Candidate choice: the model's argmin over feasible candidates, or the built-in rule.
int choose(perm_handle h, int m, int n, double density, int dtype, uint64_t cap, int* cand, float* pred) {
  bool ok[PERM_NCAND];
  feasible(m, n, density, dtype, cap, ok);
  float y[PERM_NCAND];
  const bool have_model = !h->model.empty() && h->model_in == PERM_NFEATURES && h->model_out == PERM_NCAND;
  if (have_model) {
    float x[PERM_NFEATURES];
    features(m, n, density, dtype, x);
    model_predict(h, x, y);
  } else {
    // built-in rule without the model: the combinatoric algorithm for very small
    // matrices, Glynn (integer pipes for real input) otherwise
    for (int k = 0; k < PERM_NCAND; ++k) y[k] = 0.f;
    y[PERM_CAND_COMBINATORIC] = (n <= 6) ? -2.f : 2.f;
    y[PERM_CAND_RYSER] = 3.f;
    y[PERM_CAND_GLYNN] = dtype == PERM_F64 ? 1.f : 0.f;
    y[PERM_CAND_GLYNN_FIXED] = 0.f;
    for (int k = PERM_CAND_RYSER_FP64; k < PERM_NCAND; ++k) y[k] = 4.f;  // configurations of the above
  }
  int best = -1;
  for (int k = 0; k < PERM_NCAND; ++k) {
    if (!ok[k]) y[k] = INFINITY;
    if (ok[k] && (best < 0 || y[k] < y[best])) best = k;
  }
  if (pred)
    for (int k = 0; k < PERM_NCAND; ++k) pred[k] = y[k];
  if (best < 0) return PERM_ETOOBIG;
  *cand = best;
  return PERM_OK;
}

int run_candidate(Call& c, int cand) {
  switch (cand) {
    case PERM_CAND_COMBINATORIC: {
      Call cc = c;
      cc.o.max_terms = ~0ull >> 2;  // feasibility was judged on the pruned tree
      return combinatoric_run(cc);
    }
    case PERM_CAND_RYSER: return ryser_real(c);
    case PERM_CAND_GLYNN: {
      const uint64_t terms = 1ull << (c.n - 1);
      if (c.dtype == PERM_F64) return glynn_fp64(c, false, 0, terms);
      if (c.dtype == PERM_C128) return glynn_cplx(c, false, 0, terms);
      return glynn_integer(c, false, 0, terms);
    }
    case PERM_CAND_GLYNN_FIXED: return glynn_fixed(c, false, 0, 1ull << (c.n - 1), true);
    case PERM_CAND_RYSER_FP64: {
      Call cc = c;
      cc.o.arith = PERM_ARITH_FP64;
      return ryser_real(cc);
    }
    case PERM_CAND_GLYNN_DMMA: {
      Call cc = c;
      cc.o.arith = PERM_ARITH_FP64;
      cc.o.start = PERM_START_DMMA;
      return glynn_fp64(cc, false, 0, 1ull << (c.n - 1));
    }
    case PERM_CAND_GLYNN_INT: return glynn_fixed(c, false, 0, 1ull << (c.n - 1), false);
    case PERM_CAND_GLYNN_SHORT: {
      Call cc = c;
      if (c.dtype == PERM_C128) {
        cc.o.arith = PERM_ARITH_FP64;
        return glynn_cplx(cc, false, 0, 1ull << (c.n - 1));
      }
      cc.o.chunk_log2 = 6;
      return glynn_fixed(cc, false, 0, 1ull << (c.n - 1), true);
    }
    default: return PERM_EINVAL;
  }
}





// Cauchy structure in perm_auto: real square matrices from this order on (below it a
// sweep is as fast as the precision ladder) whose entries fit 1/(x_i - y_j) within
// kCauchyFitTol relative, all of one sign.
constexpr int kCauchyAutoMin = 24;
constexpr double kCauchyFitTol = 0x1p-48;

// Fit points to a dense real square operand; *yes on success, with the points left at
// the start of the partial-record area and *rel the relative bound on per(A) - per(C').
int cauchy_fit(const Call& c, bool* yes, double* rel) {
  *yes = false;
  if (c.dtype != PERM_F64 || c.m != c.n || c.n < kCauchyAutoMin) return PERM_OK;
  double* pts = reinterpret_cast<double*>(partials_base(c.h));
  int* flag = reinterpret_cast<int*>(pts + 128);
  if (launch_cauchy_fit(static_cast<const double*>(c.dA), c.n, c.rs, c.cs, kCauchyFitTol, pts, pts + 64, flag,
                        c.stream) != cudaSuccess)
    return PERM_ECUDA;
  int ok = 0;
  if (cudaMemcpyAsync(&ok, flag, sizeof(int), cudaMemcpyDeviceToHost, c.stream) != cudaSuccess ||
      cudaStreamSynchronize(c.stream) != cudaSuccess)
    return PERM_ECUDA;
  *yes = ok != 0;
  const double nt = c.n * kCauchyFitTol;
  *rel = nt * (1.0 + nt);  // >= (1 + tol)^n - 1 for n tol << 1
  return PERM_OK;
}

// per(A) of a fitted Cauchy operand by Borchardt's theorem (points from cauchy_fit).
int cauchy_from_fit(Call& c, double rel) {
  int block = 0;
  const int grid = cauchy_grid(1, c.h->sms, &block);
  const size_t scratch = align_up(8 * cauchy_scratch_words(c.n) * (size_t)grid);
  int rc = ensure_sws(c.h, scratch + align_up(cauchy_state_bytes(1)));
  if (rc) return rc;
  char* base = static_cast<char*>(c.h->sws);
  const double* pts = reinterpret_cast<const double*>(partials_base(c.h));
  if (launch_cauchy(pts, pts + 64, c.n, 1, static_cast<double*>(c.dOut), c.dErr, reinterpret_cast<uint64_t*>(base),
                    base + scratch, grid, block, status_word(c.h), c.stream, rel) != cudaSuccess)
    return PERM_ECUDA;
  return PERM_OK;
}

}  // namespace
}  // namespace perm

using namespace perm;

extern "C" {

int perm_auto(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, void* out, void* stream,
              const perm_opts* opts) {
  Call c;
  if (dtype == PERM_CI64) return perm_glynn(h, A, m, n, ld, dtype, out, stream, opts);  // the one algorithm
  int rc = prepare(c, h, A, m, n, ld, dtype, out, stream, opts, true);
  if (rc) return rc;
  if (c.m == 0) {
    if (launch_write_one(dtype, c.dOut, c.stream) != cudaSuccess) return PERM_ECUDA;
    if (c.dErr && cudaMemsetAsync(c.dErr, 0, sizeof(double), c.stream) != cudaSuccess) return PERM_ECUDA;
    return finish(c, out_size(dtype));
  }
  double density = 1.0;
  rc = density_of(c, &density);
  if (rc) return rc;
  const uint64_t cap = max_terms(c.o);
  if (!c.o.exhaustive && density == 1.0) {
    // a Cauchy matrix up to rounding: Borchardt's theorem in O(n^3)
    bool yes = false;
    double rel = 0.0;
    if ((rc = cauchy_fit(c, &yes, &rel)) != PERM_OK) return rc;
    if (yes) {
      if ((rc = cauchy_from_fit(c, rel)) != PERM_OK) return rc;
      return finish(c, out_size(dtype));
    }
  }
  if (!c.o.exhaustive && density < 1.0) {
    // structure of the nonzero pattern: an empty row, or independent blocks
    std::vector<unsigned char> host;
    if ((rc = host_matrix(c, host)) != PERM_OK) return rc;
    const Blocks B = find_blocks(host, c.m, c.n, dtype);
    const bool floating = dtype == PERM_F64 || dtype == PERM_C128;
    if (B.zero && floating) {
      if (launch_block_product(dtype, nullptr, 0, c.dOut, c.stream) != cudaSuccess) return PERM_ECUDA;
      if (c.dErr && cudaMemsetAsync(c.dErr, 0, sizeof(double), c.stream) != cudaSuccess) return PERM_ECUDA;
      return finish(c, out_size(dtype));
    }
    if (floating && B.rows.size() > 1) {
      // gather the blocks into the staging area (the operand is no longer needed there)
      const size_t es = elem_size(dtype);
      std::vector<unsigned char> packed;
      std::vector<size_t> at;
      for (size_t k = 0; k < B.rows.size(); ++k) {
        at.push_back(packed.size());
        for (int i : B.rows[k])
          for (int j : B.cols[k]) {
            const unsigned char* e = host.data() + ((size_t)i * c.n + j) * es;
            packed.insert(packed.end(), e, e + es);
          }
      }
      char* ws = static_cast<char*>(h->ws);
      if (cudaMemcpyAsync(ws, packed.data(), packed.size(), cudaMemcpyHostToDevice, c.stream) != cudaSuccess)
        return PERM_ECUDA;
      double* slots = reinterpret_cast<double*>(ws + kStageA + 256);  // 16 bytes per block
      for (size_t k = 0; k < B.rows.size(); ++k) {
        Call cb = c;
        cb.m = (int)B.rows[k].size();
        cb.n = (int)B.cols[k].size();
        cb.rs = cb.n;
        cb.cs = 1;
        cb.dA = ws + at[k];
        cb.dOut = slots + 2 * k;
        cb.dErr = nullptr;
        cb.hOut = nullptr;
        cb.hErr = nullptr;
        int cand = 0;
        double dk = 0.0;
        size_t nz = 0;
        for (size_t b = 0; b < (size_t)cb.m * cb.n; ++b) nz += nonzero(packed.data() + at[k] + b * es, dtype);
        dk = (double)nz / ((double)cb.m * cb.n);
        if ((rc = choose(h, cb.m, cb.n, dk, dtype, cap, &cand, nullptr)) != PERM_OK) return rc;
        if ((rc = run_candidate(cb, cand)) != PERM_OK) return rc;
      }
      if (launch_block_product(dtype, slots, (int)B.rows.size(), c.dOut, c.stream) != cudaSuccess) return PERM_ECUDA;
      if (c.dErr && launch_write_double(-1.0, c.dErr, c.stream) != cudaSuccess) return PERM_ECUDA;
      // the packed blocks are pageable host memory: the copy above completed on return
      return finish(c, out_size(dtype));
    }
  }
  int cand = 0;
  if (c.o.exhaustive) {
    // time every feasible candidate, then run the fastest last so `out` holds its result
    bool ok[PERM_NCAND];
    feasible(c.m, c.n, density, dtype, cap, ok);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PERM_ECUDA;
    float best_ms = INFINITY;
    int best = -1;
    for (int k = 0; k < PERM_NCAND; ++k) {
      if (!ok[k]) continue;
      cudaEventRecord(e0, c.stream);
      if (run_candidate(c, k) != PERM_OK) continue;
      cudaEventRecord(e1, c.stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) return PERM_ECUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best = k;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best < 0) return PERM_ETOOBIG;
    cand = best;
  } else {
    rc = choose(h, c.m, c.n, density, dtype, cap, &cand, nullptr);
    if (rc) return rc;
  }
  rc = run_candidate(c, cand);
  if (rc) return rc;
  return finish(c, out_size(dtype));
}

int perm_auto_features(int64_t m, int64_t n, double density, int dtype, float* out) {
  if (!out || m < 0 || n < 0 || m > 64 || n > 64 || !(density >= 0.0 && density <= 1.0)) return PERM_EINVAL;
  if (m > n) std::swap(m, n);
  features((int)m, (int)n, density, dtype, out);
  return PERM_OK;
}

int perm_set_cost_model(perm_handle h, const float* weights, int32_t in_dim, int32_t hidden, int32_t out_dim) {
  if (!h) return PERM_EINVAL;
  if (!weights) {
    h->model.clear();
    return PERM_OK;
  }
  int64_t count = 0;
  if (perm_mlp_size(in_dim, hidden, out_dim, &count) != PERM_OK) return PERM_EINVAL;
  if (in_dim != PERM_NFEATURES || out_dim != PERM_NCAND) return PERM_EINVAL;
  for (int64_t k = 0; k < count; ++k)
    if (!std::isfinite(weights[k])) return PERM_EINVAL;  // a damaged model: keep the current one
  h->model.assign(weights, weights + count);
  h->model_in = in_dim;
  h->model_hid = hidden;
  h->model_out = out_dim;
  return PERM_OK;
}

int perm_auto_choice(perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, const perm_opts* opts,
                     int* candidate, float* predicted) {
  if (!candidate) return PERM_EINVAL;
  Call c;
  if (dtype == PERM_CI64) {  // Gaussian integers: Glynn is the one algorithm
    double dummy[4];
    int rc = prepare(c, h, A, m, n, ld, dtype, dummy, nullptr, opts, true);
    if (rc) return rc;
    *candidate = PERM_CAND_GLYNN;
    if (predicted)
      for (int k = 0; k < PERM_NCAND; ++k) predicted[k] = INFINITY;
    return PERM_OK;
  }
  double dummy_out[2];
  int rc = prepare(c, h, A, m, n, ld, dtype, dummy_out, nullptr, opts, true);
  if (rc) return rc;
  if (c.m == 0) {
    *candidate = PERM_CAND_GLYNN;
    return PERM_OK;
  }
  double density = 1.0;
  rc = density_of(c, &density);
  if (rc) return rc;
  if (!c.o.exhaustive && density == 1.0) {
    bool yes = false;
    double rel = 0.0;
    if ((rc = cauchy_fit(c, &yes, &rel)) != PERM_OK) return rc;
    if (yes) {
      *candidate = PERM_CAND_CAUCHY;
      if (predicted)
        for (int k = 0; k < PERM_NCAND; ++k) predicted[k] = INFINITY;
      return PERM_OK;
    }
  }
  return choose(h, c.m, c.n, density, dtype, max_terms(c.o), candidate, predicted);
}

}  // extern "C"
