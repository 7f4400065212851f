// Internal interface between the C ABI files (capi.cu: validation, staging and the
// dispatch to the kernel families; capi_auto.cu: the learned dispatch and the
// structure used by perm_auto).
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/perm.h"
#include "../../include/perm_mlp.h"
#include "handle.h"
#include "internal.h"

namespace perm {

constexpr size_t kStageA = 64 * 64 * 16;  // largest matrix operand (64 x 64 complex)
constexpr size_t kStageOut = 256;         // result + error staging
constexpr size_t kWsDefault = 4u << 20;
constexpr uint64_t kDefaultMaxTerms = 1ull << 44;

// Everything one single-matrix call needs after validation.
struct Call {
  perm_handle h;
  cudaStream_t stream;
  int dtype;
  int m, n;         // after the transpose rule: m <= n
  int64_t rs, cs;   // strides of the m x n operand
  const void* dA;   // device pointer of the operand
  void* dOut;       // device destination of the result
  double* dErr;     // device destination of the error bound (or null)
  void* hOut;       // host destination (or null)
  double* hErr;     // host destination of the error bound (or null)
  perm_opts o;
};

size_t elem_size(int dtype);
size_t out_size(int dtype);
int prepare(Call& c, perm_handle h, const void* A, int64_t m, int64_t n, int64_t ld, int dtype, void* out,
            void* stream, const perm_opts* opts, bool allow_transpose);
int finish(Call& c, size_t out_bytes);
int* status_word(perm_handle h);
char* partials_base(perm_handle h);
int glynn_cplx(Call& c, bool raw, uint64_t g0, uint64_t g1);
int glynn_fixed(Call& c, bool raw, uint64_t g0, uint64_t g1, bool mixed);
int glynn_fp64(Call& c, bool raw, uint64_t g0, uint64_t g1);
int glynn_integer(Call& c, bool raw, uint64_t g0, uint64_t g1);
int ryser_real(Call& c, bool raw = false, uint64_t g0 = 0, uint64_t g1 = 0);
int combinatoric_run(Call& c);
uint64_t max_terms(const perm_opts& o);
size_t align_up(size_t x);
int ensure_sws(perm_handle h, size_t need);

}  // namespace perm
