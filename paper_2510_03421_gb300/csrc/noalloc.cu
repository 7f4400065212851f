// perm_glynn_noalloc: the real FP64 Glynn sweep for callers that cannot allocate
// device memory.  Some hosts of this library own all device memory themselves: a
// runtime that carves every buffer out of a pool reserved at start-up, a plugin
// whose host forbids cudaMalloc, or code running where an allocation would
// synchronise or fail.  Those callers still need the sweep's scratch space (one
// partial-sum record per block), so this entry point takes it from a fixed array
// in device memory that the library declares at file scope.  The array lives as
// long as the library is loaded, on every GPU that loads it.
//
// Host code cannot use the array's name as a device address (in host code it names
// a host-side stand-in), so the address is looked up with cudaGetSymbolAddress once
// per device, with that device current, on the first call on that device, and kept
// for the life of the process: a cudaDeviceReset discards the array with the
// context, so after one this entry point must not be called again in that process.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/perm.h"
#include "internal.h"

namespace perm {
namespace {

// Scratch for the per-block records of the sweep: at most kNoAllocMaxBlocks blocks.
constexpr int kNoAllocMaxBlocks = 2048;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks * kRealRecord];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (looked up once).
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PERM_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return PERM_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return PERM_OK;
}

// Device or managed memory of device `dev` (a kernel on `dev` may read it); host memory
// and another GPU's memory are refused before anything is launched.
bool on_this_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace
}  // namespace perm

using namespace perm;

extern "C" int perm_glynn_noalloc(const void* A, int64_t m, int64_t n, int64_t ld, void* out, void* stream,
                                  int32_t grid) {
  if (!out || m < 0 || n < 0 || ld < n || (m > 0 && n > 0 && !A)) return PERM_EINVAL;
  if (m > 64 || n > 64) return PERM_ETOOBIG;
  if (grid < 0) return PERM_EINVAL;
  if (grid > kNoAllocMaxBlocks) return PERM_ETOOBIG;
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return PERM_ECUDA;
  if (!on_this_device(out, cur) || (m > 0 && n > 0 && !on_this_device(A, cur))) return PERM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;

  SweepArgs a;
  a.A = A;
  if (m > n) {  // per(A) = per(A^T)
    a.m = (int)n;
    a.n = (int)m;
    a.rs = 1;
    a.cs = ld;
  } else {
    a.m = (int)m;
    a.n = (int)n;
    a.rs = ld;
    a.cs = 1;
  }
  if (a.m == 0) return launch_write_one(PERM_F64, out, s) == cudaSuccess ? PERM_OK : PERM_ECUDA;
  const uint64_t terms = 1ull << (a.n - 1);
  if (terms > (1ull << 44)) return PERM_ETOOBIG;
  a.g_begin = 0;
  a.g_end = terms;
  a.chunk_log2 = 14;
  a.start_mode = PERM_START_SCALAR;
  a.partials = scratch;

  LaunchCfg lc;
  lc.block = 256;
  lc.stream = s;
  if (grid == 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return PERM_ECUDA;
    const int bps = glynn_f64_blocks_per_sm(a.n, lc.block, false);
    if (bps <= 0) return PERM_ECUDA;  // the kernel's shared-memory limit could not be raised
    grid = sms * bps;
    const uint64_t want = (terms + 256u * 16u - 1) / (256u * 16u);
    if (want < (uint64_t)grid) grid = (int)want;
    if (grid > kNoAllocMaxBlocks) grid = kNoAllocMaxBlocks;
  }
  lc.grid = grid;
  // Each block writes its own record before the final reduction reads it, so no
  // part of the scratch has to start at zero.
  if (launch_glynn_f64(a, lc, false) != cudaSuccess) return PERM_ECUDA;
  if (launch_finish_real(scratch, lc.grid, a.n - 1, a.n - a.m, 0.0, static_cast<double*>(out), nullptr, false, s) !=
      cudaSuccess)
    return PERM_ECUDA;
  return PERM_OK;
}
