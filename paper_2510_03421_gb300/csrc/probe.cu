// Issue-rate probes (include/perm_probe.h): dependent chains with eight independent
// streams per thread, enough resident warps to saturate the pipe, timed with events.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/perm.h"
#include "../../include/perm_probe.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 4;

template <int KIND>
__global__ void __launch_bounds__(256) probe_kernel(int iters, double a, double b, unsigned* sink) {
  double acc = 0.0;
  if (KIND == PERM_PROBE_DFMA) {
    double x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0 + threadIdx.x * 1e-7 + i * 1e-5;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int r = 0; r < kUnroll; ++r)
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = __fma_rn(x[i], a, b);
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc += x[i];
  } else if (KIND == PERM_PROBE_FFMA) {
    float x[kChains];
    const float fa = (float)a, fb = (float)b;
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = 1.0f + threadIdx.x * 1e-7f + i * 1e-5f;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int r = 0; r < kUnroll; ++r)
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = __fmaf_rn(x[i], fa, fb);
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc += x[i];
  } else if (KIND == PERM_PROBE_IMAD || KIND == PERM_PROBE_IADD) {
    unsigned x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = threadIdx.x * 2654435761u + i;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int r = 0; r < kUnroll; ++r)
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
          // the neighbouring chain keeps the compiler from folding the sequence
          if (KIND == PERM_PROBE_IMAD) x[i] = x[i] * x[(i + 1) % kChains] + 12345u;
          else x[i] = x[i] + x[(i + 1) % kChains];
        }
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc += x[i];
  } else if (KIND == PERM_PROBE_DMMA) {
    double c[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i][0] = c[i][1] = 0.0;
    const double av = a * (1.0 + threadIdx.x * 1e-9), bv = b;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int r = 0; r < kUnroll; ++r)
#pragma unroll
        for (int i = 0; i < 4; ++i)
          asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                       : "+d"(c[i][0]), "+d"(c[i][1])
                       : "d"(av), "d"(bv));
#pragma unroll
    for (int i = 0; i < 4; ++i) acc += c[i][0] + c[i][1];
  }
  if (acc == 1234.5678) sink[0] = 1u;  // never true in practice; keeps the chains live
}

template <int KIND>
cudaError_t time_kernel(int blocks, int iters, cudaStream_t s, unsigned* sink, float* best_ms) {
  cudaEvent_t e0, e1;
  cudaError_t err = cudaEventCreate(&e0);
  if (err != cudaSuccess) return err;
  err = cudaEventCreate(&e1);
  if (err != cudaSuccess) {
    cudaEventDestroy(e0);
    return err;
  }
  probe_kernel<KIND><<<blocks, 256, 0, s>>>(iters / 8 + 1, 1.0000001, 1e-9, sink);  // warm-up
  *best_ms = 1e30f;
  for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
    cudaEventRecord(e0, s);
    probe_kernel<KIND><<<blocks, 256, 0, s>>>(iters, 1.0000001, 1e-9, sink);
    cudaEventRecord(e1, s);
    err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && ms < *best_ms) *best_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return err;
}

}  // namespace

extern "C" int perm_probe_rate(int device, int kind, void* stream, double* rate) {
  if (!rate || kind < 0 || kind > 4) return PERM_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return PERM_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PERM_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(unsigned)) != cudaSuccess) return PERM_ECUDA;
  const int blocks = sms * 4;
  // iterations for roughly 50 ms at the rates of a GB300
  int iters = 0;
  switch (kind) {
    case PERM_PROBE_DFMA: iters = 6000; break;
    case PERM_PROBE_DMMA: iters = 1500; break;
    case PERM_PROBE_IMAD: iters = 160000; break;
    case PERM_PROBE_IADD: iters = 320000; break;
    case PERM_PROBE_FFMA: iters = 320000; break;
  }
  float ms = 0.f;
  cudaError_t err = cudaSuccess;
  switch (kind) {
    case PERM_PROBE_DFMA: err = time_kernel<PERM_PROBE_DFMA>(blocks, iters, s, sink, &ms); break;
    case PERM_PROBE_DMMA: err = time_kernel<PERM_PROBE_DMMA>(blocks, iters, s, sink, &ms); break;
    case PERM_PROBE_IMAD: err = time_kernel<PERM_PROBE_IMAD>(blocks, iters, s, sink, &ms); break;
    case PERM_PROBE_IADD: err = time_kernel<PERM_PROBE_IADD>(blocks, iters, s, sink, &ms); break;
    case PERM_PROBE_FFMA: err = time_kernel<PERM_PROBE_FFMA>(blocks, iters, s, sink, &ms); break;
  }
  cudaFree(sink);
  if (err != cudaSuccess) return PERM_ECUDA;
  const double threads = (double)blocks * 256.0;
  const double per_thread = (double)iters * kUnroll * kChains;
  double ops = threads * per_thread;
  if (kind == PERM_PROBE_DMMA) ops = (double)iters * kUnroll * 4.0 * (threads / 32.0) * (8.0 * 8.0 * 4.0 * 2.0);
  *rate = ops / (ms * 1e-3);
  return PERM_OK;
}
