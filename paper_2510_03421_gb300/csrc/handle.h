// The library handle (opaque in include/perm.h): device workspace, the cached
// batched plan and CUDA graph, and the batched launch parameters chosen by the tuner.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <vector>

namespace perm {

// Launch parameters of the batched kernels.
struct BatchTune {
  int n_small = 10;      // matrices with n <= n_small are summed one per lane
  int item_log2 = 16;    // larger matrices are cut into sub-ranges of <= 2^item_log2 terms
  int chunk_log2 = 14;   // exact rebuild of the column sums every 2^chunk_log2 terms
  int block = 128;       // threads per block of the class kernels
  int fp64_share = 0;    // complex integer-pipe classes: part of each product on the FP64 unit
};

struct BatchCache {
  uint64_t key = 0;               // hash of sizes, pointers, dtype and tune
  cudaGraphExec_t exec = nullptr;
  bool valid = false;
};

}  // namespace perm

struct perm_handle_s {
  int device = 0;
  int sms = 0;
  void* ws = nullptr;  // device workspace of the single-matrix calls
  size_t ws_bytes = 0;
  // batched calls
  void* bws = nullptr;  // device workspace of the batched plan (and staged operands)
  size_t bws_bytes = 0;
  cudaStream_t cap = nullptr;   // stream used to capture the batched graph
  cudaStream_t side[16] = {};   // branch streams of the capture
  cudaEvent_t fork = nullptr, join[16] = {};
  perm::BatchCache cache;
  perm::BatchTune tune;
  bool tuned = false;
  uint64_t tuned_hist = 0;      // size histogram the tune was chosen for
  // staging of perm_sbp operands given in host memory
  void* sws = nullptr;
  size_t sws_bytes = 0;
  // cost model of perm_auto (host copy of the weights)
  std::vector<float> model;
  int model_in = 0, model_hid = 0, model_out = 0;
};
