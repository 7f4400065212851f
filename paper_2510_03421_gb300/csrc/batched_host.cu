// Host orchestration of perm_batched: size classes, the work lists, the per-handle
// CUDA graph of the class kernels, and the launch-parameter tuner.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/perm.h"
#include "handle.h"
#include "internal.h"

namespace perm {
namespace {

constexpr int kMaxBatchN = 32;  // padded orders 4..32
constexpr int kClasses = 2 * (kMaxBatchN / 4);  // lane and warp kinds x 8 orders

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

uint64_t mix(uint64_t h, uint64_t v) {
  h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
  return h;
}

// Device-side plan of one batched call: arrays laid out in the handle's batch workspace.
struct Plan {
  std::vector<int32_t> order, part_base;
  std::vector<BatchItem> items;
  struct Cls {
    int npad = 0;
    bool lane = false;
    bool fx = false;  // complex warp items on the integer pipes (batched_fx.cu)
    int first_item = 0, nitems = 0;
    double cost = 0.0;
    int grid = 1;  // blocks of the class kernel (set before capture)
  };
  std::vector<Cls> classes;
  int64_t slots = 0;
  std::vector<int32_t> fx_list;    // matrices of the integer-pipe classes
  std::vector<int64_t> fx_offset;  // their table offsets (int64 elements), 0 for the others
  int64_t fx_elems = 0;            // table size (int64 elements)
};

// The integer-pipe classes: real and complex warp items of padded order >= 16.
inline bool fx_class(bool fixed, int dtype, bool lane, int npad) {
  return fixed && (dtype == PERM_C128 || dtype == PERM_F64) && !lane && npad >= 16 && batched_fx_has_class(dtype, npad);
}

// Order of matrix b after the transpose rule.
inline int order_of(int m, int n) { return m > n ? m : n; }
inline int rows_of(int m, int n) { return m > n ? n : m; }

Plan build_plan(const std::vector<int32_t>& M, const std::vector<int32_t>& N, const BatchTune& t, bool fixed,
                int dtype, const std::vector<int32_t>* subset = nullptr) {
  Plan p;
  const int64_t count = (int64_t)M.size();
  std::vector<std::vector<int32_t>> bucket(kClasses);
  const int64_t nb = subset ? (int64_t)subset->size() : count;
  for (int64_t q = 0; q < nb; ++q) {
    const int64_t b = subset ? (*subset)[q] : q;
    const int n = order_of(M[b], N[b]);
    const int npad = n <= 4 ? 4 : ((n + 3) & ~3);
    const bool lane = n <= t.n_small && npad <= 16;
    bucket[(lane ? 0 : kClasses / 2) + npad / 4 - 1].push_back((int32_t)b);
  }
  p.part_base.assign(count, 0);
  for (int c = 0; c < kClasses; ++c) {
    if (bucket[c].empty()) continue;
    const bool lane = c < kClasses / 2;
    const int npad = 4 * (c % (kClasses / 2) + 1);
    std::vector<int32_t>& v = bucket[c];
    // longest matrices first
    std::stable_sort(v.begin(), v.end(), [&](int32_t x, int32_t y) {
      return order_of(M[x], N[x]) > order_of(M[y], N[y]);
    });
    Plan::Cls cls;
    cls.npad = npad;
    cls.lane = lane;
    cls.fx = fx_class(fixed, dtype, lane, npad);
    cls.first_item = (int)p.items.size();
    const int base = (int)p.order.size();
    p.order.insert(p.order.end(), v.begin(), v.end());
    if (lane) {
      for (size_t i = 0; i < v.size(); i += 32) {
        BatchItem it;
        it.first = base + (int)i;
        it.count = (int)std::min<size_t>(32, v.size() - i);
        it.parts = 1;
        it.pad = 0;
        p.items.push_back(it);
        const int n = order_of(M[v[i]], N[v[i]]);
        cls.cost += (double)(1ull << (n > 0 ? n - 1 : 0)) * n;
      }
    } else {
      std::vector<BatchItem> its;
      for (size_t i = 0; i < v.size(); ++i) {
        const int b = v[i];
        const int n = order_of(M[b], N[b]);
        const int m = rows_of(M[b], N[b]);
        const uint64_t terms = (m > 0) ? (1ull << (n - 1)) : 1;
        int parts = 1;
        if (terms > (1ull << t.item_log2)) parts = (int)(terms >> t.item_log2);
        p.part_base[b] = (int32_t)p.slots;
        if (parts > 1) p.slots += parts;
        for (int k = 0; k < parts; ++k) {
          BatchItem it;
          it.first = base + (int)i;
          it.count = k;
          it.parts = parts;
          it.pad = 0;
          its.push_back(it);
        }
        cls.cost += (double)terms * n / 32.0;
      }
      p.items.insert(p.items.end(), its.begin(), its.end());
    }
    cls.nitems = (int)p.items.size() - cls.first_item;
    if (cls.fx) p.fx_list.insert(p.fx_list.end(), v.begin(), v.end());
    p.classes.push_back(cls);
  }
  p.fx_offset.assign(count, 0);
  for (int32_t b : p.fx_list) {
    const int n = order_of(M[b], N[b]);
    p.fx_offset[b] = p.fx_elems;
    p.fx_elems += (dtype == PERM_C128 ? 2 : 1) * (int64_t)n * n;
  }
  // largest class first: it starts the graph's branches
  std::stable_sort(p.classes.begin(), p.classes.end(),
                   [](const Plan::Cls& x, const Plan::Cls& y) { return x.cost > y.cost; });
  return p;
}

int ensure_bws(perm_handle_s* h, size_t bytes) {
  if (h->bws_bytes >= bytes) return PERM_OK;
  if (h->bws) {
    if (cudaDeviceSynchronize() != cudaSuccess) return PERM_ECUDA;
    cudaFree(h->bws);
    h->bws = nullptr;
    h->bws_bytes = 0;
  }
  if (h->cache.valid) {
    cudaGraphExecDestroy(h->cache.exec);
    h->cache.valid = false;
  }
  size_t want = bytes + bytes / 4 + (1u << 20);
  if (cudaMalloc(&h->bws, want) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  h->bws_bytes = want;
  return PERM_OK;
}

int ensure_streams(perm_handle_s* h) {
  if (h->cap) return PERM_OK;
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) return PERM_ECUDA;
  for (int i = 0; i < 16; ++i) {
    if (cudaStreamCreateWithFlags(&h->side[i], cudaStreamNonBlocking) != cudaSuccess) return PERM_ECUDA;
    if (cudaEventCreateWithFlags(&h->join[i], cudaEventDisableTiming) != cudaSuccess) return PERM_ECUDA;
  }
  if (cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess) return PERM_ECUDA;
  return PERM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device layout of a plan inside bws (after the staged operand / result, if any).
struct Layout {
  size_t order, part_base, items, partials, done, counters, fx_list, fx_offset, fx_esum, fx_table, end;
};

Layout layout_of(const Plan& p, int64_t count, size_t start) {
  Layout L;
  L.order = align256(start);
  L.part_base = align256(L.order + 4 * count);
  L.items = align256(L.part_base + 4 * count);
  L.partials = align256(L.items + sizeof(BatchItem) * p.items.size());
  L.done = align256(L.partials + 32 * (size_t)std::max<int64_t>(p.slots, 1));
  L.counters = align256(L.done + 4 * count);
  L.fx_list = align256(L.counters + 4 * kClasses);
  L.fx_offset = align256(L.fx_list + 4 * p.fx_list.size());
  L.fx_esum = align256(L.fx_offset + (p.fx_list.empty() ? 0 : 8 * count));
  L.fx_table = align256(L.fx_esum + (p.fx_list.empty() ? 0 : 4 * count));
  L.end = align256(L.fx_table + 8 * (size_t)p.fx_elems);
  return L;
}

// Workspace for any plan of these sizes: order, part_base, done (4 B each per matrix),
// items and partial slots at the finest cut, and the integer-pipe tables.
size_t plan_bound(int64_t count, size_t max_parts, size_t fx_elems_bound) {
  return 12 * (size_t)count + 48 * (max_parts + (size_t)count) + 4 * kClasses + 16 * (size_t)count +
         8 * fx_elems_bound + 12 * 256;
}

// Enqueue the whole batched computation of plan p on stream s (class kernels on the
// side streams, joined back into s).
int enqueue(perm_handle_s* h, const Plan& p, const Layout& L, const BatchArgs& args_base, int dtype,
            const BatchTune& t, int64_t count, cudaStream_t s) {
  char* base = static_cast<char*>(h->bws);
  if (cudaMemsetAsync(base + L.done, 0, L.counters + 4 * kClasses - L.done, s) != cudaSuccess) return PERM_ECUDA;
  if (!p.fx_list.empty() &&
      launch_batched_fx_prep(args_base, dtype, reinterpret_cast<const int32_t*>(base + L.fx_list),
                             (int)p.fx_list.size(), s) != cudaSuccess)
    return PERM_ECUDA;
  if (cudaEventRecord(h->fork, s) != cudaSuccess) return PERM_ECUDA;
  int k = 0;
  for (const Plan::Cls& c : p.classes) {
    cudaStream_t br = h->side[k % 16];
    if (cudaStreamWaitEvent(br, h->fork, 0) != cudaSuccess) return PERM_ECUDA;
    ClassWork cw;
    cw.items = reinterpret_cast<const BatchItem*>(base + L.items) + c.first_item;
    cw.nitems = c.nitems;
    cw.counter = reinterpret_cast<int*>(base + L.counters) + k;
    LaunchCfg lc;
    lc.block = t.block;
    lc.grid = c.grid;
    lc.stream = br;
    const cudaError_t e = c.fx ? launch_batched_fx(args_base, cw, dtype, c.npad, lc, t.fp64_share != 0)
                               : launch_batched_class(args_base, cw, dtype, c.npad, c.lane, lc);
    if (e != cudaSuccess) return PERM_ECUDA;
    if (cudaEventRecord(h->join[k % 16], br) != cudaSuccess) return PERM_ECUDA;
    if (cudaStreamWaitEvent(s, h->join[k % 16], 0) != cudaSuccess) return PERM_ECUDA;
    ++k;
  }
  (void)count;
  return PERM_OK;
}

int upload_plan(perm_handle_s* h, const Plan& p, const Layout& L, int64_t count, cudaStream_t s) {
  char* base = static_cast<char*>(h->bws);
  if (count && cudaMemcpyAsync(base + L.order, p.order.data(), 4 * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return PERM_ECUDA;
  if (count && cudaMemcpyAsync(base + L.part_base, p.part_base.data(), 4 * count, cudaMemcpyHostToDevice, s) !=
                   cudaSuccess)
    return PERM_ECUDA;
  if (!p.items.empty() && cudaMemcpyAsync(base + L.items, p.items.data(), sizeof(BatchItem) * p.items.size(),
                                          cudaMemcpyHostToDevice, s) != cudaSuccess)
    return PERM_ECUDA;
  if (!p.fx_list.empty()) {
    if (cudaMemcpyAsync(base + L.fx_list, p.fx_list.data(), 4 * p.fx_list.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(base + L.fx_offset, p.fx_offset.data(), 8 * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return PERM_ECUDA;
  }
  // the host vectors are pageable: the copies above are complete when they return
  return PERM_OK;
}

void set_fx(BatchArgs& a, perm_handle_s* h, const Layout& L) {
  char* base = static_cast<char*>(h->bws);
  a.fx_table = reinterpret_cast<long long*>(base + L.fx_table);
  a.fx_offset = reinterpret_cast<const int64_t*>(base + L.fx_offset);
  a.fx_esum = reinterpret_cast<int*>(base + L.fx_esum);
}

BatchArgs args_for(perm_handle_s* h, const Layout& L, const double* dpacked, const int64_t* doff, const int32_t* dM,
                   const int32_t* dN, double* dout, int chunk_log2) {
  char* base = static_cast<char*>(h->bws);
  BatchArgs a;
  a.packed = dpacked;
  a.offsets = doff;
  a.M = dM;
  a.N = dN;
  a.order = reinterpret_cast<const int32_t*>(base + L.order);
  a.part_base = reinterpret_cast<const int32_t*>(base + L.part_base);
  a.partials = reinterpret_cast<double*>(base + L.partials);
  a.done = reinterpret_cast<int*>(base + L.done);
  a.out = dout;
  a.chunk_log2 = chunk_log2;
  set_fx(a, h, L);
  return a;
}

// Launch-parameter tuner: time the class kernels on an evenly spaced sample of the
// batch (at most 4096 matrices) for each candidate setting and keep the fastest.
int tune_batch(perm_handle_s* h, const std::vector<int32_t>& hM, const std::vector<int32_t>& hN, int dtype,
               bool fixed, const BatchArgs& base_args, size_t start, cudaStream_t s, BatchTune* best) {
  const int64_t count = (int64_t)hM.size();
  std::vector<int32_t> sample;
  const int64_t stride = count > 4096 ? count / 4096 : 1;
  for (int64_t b = 0; b < count; b += stride) sample.push_back((int32_t)b);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PERM_ECUDA;
  float best_ms = INFINITY;
  const int smalls[] = {6, 8, 10, 12};
  const int items[] = {14, 16, 18};
  const int blocks[] = {64, 128};
  const int shares = fixed ? 2 : 1;  // the FP64 share only exists for the integer-pipe classes
  int rc = PERM_OK;
  for (int ns : smalls)
    for (int il : items)
      for (int bl : blocks)
        for (int sh = 0; sh < shares; ++sh) {
          BatchTune t = *best;
          t.n_small = ns;
          t.item_log2 = il;
          t.block = bl;
          t.fp64_share = sh;
          Plan p = build_plan(hM, hN, t, fixed, dtype, &sample);
          for (Plan::Cls& c : p.classes) {
            const int bps = c.fx ? batched_fx_blocks_per_sm(dtype, c.npad, t.block, t.fp64_share != 0)
                                 : batched_blocks_per_sm(dtype, c.npad, c.lane, t.block);
            int grid = h->sms * (bps > 0 ? bps : 1);
            const int need = (c.nitems + t.block / 32 - 1) / (t.block / 32);
            c.grid = need < grid ? (need > 0 ? need : 1) : grid;
          }
          Layout L = layout_of(p, count, start);
          if ((rc = ensure_bws(h, L.end)) != PERM_OK) goto done;
          if ((rc = upload_plan(h, p, L, count, s)) != PERM_OK) goto done;
          {
            BatchArgs a = base_args;
            char* base = static_cast<char*>(h->bws);
            a.order = reinterpret_cast<const int32_t*>(base + L.order);
            a.part_base = reinterpret_cast<const int32_t*>(base + L.part_base);
            a.partials = reinterpret_cast<double*>(base + L.partials);
            a.done = reinterpret_cast<int*>(base + L.done);
            a.chunk_log2 = t.chunk_log2;
            set_fx(a, h, L);
            if ((rc = enqueue(h, p, L, a, dtype, t, count, s)) != PERM_OK) goto done;  // warm-up
            cudaEventRecord(e0, s);
            if ((rc = enqueue(h, p, L, a, dtype, t, count, s)) != PERM_OK) goto done;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
              rc = PERM_ECUDA;
              goto done;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
              best_ms = ms;
              *best = t;
            }
          }
        }
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace

void batched_release(perm_handle_s* h) {
  if (h->cache.valid) cudaGraphExecDestroy(h->cache.exec);
  h->cache.valid = false;
  if (h->bws) cudaFree(h->bws);
  h->bws = nullptr;
  if (h->cap) {
    cudaStreamDestroy(h->cap);
    for (int i = 0; i < 16; ++i) {
      cudaStreamDestroy(h->side[i]);
      cudaEventDestroy(h->join[i]);
    }
    cudaEventDestroy(h->fork);
    h->cap = nullptr;
  }
}

int batched_run(perm_handle_s* h, const void* packed, const int64_t* offsets, const int32_t* M, const int32_t* N,
                int64_t count, int dtype, void* out, cudaStream_t s, const void* opts_v) {
  const perm_opts* opts = static_cast<const perm_opts*>(opts_v);
  if (count < 0 || (count > 0 && (!packed || !offsets || !M || !N || !out))) return PERM_EINVAL;
  if (dtype != PERM_F64 && dtype != PERM_C128) return PERM_EINVAL;
  if (count == 0) return PERM_OK;
  if (count > (1ll << 30)) return PERM_ETOOBIG;
  const int W = dtype == PERM_C128 ? 2 : 1;
  int rc = ensure_streams(h);
  if (rc) return rc;
  // sizes on the host
  std::vector<int64_t> hoff(count);
  std::vector<int32_t> hM(count), hN(count);
  const bool dev_off = on_device(offsets), dev_M = on_device(M), dev_N = on_device(N);
  if (dev_off || dev_M || dev_N) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return PERM_ECUDA;
  }
  if (cudaMemcpy(hoff.data(), offsets, 8 * count, dev_off ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost) !=
          cudaSuccess ||
      cudaMemcpy(hM.data(), M, 4 * count, dev_M ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost) != cudaSuccess ||
      cudaMemcpy(hN.data(), N, 4 * count, dev_N ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost) != cudaSuccess)
    return PERM_ECUDA;
  int64_t elems = 0;
  uint64_t hist = 0;
  size_t max_parts = 0;  // sub-ranges at the finest cut the tuner tries (2^14 terms)
  size_t fx_elems = 0;   // integer-pipe tables if every matrix took them
  for (int64_t b = 0; b < count; ++b) {
    if (hM[b] < 0 || hN[b] < 0 || hoff[b] < 0) return PERM_EINVAL;
    const int n = order_of(hM[b], hN[b]);
    if (n > kMaxBatchN) return PERM_ETOOBIG;
    elems = std::max<int64_t>(elems, hoff[b] + (int64_t)hM[b] * hN[b]);
    max_parts += (n > 15) ? ((size_t)1 << (n - 15)) : 1;
    fx_elems += 2 * (size_t)n * n;
  }
  for (int64_t b = 0; b < count; ++b) hist = mix(hist, (uint64_t)hM[b] * 131 + hN[b]);

  BatchTune t = h->tuned && h->tuned_hist == hist ? h->tune : BatchTune();
  if (opts && opts->chunk_log2) t.chunk_log2 = opts->chunk_log2;
  if (opts && opts->block) {
    if (opts->block % 32 || opts->block > 128) return PERM_EINVAL;
    t.block = opts->block;
  }

  // staged operands (host packed / out / sizes) live at the start of the batch workspace
  const bool host_packed = !on_device(packed), host_out = !on_device(out);
  const bool host_sizes = !dev_off || !dev_M || !dev_N;
  size_t start = 0, packed_at = 0, out_at = 0, sizes_at = 0;
  if (host_packed) {
    packed_at = start;
    start = align256(start + 8 * W * (size_t)elems);
  }
  if (host_out) {
    out_at = start;
    start = align256(start + 8 * W * (size_t)count);
  }
  if (host_sizes) {
    sizes_at = start;
    start = align256(start + 16 * (size_t)count);
  }
  // room for any plan: order, part_base, done (4 B each per matrix), items and partial slots
  // warp items of order >= 13 run on the integer pipes unless FP64 arithmetic is asked for
  const bool fixed = !(opts && opts->arith == PERM_ARITH_FP64);
  rc = ensure_bws(h, start + plan_bound(count, max_parts, fixed ? fx_elems : 0));
  if (rc) return rc;
  char* base = static_cast<char*>(h->bws);
  const double* dpacked = static_cast<const double*>(packed);
  double* dout = static_cast<double*>(out);
  const int64_t* doff = offsets;
  const int32_t* dM = M;
  const int32_t* dN = N;
  if (host_packed) {
    if (cudaMemcpyAsync(base + packed_at, packed, 8 * W * (size_t)elems, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return PERM_ECUDA;
    dpacked = reinterpret_cast<const double*>(base + packed_at);
  }
  if (host_out) dout = reinterpret_cast<double*>(base + out_at);
  if (host_sizes) {
    char* sz = base + sizes_at;
    if (cudaMemcpyAsync(sz, hoff.data(), 8 * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(sz + 8 * count, hM.data(), 4 * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(sz + 12 * count, hN.data(), 4 * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return PERM_ECUDA;
    doff = reinterpret_cast<const int64_t*>(sz);
    dM = reinterpret_cast<const int32_t*>(sz + 8 * count);
    dN = reinterpret_cast<const int32_t*>(sz + 12 * count);
  }

  if (opts && opts->exhaustive && !(h->tuned && h->tuned_hist == hist)) {
    // tune on a sample of this batch; kept for later batches with the same sizes
    if (h->cache.valid) {
      cudaGraphExecDestroy(h->cache.exec);
      h->cache.valid = false;
    }
    BatchArgs probe;
    probe.packed = dpacked;
    probe.offsets = doff;
    probe.M = dM;
    probe.N = dN;
    probe.out = dout;
    BatchTune best = t;
    rc = tune_batch(h, hM, hN, dtype, fixed, probe, start, s, &best);
    if (rc) return rc;
    if (opts->chunk_log2) best.chunk_log2 = opts->chunk_log2;
    h->tune = best;
    h->tuned = true;
    h->tuned_hist = hist;
    t = best;
  }

  // an explicit arithmetic overrides the tuner's FP64 share: MIXED takes it, FIXED not
  if (opts && opts->arith == PERM_ARITH_MIXED) t.fp64_share = 1;
  if (opts && opts->arith == PERM_ARITH_FIXED) t.fp64_share = 0;
  Plan p = build_plan(hM, hN, t, fixed, dtype);
  for (Plan::Cls& c : p.classes) {  // grid sizes (queried outside any stream capture)
    const int bps = c.fx ? batched_fx_blocks_per_sm(dtype, c.npad, t.block, t.fp64_share != 0)
                         : batched_blocks_per_sm(dtype, c.npad, c.lane, t.block);
    const int warps_per_block = t.block / 32;
    int grid = h->sms * (bps > 0 ? bps : 1);
    const int need = (c.nitems + warps_per_block - 1) / warps_per_block;
    if (need < grid) grid = need > 0 ? need : 1;
    c.grid = grid;
  }
  Layout L = layout_of(p, count, start);
  if (L.end > h->bws_bytes) return PERM_ENOMEM;  // cannot happen: plan_bound covers every plan

  uint64_t key = mix(hist, (uint64_t)count);
  key = mix(key, (uint64_t)dtype);
  key = mix(key, (uint64_t)(uintptr_t)dpacked);
  key = mix(key, (uint64_t)(uintptr_t)dout);
  key = mix(key, (uint64_t)(uintptr_t)doff);
  key = mix(key, (uint64_t)(uintptr_t)dM);
  key = mix(key, (uint64_t)(uintptr_t)dN);
  key = mix(key, (uint64_t)t.n_small * 1000003ull + t.item_log2 * 1009 + t.chunk_log2 * 31 + t.block);
  key = mix(key, (uint64_t)t.fp64_share);
  key = mix(key, (uint64_t)(uintptr_t)h->bws);
  key = mix(key, fixed ? 1u : 0u);

  BatchArgs args = args_for(h, L, dpacked, doff, dM, dN, dout, t.chunk_log2);
  if (!(h->cache.valid && h->cache.key == key)) {
    if (h->cache.valid) {
      cudaGraphExecDestroy(h->cache.exec);
      h->cache.valid = false;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return PERM_ECUDA;
    rc = upload_plan(h, p, L, count, h->cap);
    if (rc) return rc;
    if (cudaStreamSynchronize(h->cap) != cudaSuccess) return PERM_ECUDA;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PERM_ECUDA;
    rc = enqueue(h, p, L, args, dtype, t, count, h->cap);
    cudaError_t ce = cudaStreamEndCapture(h->cap, &graph);
    if (rc || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc ? rc : PERM_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return PERM_ECUDA;
    h->cache.exec = exec;
    h->cache.key = key;
    h->cache.valid = true;
  }
  if (cudaGraphLaunch(h->cache.exec, s) != cudaSuccess) return PERM_ECUDA;
  if (host_out) {
    if (cudaMemcpyAsync(out, dout, 8 * W * (size_t)count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return PERM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PERM_ECUDA;
  }
  return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

int batched_int_run(perm_handle_s* h, const void* packed, const int64_t* offsets, const int32_t* M, const int32_t* N,
                    int64_t count, int dtype, void* out, int* status, cudaStream_t s) {
  if (count < 0 || (count > 0 && (!packed || !offsets || !M || !N || !out))) return PERM_EINVAL;
  if (count == 0) return PERM_OK;
  if (count > (1ll << 30)) return PERM_ETOOBIG;
  std::vector<int64_t> hoff(count);
  std::vector<int32_t> hM(count), hN(count);
  const bool dev_off = on_device(offsets), dev_M = on_device(M), dev_N = on_device(N);
  if (dev_off || dev_M || dev_N) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return PERM_ECUDA;
  }
  if (cudaMemcpy(hoff.data(), offsets, 8 * count, dev_off ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost) !=
          cudaSuccess ||
      cudaMemcpy(hM.data(), M, 4 * count, dev_M ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost) != cudaSuccess ||
      cudaMemcpy(hN.data(), N, 4 * count, dev_N ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost) != cudaSuccess)
    return PERM_ECUDA;
  // matrices by padded order: lists of indices, one launch per class
  const int pads[4] = {8, 16, 24, 32};
  std::vector<int32_t> lists[4];
  int64_t elems = 0;
  for (int64_t b = 0; b < count; ++b) {
    if (hM[b] < 0 || hN[b] < 0 || hoff[b] < 0) return PERM_EINVAL;
    const int n = order_of(hM[b], hN[b]);
    if (n > batched_int_max_n()) return PERM_ETOOBIG;
    elems = std::max<int64_t>(elems, hoff[b] + (int64_t)hM[b] * hN[b]);
    const int np = batched_int_class(n);
    for (int c = 0; c < 4; ++c)
      if (pads[c] == np) lists[c].push_back((int32_t)b);
  }
  const size_t es = dtype == PERM_U8 ? 1 : dtype == PERM_CI64 ? 16 : 8;
  const size_t os = dtype == PERM_CI64 ? 32 : 16;  // bytes of one result
  const bool host_packed = !on_device(packed), host_out = !on_device(out);
  const bool host_sizes = !dev_off || !dev_M || !dev_N;
  size_t at = 0, packed_at = 0, out_at = 0, sizes_at = 0, list_at = 0;
  if (host_packed) {
    packed_at = at;
    at = align256(at + es * (size_t)elems);
  }
  if (host_out) {
    out_at = at;
    at = align256(at + os * (size_t)count);
  }
  if (host_sizes) {
    sizes_at = at;
    at = align256(at + 16 * (size_t)count);
  }
  list_at = at;
  at = align256(at + 4 * (size_t)count);
  int rc = ensure_bws(h, at);
  if (rc) return rc;
  // the batch workspace is about to hold these operands instead of a float plan
  if (h->cache.valid) {
    cudaGraphExecDestroy(h->cache.exec);
    h->cache.valid = false;
  }
  char* base = static_cast<char*>(h->bws);
  const void* dpacked = packed;
  unsigned long long* dout = static_cast<unsigned long long*>(out);
  const int64_t* doff = offsets;
  const int32_t* dM = M;
  const int32_t* dN = N;
  if (host_packed) {
    if (cudaMemcpyAsync(base + packed_at, packed, es * (size_t)elems, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return PERM_ECUDA;
    dpacked = base + packed_at;
  }
  if (host_out) dout = reinterpret_cast<unsigned long long*>(base + out_at);
  if (host_sizes) {
    char* sz = base + sizes_at;
    if (cudaMemcpyAsync(sz, hoff.data(), 8 * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(sz + 8 * count, hM.data(), 4 * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(sz + 12 * count, hN.data(), 4 * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return PERM_ECUDA;
    doff = reinterpret_cast<const int64_t*>(sz);
    dM = reinterpret_cast<const int32_t*>(sz + 8 * count);
    dN = reinterpret_cast<const int32_t*>(sz + 12 * count);
  }
  std::vector<int32_t> all;
  all.reserve(count);
  size_t first[4];
  for (int c = 0; c < 4; ++c) {
    first[c] = all.size();
    all.insert(all.end(), lists[c].begin(), lists[c].end());
  }
  int32_t* dlist = reinterpret_cast<int32_t*>(base + list_at);
  if (cudaMemcpyAsync(dlist, all.data(), 4 * all.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return PERM_ECUDA;
  for (int c = 0; c < 4; ++c) {
    if (lists[c].empty()) continue;
    if (launch_batched_int(dpacked, doff, dM, dN, dlist + first[c], (int)lists[c].size(), dtype, pads[c], dout,
                           status, h->sms, s) != cudaSuccess)
      return PERM_ECUDA;
  }
  if (host_out && cudaMemcpyAsync(out, dout, os * (size_t)count, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PERM_ECUDA;
  // pageable host vectors above were copied asynchronously: finish before they go away
  if (cudaStreamSynchronize(s) != cudaSuccess) return PERM_ECUDA;
  return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

}  // namespace perm
