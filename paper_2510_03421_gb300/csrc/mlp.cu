// The cost model of perm_auto: a three-layer perceptron in FP32,
//     h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3,
// trained on the GPU by these kernels (forward, backward, Adam) with a masked mean
// squared error on log2 run times.  The layers are tiny (at most 64 wide), so each
// kernel assigns one thread per output element and loops over the inner dimension
// in a fixed order: results are deterministic.  Not a tensor-core workload.
//
// Flat weight layout (floats): W1 [in x hid], b1 [hid], W2 [hid x hid], b2 [hid],
// W3 [hid x out], b3 [out].
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/perm.h"
#include "../../include/perm_mlp.h"

namespace perm {
namespace {

struct Dims {
  int in, hid, out;
  __host__ __device__ size_t w1() const { return 0; }
  __host__ __device__ size_t b1() const { return (size_t)in * hid; }
  __host__ __device__ size_t w2() const { return b1() + hid; }
  __host__ __device__ size_t b2() const { return w2() + (size_t)hid * hid; }
  __host__ __device__ size_t w3() const { return b2() + hid; }
  __host__ __device__ size_t b3() const { return w3() + (size_t)hid * out; }
  __host__ __device__ size_t total() const { return b3() + out; }
};

// Z = X W + b; A = relu(Z) (or Z for the output layer)
__global__ void linear_fwd(const float* __restrict__ X, int64_t rows, int din, const float* __restrict__ W,
                           const float* __restrict__ b, int dout, float* __restrict__ Z, float* __restrict__ A,
                           int relu) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * dout) return;
  const int64_t r = idx / dout;
  const int o = (int)(idx - r * dout);
  float z = b[o];
  for (int i = 0; i < din; ++i) z = __fmaf_rn(X[r * din + i], W[(size_t)i * dout + o], z);
  if (Z) Z[idx] = z;
  A[idx] = (relu && z < 0.f) ? 0.f : z;
}

// dY = 2 mask (Y - T) / msum, and per-block partial sums of mask (Y - T)^2.
__global__ void mse_grad(const float* __restrict__ Y, const float* __restrict__ T, const float* __restrict__ mask,
                         int64_t n, float inv_msum, float* __restrict__ dY, float* __restrict__ partial) {
  __shared__ float s[256];
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (idx < n) {
    const float d = Y[idx] - T[idx];
    const float mk = mask[idx];
    dY[idx] = 2.f * mk * d * inv_msum;
    l = mk * d * d;
  }
  s[threadIdx.x] = l;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void sum_partials(const float* __restrict__ partial, int n, float scale, float* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float t = 0.f;
  for (int i = 0; i < n; ++i) t += partial[i];
  out[0] = t * scale;
}

// dX = (dZ W^T) * relu'(Zprev)
__global__ void linear_bwd_input(const float* __restrict__ dZ, int64_t rows, int dout, const float* __restrict__ W,
                                 int din, const float* __restrict__ Zprev, float* __restrict__ dX) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * din) return;
  const int64_t r = idx / din;
  const int i = (int)(idx - r * din);
  float g = 0.f;
  for (int o = 0; o < dout; ++o) g = __fmaf_rn(dZ[r * dout + o], W[(size_t)i * dout + o], g);
  dX[idx] = (Zprev[idx] > 0.f) ? g : 0.f;
}

// dW = X^T dZ, db = sum over rows of dZ (one thread per weight, rows in order)
__global__ void linear_bwd_weight(const float* __restrict__ X, const float* __restrict__ dZ, int64_t rows, int din,
                                  int dout, float* __restrict__ dW, float* __restrict__ db) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < din * dout) {
    const int i = idx / dout, o = idx - i * dout;
    float g = 0.f;
    for (int64_t r = 0; r < rows; ++r) g = __fmaf_rn(X[r * din + i], dZ[r * dout + o], g);
    dW[idx] = g;
  } else if (idx < din * dout + dout) {
    const int o = idx - din * dout;
    float g = 0.f;
    for (int64_t r = 0; r < rows; ++r) g += dZ[r * dout + o];
    db[o] = g;
  }
}

__global__ void adam_step(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                          float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                          float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Counter-based uniform in [-1, 1) from (seed, index): splitmix64.
__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + 0x9e3779b97f4a7c15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (float)((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.f - 1.f;
}

// He-style initialisation: weights uniform in +-sqrt(6 / fan_in), biases zero.
__global__ void init_weights(float* __restrict__ w, int in, int hid, int out, uint64_t seed) {
  const Dims d{in, hid, out};
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)d.total()) return;
  float scale = 0.f;
  if (i < (int64_t)d.b1()) scale = sqrtf(6.f / in);
  else if (i >= (int64_t)d.w2() && i < (int64_t)d.b2()) scale = sqrtf(6.f / hid);
  else if (i >= (int64_t)d.w3() && i < (int64_t)d.b3()) scale = sqrtf(3.f / hid);
  w[i] = scale * hash_uniform(seed, (uint64_t)i);
}

inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

// Scratch of one forward/backward pass over `rows` rows.
struct Pass {
  float *z1, *a1, *z2, *a2, *y, *dy, *d2, *d1, *partial;
};

cudaError_t forward(const Dims& d, const float* w, const float* X, int64_t rows, Pass& p, cudaStream_t s) {
  const int T = 256;
  linear_fwd<<<blocks_for(rows * d.hid, T), T, 0, s>>>(X, rows, d.in, w + d.w1(), w + d.b1(), d.hid, p.z1, p.a1, 1);
  linear_fwd<<<blocks_for(rows * d.hid, T), T, 0, s>>>(p.a1, rows, d.hid, w + d.w2(), w + d.b2(), d.hid, p.z2, p.a2,
                                                       1);
  linear_fwd<<<blocks_for(rows * d.out, T), T, 0, s>>>(p.a2, rows, d.hid, w + d.w3(), w + d.b3(), d.out, nullptr, p.y,
                                                       0);
  return cudaGetLastError();
}

cudaError_t backward(const Dims& d, const float* w, const float* X, const float* T_, const float* mask, int64_t rows,
                     float inv_msum, Pass& p, float* grad, float* loss, cudaStream_t s) {
  const int T = 256;
  const int64_t ny = rows * d.out;
  const int nb = blocks_for(ny, T);
  mse_grad<<<nb, T, 0, s>>>(p.y, T_, mask, ny, inv_msum, p.dy, p.partial);
  if (loss) sum_partials<<<1, 32, 0, s>>>(p.partial, nb, inv_msum, loss);
  linear_bwd_weight<<<blocks_for(d.hid * d.out + d.out, T), T, 0, s>>>(p.a2, p.dy, rows, d.hid, d.out, grad + d.w3(),
                                                                       grad + d.b3());
  linear_bwd_input<<<blocks_for(rows * d.hid, T), T, 0, s>>>(p.dy, rows, d.out, w + d.w3(), d.hid, p.z2, p.d2);
  linear_bwd_weight<<<blocks_for(d.hid * d.hid + d.hid, T), T, 0, s>>>(p.a1, p.d2, rows, d.hid, d.hid, grad + d.w2(),
                                                                       grad + d.b2());
  linear_bwd_input<<<blocks_for(rows * d.hid, T), T, 0, s>>>(p.d2, rows, d.hid, w + d.w2(), d.hid, p.z1, p.d1);
  linear_bwd_weight<<<blocks_for(d.in * d.hid + d.hid, T), T, 0, s>>>(X, p.d1, rows, d.in, d.hid, grad + d.w1(),
                                                                      grad + d.b1());
  return cudaGetLastError();
}

bool dims_ok(int in, int hid, int out) { return in >= 1 && in <= 64 && hid >= 1 && hid <= 256 && out >= 1 && out <= 64; }

size_t pass_floats(const Dims& d, int64_t rows) {
  return (size_t)rows * (4 * d.hid + 2 * d.out + 2 * d.hid) + (size_t)(rows * d.out / 256 + 2);
}

Pass carve(float* base, const Dims& d, int64_t rows) {
  Pass p;
  float* q = base;
  p.z1 = q, q += rows * d.hid;
  p.a1 = q, q += rows * d.hid;
  p.z2 = q, q += rows * d.hid;
  p.a2 = q, q += rows * d.hid;
  p.y = q, q += rows * d.out;
  p.dy = q, q += rows * d.out;
  p.d2 = q, q += rows * d.hid;
  p.d1 = q, q += rows * d.hid;
  p.partial = q;
  return p;
}

}  // namespace
}  // namespace perm

using namespace perm;

extern "C" {

int perm_mlp_size(int32_t in_dim, int32_t hidden, int32_t out_dim, int64_t* count) {
  if (!count || !dims_ok(in_dim, hidden, out_dim)) return PERM_EINVAL;
  *count = (int64_t)Dims{in_dim, hidden, out_dim}.total();
  return PERM_OK;
}

int perm_mlp_forward(const float* weights, int32_t in_dim, int32_t hidden, int32_t out_dim, const float* X,
                     int64_t rows, float* Y, void* stream) {
  if (!weights || !X || !Y || rows < 0 || !dims_ok(in_dim, hidden, out_dim)) return PERM_EINVAL;
  if (rows == 0) return PERM_OK;
  const Dims d{in_dim, hidden, out_dim};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* scratch = nullptr;
  if (cudaMallocAsync(&scratch, sizeof(float) * pass_floats(d, rows), s) != cudaSuccess) return PERM_ENOMEM;
  Pass p = carve(scratch, d, rows);
  p.y = Y;
  cudaError_t e = forward(d, weights, X, rows, p, s);
  cudaFreeAsync(scratch, s);
  return e == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

int perm_mlp_grad(const float* weights, int32_t in_dim, int32_t hidden, int32_t out_dim, const float* X,
                  const float* T, const float* mask, int64_t rows, float* grad, float* loss, void* stream) {
  if (!weights || !X || !T || !mask || !grad || rows <= 0 || !dims_ok(in_dim, hidden, out_dim)) return PERM_EINVAL;
  const Dims d{in_dim, hidden, out_dim};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // mask sum on the host side of the contract: the caller's mask is read on the device
  std::vector<float> hm((size_t)rows * out_dim);
  if (cudaMemcpyAsync(hm.data(), mask, sizeof(float) * hm.size(), cudaMemcpyDefault, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PERM_ECUDA;
  double msum = 0.0;
  for (float v : hm) msum += v;
  if (msum <= 0.0) return PERM_EINVAL;
  float* scratch = nullptr;
  if (cudaMallocAsync(&scratch, sizeof(float) * pass_floats(d, rows), s) != cudaSuccess) return PERM_ENOMEM;
  Pass p = carve(scratch, d, rows);
  cudaError_t e = forward(d, weights, X, rows, p, s);
  if (e == cudaSuccess) e = backward(d, weights, X, T, mask, rows, (float)(1.0 / msum), p, grad, loss, s);
  cudaFreeAsync(scratch, s);
  return e == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

int perm_mlp_train(const float* X, const float* T, const float* mask, int64_t rows, int32_t in_dim, int32_t hidden,
                   int32_t out_dim, int32_t epochs, int32_t batch, float lr, uint64_t seed, float* weights,
                   float* loss_history, void* stream) {
  if (!X || !T || !mask || !weights || rows <= 0 || epochs < 0 || batch <= 0 || !(lr > 0.f) ||
      !dims_ok(in_dim, hidden, out_dim))
    return PERM_EINVAL;
  const Dims d{in_dim, hidden, out_dim};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t B = batch < rows ? batch : rows;
  const int64_t nw = (int64_t)d.total();
  std::vector<float> hm((size_t)rows * out_dim);
  if (cudaMemcpyAsync(hm.data(), mask, sizeof(float) * hm.size(), cudaMemcpyDefault, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PERM_ECUDA;
  // mask weight of each mini-batch (rows are taken in order, the last batch may be short)
  const int64_t nbatch = (rows + B - 1) / B;
  std::vector<float> inv(nbatch);
  for (int64_t k = 0; k < nbatch; ++k) {
    double ms = 0.0;
    for (int64_t r = k * B; r < rows && r < (k + 1) * B; ++r)
      for (int o = 0; o < out_dim; ++o) ms += hm[(size_t)r * out_dim + o];
    inv[k] = ms > 0.0 ? (float)(1.0 / ms) : 0.f;
  }
  float* buf = nullptr;
  const size_t floats = pass_floats(d, B) + 3 * (size_t)nw + 1;
  if (cudaMallocAsync(&buf, sizeof(float) * floats, s) != cudaSuccess) return PERM_ENOMEM;
  float* grad = buf;
  float* m1 = grad + nw;
  float* m2 = m1 + nw;
  float* lossbuf = m2 + nw;
  Pass p = carve(lossbuf + 1, d, B);
  cudaError_t e = cudaSuccess;
  const int T_ = 256;
  init_weights<<<blocks_for(nw, T_), T_, 0, s>>>(weights, in_dim, hidden, out_dim, seed);
  cudaMemsetAsync(m1, 0, sizeof(float) * 2 * nw, s);
  int64_t step = 0;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    for (int64_t k = 0; k < nbatch && e == cudaSuccess; ++k) {
      if (inv[k] == 0.f) continue;
      const int64_t r0 = k * B, nr = (r0 + B <= rows) ? B : rows - r0;
      const float* Xb = X + r0 * in_dim;
      e = forward(d, weights, Xb, nr, p, s);
      if (e != cudaSuccess) break;
      const bool last = (k == nbatch - 1) && loss_history;
      e = backward(d, weights, Xb, T + r0 * out_dim, mask + r0 * out_dim, nr, inv[k], p, grad,
                   last ? lossbuf : nullptr, s);
      if (e != cudaSuccess) break;
      ++step;
      const float b1 = 0.9f, b2 = 0.999f;
      const float c1 = 1.f - (float)std::pow((double)b1, (double)step);
      const float c2 = 1.f - (float)std::pow((double)b2, (double)step);
      adam_step<<<blocks_for(nw, T_), T_, 0, s>>>(weights, grad, m1, m2, nw, lr, b1, b2, 1e-8f, c1, c2);
      e = cudaGetLastError();
      if (last && e == cudaSuccess)
        e = cudaMemcpyAsync(loss_history + ep, lossbuf, sizeof(float), cudaMemcpyDefault, s);
    }
  }
  cudaFreeAsync(buf, s);
  if (e != cudaSuccess) return PERM_ECUDA;
  return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

}  // extern "C"
