// A small fully connected network (FP32) that predicts the time of a join
// from its shape and operand densities: the learned cost model behind the
// PA_ORDER_LEARNED join order.  Forward, backward and Adam kernels are plain
// CUDA; all reductions are deterministic (no atomics), so a gradient computed
// twice is the same bit for bit.
//
// Layout of the parameters (one flat FP32 vector): for every layer l, the
// weights W_l[out][in] row-major, then the biases b_l[out].  Hidden layers use
// ReLU, the output layer is linear with one output.
#include <math.h>
#include <string.h>

#include <vector>

#include "mlp.h"

namespace pa {

// y[n][o] = act(sum_i W[o][i] x[n][i] + b[o]); also keeps the pre-activation
// when `pre` is given.  Block: blockDim.x threads own outputs o, 32 samples per
// block, staged in shared memory.
__global__ void mlp_layer_fwd(const float* __restrict__ x, int n, int nin, const float* __restrict__ W,
                              const float* __restrict__ b, int nout, int relu, float* __restrict__ y,
                              float* __restrict__ pre) {
  extern __shared__ float xs[];  // [32][nin]
  const int n0 = blockIdx.x * 32;
  const int rows = min(32, n - n0);
  for (int t = threadIdx.x; t < rows * nin; t += blockDim.x) xs[t] = x[(size_t)n0 * nin + t];
  __syncthreads();
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const float* w = W + (size_t)o * nin;
    for (int r = 0; r < rows; ++r) {
      float acc = b[o];
      const float* xr = xs + r * nin;
      for (int i = 0; i < nin; ++i) acc = fmaf(w[i], xr[i], acc);
      const size_t k = (size_t)(n0 + r) * nout + o;
      if (pre) pre[k] = acc;
      y[k] = (relu && acc < 0.0f) ? 0.0f : acc;
    }
  }
}

// d = (y - t) / n  for the loss 0.5 * mean (y - t)^2, and the loss itself
// (single block, deterministic tree reduction)
__global__ void mlp_loss(const float* __restrict__ y, const float* __restrict__ t, int n,
                         float* __restrict__ d, float* __restrict__ loss) {
  __shared__ float part[256];
  float s = 0.0f;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const float e = y[k] - t[k];
    d[k] = e / (float)n;
    s += e * e;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = 0.5f * part[0] / (float)n;
}

// dW[o][i] = sum_n d[n][o] x[n][i]; db[o] = sum_n d[n][o]   (thread per weight)
__global__ void mlp_layer_dw(const float* __restrict__ d, const float* __restrict__ x, int n,
                             int nin, int nout, float* __restrict__ dW, float* __restrict__ db) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = nout * (nin + 1);
  if (k >= total) return;
  const int o = k / (nin + 1), i = k % (nin + 1);
  float acc = 0.0f;
  if (i < nin) {
    for (int r = 0; r < n; ++r) acc = fmaf(d[(size_t)r * nout + o], x[(size_t)r * nin + i], acc);
    dW[(size_t)o * nin + i] = acc;
  } else {
    for (int r = 0; r < n; ++r) acc += d[(size_t)r * nout + o];
    db[o] = acc;
  }
}

// dx[n][i] = (sum_o d[n][o] W[o][i]) * [pre_prev[n][i] > 0]   (thread per input)
__global__ void mlp_layer_dx(const float* __restrict__ d, const float* __restrict__ W, int n,
                             int nin, int nout, const float* __restrict__ pre_prev,
                             float* __restrict__ dx) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (size_t)n * nin) return;
  const int r = (int)(k / nin), i = (int)(k % nin);
  float acc = 0.0f;
  for (int o = 0; o < nout; ++o) acc = fmaf(d[(size_t)r * nout + o], W[(size_t)o * nin + i], acc);
  if (pre_prev && !(pre_prev[k] > 0.0f)) acc = 0.0f;
  dx[k] = acc;
}

// Adam (Kingma and Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * mhat / (sqrt(vhat) + eps), with bias corrections c1, c2.
__global__ void mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                         float* __restrict__ v, int np, float lr, float b1, float b2, float eps,
                         float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.0f - b1) * gk;
  const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// ------------------------------------------------------------------ host
Mlp::Mlp(int nin_, int hidden_, int nlayers_) : nin(nin_), hidden(hidden_), nlayers(nlayers_) {
  sizes.push_back(nin);
  for (int l = 0; l < nlayers; ++l) sizes.push_back(hidden);
  sizes.push_back(1);
  np = 0;
  for (size_t l = 0; l + 1 < sizes.size(); ++l) {
    woff.push_back(np);
    np += (int64_t)sizes[l + 1] * sizes[l];
    boff.push_back(np);
    np += sizes[l + 1];
  }
}

cudaError_t Mlp::alloc_params() {
  cudaError_t e;
  if ((e = cudaMalloc(&p, np * 4)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&g, np * 4)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&m, np * 4)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&v, np * 4)) != cudaSuccess) return e;
  if ((e = cudaMemset(m, 0, np * 4)) != cudaSuccess) return e;
  if ((e = cudaMemset(v, 0, np * 4)) != cudaSuccess) return e;
  if ((e = cudaMemset(g, 0, np * 4)) != cudaSuccess) return e;
  return cudaMalloc(&loss, 4);
}

cudaError_t Mlp::reserve(int n) {
  if (n <= cap) return cudaSuccess;
  free_acts();
  const int L = (int)sizes.size() - 1;
  acts.assign(L + 1, nullptr);
  pres.assign(L + 1, nullptr);
  cudaError_t e;
  for (int l = 1; l <= L; ++l) {
    if ((e = cudaMalloc(&acts[l], (size_t)n * sizes[l] * 4)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&pres[l], (size_t)n * sizes[l] * 4)) != cudaSuccess) return e;
  }
  size_t dmax = 0;
  for (int s : sizes) dmax = std::max(dmax, (size_t)s);
  if ((e = cudaMalloc(&dbuf0, (size_t)n * dmax * 4)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&dbuf1, (size_t)n * dmax * 4)) != cudaSuccess) return e;
  cap = n;
  return cudaSuccess;
}

void Mlp::free_acts() {
  for (float* a : acts) if (a) cudaFree(a);
  for (float* a : pres) if (a) cudaFree(a);
  acts.clear();
  pres.clear();
  if (dbuf0) cudaFree(dbuf0);
  if (dbuf1) cudaFree(dbuf1);
  dbuf0 = dbuf1 = nullptr;
  cap = 0;
}

Mlp::~Mlp() {
  free_acts();
  if (p) cudaFree(p);
  if (g) cudaFree(g);
  if (m) cudaFree(m);
  if (v) cudaFree(v);
  if (loss) cudaFree(loss);
}

cudaError_t Mlp::forward(const float* x, int n, float* y, cudaStream_t s) {
  cudaError_t e = reserve(n);
  if (e != cudaSuccess) return e;
  const int L = (int)sizes.size() - 1;
  const float* in = x;
  for (int l = 0; l < L; ++l) {
    const int ni = sizes[l], no = sizes[l + 1];
    const unsigned blocks = (unsigned)((n + 31) / 32);
    mlp_layer_fwd<<<blocks, 128, (size_t)32 * ni * 4, s>>>(in, n, ni, p + woff[l], p + boff[l], no,
                                                        l < L - 1 ? 1 : 0, acts[l + 1], pres[l + 1]);
    in = acts[l + 1];
  }
  if (y) cudaMemcpyAsync(y, acts[L], (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

cudaError_t Mlp::backward(const float* x, const float* t, int n, cudaStream_t s) {
  cudaError_t e = forward(x, n, nullptr, s);
  if (e != cudaSuccess) return e;
  const int L = (int)sizes.size() - 1;
  mlp_loss<<<1, 256, 0, s>>>(acts[L], t, n, dbuf0, loss);
  float* d = dbuf0;
  float* dn = dbuf1;
  for (int l = L - 1; l >= 0; --l) {
    const int ni = sizes[l], no = sizes[l + 1];
    const float* xin = (l == 0) ? x : acts[l];
    const int tw = no * (ni + 1);
    mlp_layer_dw<<<(tw + 255) / 256, 256, 0, s>>>(d, xin, n, ni, no, g + woff[l], g + boff[l]);
    if (l > 0) {
      const size_t tx = (size_t)n * ni;
      mlp_layer_dx<<<(unsigned)((tx + 255) / 256), 256, 0, s>>>(d, p + woff[l], n, ni, no, pres[l],
                                                                dn);
      std::swap(d, dn);
    }
  }
  return cudaGetLastError();
}

cudaError_t Mlp::adam(float lr, float b1, float b2, float eps, cudaStream_t s) {
  ++step;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  mlp_adam<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(p, g, m, v, (int)np, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace pa
