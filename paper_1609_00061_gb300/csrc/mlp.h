// The learned join-cost model: a small FP32 MLP with its own CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace pa {

struct Mlp {
  int nin, hidden, nlayers;
  std::vector<int> sizes;       // nin, hidden x nlayers, 1
  std::vector<int64_t> woff, boff;
  int64_t np = 0;               // number of parameters
  float* p = nullptr;           // parameters (device)
  float* g = nullptr;           // gradient of the last backward()
  float* m = nullptr;           // Adam first moment
  float* v = nullptr;           // Adam second moment
  float* loss = nullptr;        // device scalar: loss of the last backward()
  int64_t step = 0;
  int cap = 0;                  // samples the activation buffers hold
  std::vector<float*> acts, pres;
  float* dbuf0 = nullptr;
  float* dbuf1 = nullptr;

  Mlp(int nin, int hidden, int nlayers);
  ~Mlp();
  cudaError_t alloc_params();
  cudaError_t reserve(int n);
  void free_acts();
  // y[n] = net(x[n][nin]) (device pointers; y may be null to keep only acts)
  cudaError_t forward(const float* x, int n, float* y, cudaStream_t s);
  // forward, loss 0.5 mean (y - t)^2 into *loss, gradient into g
  cudaError_t backward(const float* x, const float* t, int n, cudaStream_t s);
  cudaError_t adam(float lr, float b1, float b2, float eps, cudaStream_t s);
};

}  // namespace pa
