// Throughput probes of the pipes the kernels of this library run on, so that
// their rooflines are measured on the GPU at hand rather than taken from a
// data sheet: 32-bit logic operations (LOP3, the bit path of the Boolean
// contraction), shared-memory loads (the row-OR's table lookups), FP32 fused
// multiply-adds (the plot's filter) and FP64 adds and multiplies (the plot's
// exact decisions).
//
// Every probe runs long chains of independent operations in every thread of a
// grid that fills all SMs, times the launch with CUDA events after a warm-up
// launch, and also reads each block's SM cycle counter, so the result comes
// both per second and per SM per clock.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "pa_internal.h"

namespace pa {
namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeUnroll = 16;

// start/end cycle of every block (the widest block span gives the clock)
__device__ __forceinline__ void record_cycles(long long* cyc, long long t0) {
  __syncthreads();
  if (threadIdx.x == 0) {
    cyc[2 * blockIdx.x] = t0;
    cyc[2 * blockIdx.x + 1] = clock64();
  }
}

__global__ void __launch_bounds__(kProbeThreads)
lop3_probe_kernel(uint32_t* sink, long long* cyc, int iters) {
  const long long t0 = clock64();
  uint32_t a[8];
  const uint32_t b = 0x9E3779B9u * (threadIdx.x + 1), c = 0x85EBCA6Bu ^ blockIdx.x;
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = threadIdx.x * 2654435761u + j;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(b), "r"(c));
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) x ^= a[j];
  if (x == 0x12345678u) sink[threadIdx.x] = x;  // keeps the chains alive
  record_cycles(cyc, t0);
}

// Every warp reads 32 consecutive 8-byte words per load (256 bytes, no bank
// conflict), walking a 16 KB buffer.
__global__ void __launch_bounds__(kProbeThreads)
smem_probe_kernel(uint32_t* sink, long long* cyc, int iters) {
  __shared__ uint2 buf[2048];
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) buf[i] = make_uint2(i * 3u, i * 7u);
  __syncthreads();
  const long long t0 = clock64();
  const uint32_t base = static_cast<uint32_t>(__cvta_generic_to_shared(buf));
  uint32_t x0 = 0, x1 = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
      const uint32_t idx = (uint32_t)((warp * 64 + u * 32 + lane + it * 8) & 2047);
      uint32_t v0, v1;
      asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v0), "=r"(v1) : "r"(base + idx * 8));
      x0 ^= v0;
      x1 ^= v1;
    }
  }
  if ((x0 ^ x1) == 0x12345678u) sink[threadIdx.x] = x0;
  record_cycles(cyc, t0);
}

__global__ void __launch_bounds__(kProbeThreads)
ffma_probe_kernel(uint32_t* sink, long long* cyc, int iters) {
  const long long t0 = clock64();
  float a[8];
  const float b = 0.999999f, c = 1e-7f * (float)(threadIdx.x & 7);
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 1.0f + 0.001f * j;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < 8; ++j) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[j]) : "f"(b), "f"(c));
    }
  }
  float x = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) x += a[j];
  if (x == 12345.0f) sink[threadIdx.x] = 1;
  record_cycles(cyc, t0);
}

// FP64 without fused multiply-add, as the exact plot decisions use it: one
// multiply and one add per step of each chain.
__global__ void __launch_bounds__(kProbeThreads)
dmuladd_probe_kernel(uint32_t* sink, long long* cyc, int iters) {
  const long long t0 = clock64();
  double a[4];
  const double b = 0.9999999999, c = 1e-12 * (double)(threadIdx.x & 7);
#pragma unroll
  for (int j = 0; j < 4; ++j) a[j] = 1.0 + 0.001 * j;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        asm volatile("mul.rn.f64 %0, %0, %1;" : "+d"(a[j]) : "d"(b));
        asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(a[j]) : "d"(c));
      }
    }
  }
  double x = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) x += a[j];
  if (x == 12345.0) sink[threadIdx.x] = 1;
  record_cycles(cyc, t0);
}

}  // namespace

// Runs one probe: `ops_per_thread_iter` counted operations per thread and
// iteration.  Returns operations per second and, through *per_clk_sm, per SM
// per cycle (cycles from the widest block span, which also gives *clock_hz).
cudaError_t run_probe(int which, int sms, cudaStream_t s, double* per_s, double* per_clk_sm,
                      double* clock_hz) {
  const int blocks = sms;  // one 1024-thread block per SM: 32 warps, 8 chains each
  int iters = which == 3 ? 256 : 2048;
  uint32_t* sink = nullptr;
  long long* cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaMalloc(&sink, kProbeThreads * sizeof(uint32_t));
  if (err == cudaSuccess) err = cudaMalloc(&cyc, (size_t)blocks * 2 * sizeof(long long));
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  auto launch = [&]() {
    switch (which) {
      case 0: lop3_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(sink, cyc, iters); break;
      case 1: smem_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(sink, cyc, iters); break;
      case 2: ffma_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(sink, cyc, iters); break;
      default: dmuladd_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(sink, cyc, iters); break;
    }
  };
  float ms = 0.0f;
  std::vector<long long> h((size_t)blocks * 2);
  if (err == cudaSuccess) {
    launch();  // warm-up
    err = cudaEventRecord(e0, s);
  }
  if (err == cudaSuccess) {
    launch();
    err = cudaEventRecord(e1, s);
  }
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess)
    err = cudaMemcpy(h.data(), cyc, h.size() * sizeof(long long), cudaMemcpyDeviceToHost);
  if (err == cudaSuccess) {
    // operations per thread and iteration: 8 chains x unroll (LOP3, FFMA),
    // 8 bytes x unroll (shared loads), 4 chains x 2 x unroll (FP64)
    const double per_iter = which == 0 ? 8.0 * kProbeUnroll
                            : which == 1 ? 8.0 * kProbeUnroll
                            : which == 2 ? 2.0 * 8.0 * kProbeUnroll  // an FMA is 2 flops
                                         : 2.0 * 4.0 * kProbeUnroll;
    const double ops = (double)blocks * kProbeThreads * iters * per_iter;
    long long span = 0;
    for (int b = 0; b < blocks; ++b) span = std::max(span, h[2 * b + 1] - h[2 * b]);
    *per_s = ops / (ms * 1e-3);
    *clock_hz = 0.0;
    *per_clk_sm = 0.0;
    if (span > 0) {
      const double cycles = (double)span;
      *clock_hz = cycles / (ms * 1e-3);
      *per_clk_sm = ops / ((double)sms * cycles);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (cyc) cudaFree(cyc);
  return err;
}

}  // namespace pa
