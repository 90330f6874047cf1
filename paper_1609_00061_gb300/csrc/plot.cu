// Plot kernels: the sample-in-center plot of Sec. 3.2 for polynomial relations.
//
// Pixel e is on when f(c_e) is finite and |f(c_e)| <= eps (PA_EQ; f <= eps for
// PA_LE, f < eps for PA_LT; strict makes every test "<").  The decision is
// defined by the IEEE double evaluation fixed in pa.h.  GB300 runs FP64 at a
// small fraction of its FP32 rate, so each pixel is first evaluated in FP32
// together with a rigorous bound on |f32 - f64|; only pixels whose FP32 value
// lies within that bound of eps are evaluated again in FP64.  The result is
// therefore the FP64 decision, bit for bit.
//
// Error bound (row-hoisted evaluation, f = sum_j g_j y^j, y the last port):
//   g_j are computed once per row in FP64 (exactly as the nested evaluation
//   does) and rounded to FP32; y32 = fl32(y64).  Then
//   |f32 - f64| <= (2D+1) u a + (D+1) u a + (2D+1) u64 a  (u = 2^-24),
//   a = sum_j |g_j| |y|^j, from the FP32 evaluation error, the rounding of
//   g_j and y, and the FP64 evaluation error.  The kernel uses
//   B = (4D + 8) u * 1.01 * a32 + 2^-21 eps + 1e-30, which also covers the
//   rounding of a32, of eps to FP32 and of the comparisons themselves.
#include <float.h>

#include "pa_internal.h"

namespace pa {

// ---------------------------------------------------------------- centres
__global__ void axis_table_kernel(const AxisTableJob* __restrict__ jobs, int njobs, int64_t total,
                                  double* __restrict__ x64, float* __restrict__ x32) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].off <= g) lo = mid; else hi = mid - 1;
    }
    const AxisTableJob j = jobs[lo];
    const int64_t i = g - j.off;
    const double delta = __ddiv_rn(__dsub_rn(j.hi, j.lo), (double)j.res);
    const double t = __dadd_rn((double)i, 0.5);
    const double x = __dadd_rn(j.lo, __dmul_rn(t, delta));
    x64[g] = x;
    x32[g] = __double2float_rn(x);
  }
}

void launch_axis_tables(const AxisTableJob* d_jobs, int njobs, int64_t total, double* x64,
                        float* x32, cudaStream_t s) {
  if (total <= 0) return;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  axis_table_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_jobs, njobs, total, x64, x32);
}

// -------------------------------------------------------- nested evaluation
// sum_{e_k = 0}^{rem} nest(k-1, rem - e_k) * x_k^{e_k}; coefficients are read
// in nest order through cp.
__device__ double nest_dev(int k, int rem, const double*& cp, const double* x) {
  if (k < 0) return *cp++;
  double s = 0.0, pw = 1.0;
  for (int e = 0; e <= rem; ++e) {
    const double term = __dmul_rn(nest_dev(k - 1, rem - e, cp, x), pw);
    s = (e == 0) ? term : __dadd_rn(s, term);
    pw = __dmul_rn(pw, x[k]);
  }
  return s;
}

__device__ __forceinline__ bool decide64(double f, int kind, double eps, int strict) {
  if (!isfinite(f)) return false;
  if (kind == PA_EQ) {
    const double d = fabs(f);
    return strict ? (d < eps) : (d <= eps);
  }
  if (kind == PA_LE) return strict ? (f < eps) : (f <= eps);
  return f < eps;
}

// --------------------------------------------------------------- plot kernel
constexpr int kPlotThreads = 256;

// FP32 filter for one pixel of a hoisted row: 1 = on, 0 = off, 2 = undecided
// (the FP64 evaluation decides).  DS is the degree when known at compile time.
template <int DS>
__device__ __forceinline__ int filter32(float y, const float* g, const float* ga, int D, int kind,
                                        float eps32, float kfac, float amarg) {
  const int deg = DS >= 0 ? DS : D;
  float s = g[0], a = ga[0], pw = 1.0f;
#pragma unroll
  for (int j = 1; j <= (DS >= 0 ? DS : kMaxDeg); ++j) {
    if (DS < 0 && j > deg) break;
    pw = __fmul_rn(pw, y);
    s = __fmaf_rn(g[j], pw, s);
    a = __fmaf_rn(ga[j], fabsf(pw), a);
  }
  const float d = (kind == PA_EQ) ? fabsf(s) : s;
  const float B = __fmaf_rn(a, kfac, amarg);
  if (!(a <= FLT_MAX)) return 2;
  if (d > __fadd_rn(eps32, B)) return 0;
  if (d < __fsub_rn(eps32, B)) return 1;
  return 2;
}

// exact FP64 value of sum_j g_j y^j in the order fixed by pa.h
__device__ __noinline__ bool exact64(double y64, const double* g6, int D, int kind, double eps,
                                     int strict) {
  double s6 = g6[0], p6 = 1.0;
  for (int j = 1; j <= D; ++j) {
    p6 = __dmul_rn(p6, y64);
    s6 = __dadd_rn(s6, __dmul_rn(g6[j], p6));
  }
  return decide64(s6, kind, eps, strict);
}

// general path (a variable on several ports): full nested FP64 evaluation
__device__ __noinline__ bool general64(const PlotJob* J, int64_t row, int64_t i) {
  const int ndim = J->ndim;
  int64_t rest = row;
  int idx[kMaxDim];
  idx[ndim - 1] = (int)i;
  for (int a = ndim - 2; a >= 0; --a) {
    idx[a] = (int)(rest % J->res[a]);
    rest /= J->res[a];
  }
  double x[kMaxDim];
  for (int p = 0; p < J->arity; ++p) x[p] = J->x64[p][idx[J->port_axis[p]]];
  const double* cp = J->coeffs;
  return decide64(nest_dev(J->arity - 1, J->degree, cp, x), J->kind, J->eps, J->strict);
}

// phase A: one thread per row computes the row's polynomial in the last port,
// g_j = the inner nested sums (FP64, the order of pa.h), and its FP32 copies
__device__ __noinline__ void row_polynomial(const PlotJob* J, int64_t row, int D, double* g64,
                                            float* g32, float* ga32) {
  const int ndim = J->ndim;
  int64_t rest = row;
  int idx[kMaxDim];
  for (int a = ndim - 2; a >= 0; --a) {
    idx[a] = (int)(rest % J->res[a]);
    rest /= J->res[a];
  }
  double x[kMaxDim];
  for (int p = 0; p < J->arity - 1; ++p) x[p] = J->x64[p][idx[J->port_axis[p]]];
  const double* cp = J->coeffs;
  for (int j = 0; j <= D; ++j) {
    const double g = nest_dev(J->arity - 2, D - j, cp, x);
    g64[j] = g;
    const float g1 = __double2float_rn(g);
    g32[j] = g1;
    ga32[j] = fabsf(g1);
  }
}

template <int DS>
__global__ void __launch_bounds__(kPlotThreads)
plot_kernel(const PlotJob* __restrict__ jobs, int njobs, int smem_stride) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_job;
  if (threadIdx.x == 0) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].tile0 <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_job = lo;
  }
  __syncthreads();
  const PlotJob* J = jobs + s_job;
  const int D = DS >= 0 ? DS : J->degree;
  const int D1 = D + 1;
  const int arity = J->arity;
  const int64_t row_words = J->row_words;
  const int res_last = J->res[J->ndim - 1];
  const int R = J->rows_per_tile;
  const int64_t row0 = ((int64_t)blockIdx.x - J->tile0) * R;
  const int nr = (int)min((int64_t)R, J->nrows - row0);
  const int kind = J->kind, strict = J->strict;
  const double eps = J->eps;
  const bool hoisted = J->hoisted != 0;

  double* g64 = reinterpret_cast<double*>(smem);
  float* g32 = reinterpret_cast<float*>(g64 + smem_stride);
  float* ga32 = g32 + smem_stride;

  if (hoisted) {
    for (int r = threadIdx.x; r < nr; r += blockDim.x) row_polynomial(J, row0 + r, D, g64 + r * D1, g32 + r * D1, ga32 + r * D1);
    __syncthreads();
  }

  // phase B: a warp task is (row, run of up to 32 words); lane l evaluates the
  // pixels 64w + l and 64w + 32 + l of every word w of the run
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int64_t runs_per_row = (row_words + 31) / 32;
  const int64_t ntasks = (int64_t)nr * runs_per_row;
  const float* __restrict__ y32t = J->x32_last;
  const double* __restrict__ y64t = J->x64[arity - 1];
  const float eps32 = J->eps32, kfac = J->kfac, amarg = J->abs_margin;
  uint64_t* __restrict__ out = J->out;
  constexpr int kG = DS >= 0 ? DS + 1 : kMaxDeg + 1;
  float g[kG], ga[kG];

  for (int64_t t = warp; t < ntasks; t += nwarps) {
    const int r = (int)(t / runs_per_row);
    const int64_t w0 = (t % runs_per_row) * 32;
    const int nw = (int)min((int64_t)32, row_words - w0);
    if (hoisted) {
#pragma unroll
      for (int j = 0; j < kG; ++j) {
        if (DS < 0 && j > D) break;
        g[j] = g32[r * D1 + j];
        ga[j] = ga32[r * D1 + j];
      }
    }
    uint64_t mine = 0;
    for (int it = 0; it < nw; ++it) {
      const int64_t i0 = (w0 + it) * 64 + lane;
      const int64_t i1 = i0 + 32;
      bool b0 = false, b1 = false;
      if (hoisted) {
        const float y0 = (i0 < res_last) ? y32t[i0] : 0.0f;
        const float y1 = (i1 < res_last) ? y32t[i1] : 0.0f;
        int c0 = filter32<DS>(y0, g, ga, D, kind, eps32, kfac, amarg);
        int c1 = filter32<DS>(y1, g, ga, D, kind, eps32, kfac, amarg);
        if (i0 >= res_last) c0 = 0;
        if (i1 >= res_last) c1 = 0;
        if (c0 == 2) c0 = exact64(y64t[i0], g64 + r * D1, D, kind, eps, strict);
        if (c1 == 2) c1 = exact64(y64t[i1], g64 + r * D1, D, kind, eps, strict);
        b0 = c0 != 0;
        b1 = c1 != 0;
      } else {
        if (i0 < res_last) b0 = general64(J, row0 + r, i0);
        if (i1 < res_last) b1 = general64(J, row0 + r, i1);
      }
      const unsigned lo = __ballot_sync(0xffffffffu, b0);
      const unsigned hi = __ballot_sync(0xffffffffu, b1);
      if (lane == it) mine = ((uint64_t)hi << 32) | lo;
    }
    if (lane < nw) out[(row0 + r) * row_words + w0 + lane] = mine;
  }
}

cudaError_t probe_kernel_image() {
  cudaFuncAttributes attr;
  return cudaFuncGetAttributes(&attr, plot_kernel<-1>);
}

void launch_plot(const PlotJob* d_jobs, int njobs, int64_t total_tiles, int max_rows_per_tile,
                 int max_degree, int common_degree, cudaStream_t s) {
  if (total_tiles <= 0) return;
  const int stride = max_rows_per_tile * (max_degree + 1);
  const size_t smem = (size_t)stride * (sizeof(double) + 2 * sizeof(float));
  const unsigned grid = (unsigned)total_tiles;
  switch (common_degree) {
    case 1: plot_kernel<1><<<grid, kPlotThreads, smem, s>>>(d_jobs, njobs, stride); break;
    case 2: plot_kernel<2><<<grid, kPlotThreads, smem, s>>>(d_jobs, njobs, stride); break;
    case 3: plot_kernel<3><<<grid, kPlotThreads, smem, s>>>(d_jobs, njobs, stride); break;
    case 4: plot_kernel<4><<<grid, kPlotThreads, smem, s>>>(d_jobs, njobs, stride); break;
    default: plot_kernel<-1><<<grid, kPlotThreads, smem, s>>>(d_jobs, njobs, stride); break;
  }
}

}  // namespace pa
