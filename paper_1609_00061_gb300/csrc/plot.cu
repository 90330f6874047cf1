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
// One block plots a tile of rows (all axes but the last fixed):
//   A1. thread (r, j) computes the row polynomial's coefficient g_j in FP64
//       (the inner nested sums, exactly as pa.h orders them) and its FP32 copy;
//       the FP32 centres of the last axis are copied to shared memory;
//   A2. thread r bounds the FP32 evaluation error of its row,
//       B_r = (4D+8) u 1.01 a_r + 2^-21 eps + 1e-30, a_r = sum_j |g_j| Y^j with
//       Y >= every |y| of the axis, and stores the thresholds eps -+ B_r;
//   B.  thread per output word: the 64 pixels of the word are evaluated in FP32
//       (f = g_0 + g_1 y + ... by fused multiply-adds); |f| below eps - B_r is
//       on, above eps + B_r is off, anything else is decided by the exact FP64
//       evaluation.  Bits are set directly in the thread's word, so no warp
//       vote is needed and the row's words are stored coalesced.
constexpr int kPlotThreads = 256;
constexpr int kYTabCap = 12288;  // largest last axis whose centres are staged in shared memory

__device__ __forceinline__ int ypad(int i) { return i + (i >> 6); }

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

// g_j of one row: the nested sums over the first arity-1 ports with e_last = j
__device__ __noinline__ double row_coeff(const PlotJob* J, int64_t row, int j) {
  const int ndim = J->ndim;
  int64_t rest = row;
  int idx[kMaxDim];
  for (int a = ndim - 2; a >= 0; --a) {
    idx[a] = (int)(rest % J->res[a]);
    rest /= J->res[a];
  }
  double x[kMaxDim];
  for (int p = 0; p < J->arity - 1; ++p) x[p] = J->x64[p][idx[J->port_axis[p]]];
  const double* cp = J->coeffs + J->block_off[j];
  return nest_dev(J->arity - 2, J->degree - j, cp, x);
}

// The 64 pixels of one word in FP32: bit b of *on is set when the pixel is
// certainly on, bit b of *pending when only the FP64 evaluation can decide.
template <int DS, bool EQ, bool YS>
__device__ __forceinline__ void eval_word(const float* g, int D, float lo, float hi,
                                          const float* ytab_w, const float* __restrict__ y32_w,
                                          int nb, uint64_t* on, uint64_t* pending) {
  uint32_t on_lo = 0, on_hi = 0, pe_lo = 0, pe_hi = 0;
#pragma unroll
  for (int bb = 0; bb < 64; ++bb) {
    if (bb < nb) {
      const float y = YS ? ytab_w[bb] : __ldg(y32_w + bb);
      float s = g[0], pw = y;
      if (DS >= 0) {
#pragma unroll
        for (int j = 1; j <= (DS >= 0 ? DS : 1); ++j) {
          if (j > 1) pw = __fmul_rn(pw, y);
          s = __fmaf_rn(g[j], pw, s);
        }
      } else {
        for (int j = 1; j <= D; ++j) {
          if (j > 1) pw = __fmul_rn(pw, y);
          s = __fmaf_rn(g[j], pw, s);
        }
      }
      const float dd = EQ ? fabsf(s) : s;
      const bool c_on = dd < lo;
      const bool c_pe = !c_on && !(dd > hi);
      if (bb < 32) {
        if (c_on) on_lo |= 1u << bb;
        if (c_pe) pe_lo |= 1u << bb;
      } else {
        if (c_on) on_hi |= 1u << (bb - 32);
        if (c_pe) pe_hi |= 1u << (bb - 32);
      }
    }
  }
  *on = ((uint64_t)on_hi << 32) | on_lo;
  *pending = ((uint64_t)pe_hi << 32) | pe_lo;
}

template <int DS>
__global__ void __launch_bounds__(kPlotThreads)
plot_kernel(const PlotJob* __restrict__ jobs, int njobs, int gstride, int rows_cap, int ytab_cap) {
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
  const int row_words = (int)J->row_words;
  const int res_last = J->res[J->ndim - 1];
  const int R = J->rows_per_tile;
  const int64_t row0 = ((int64_t)blockIdx.x - J->tile0) * R;
  const int nr = (int)min((int64_t)R, J->nrows - row0);
  const int kind = J->kind, strict = J->strict;
  const double eps = J->eps;
  const bool hoisted = J->hoisted != 0;

  double* g64 = reinterpret_cast<double*>(smem);
  float* g32 = reinterpret_cast<float*>(g64 + gstride);
  float* thr = g32 + gstride;                 // [R][2]: eps - B_r, eps + B_r
  float* ytab = thr + 2 * rows_cap;
  const bool ysmem = res_last <= ytab_cap;
  const float* __restrict__ y32g = J->x32_last;

  if (hoisted) {
    for (int t = threadIdx.x; t < nr * D1; t += blockDim.x) {
      const int r = t / D1, j = t % D1;
      const double g = row_coeff(J, row0 + r, j);
      g64[r * D1 + j] = g;
      g32[r * D1 + j] = __double2float_rn(g);
    }
    if (ysmem)
      for (int i = threadIdx.x; i < res_last; i += blockDim.x) ytab[ypad(i)] = y32g[i];
    __syncthreads();
    const float Y = J->ymax, kfac = J->kfac, amarg = J->abs_margin, eps32 = J->eps32;
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      float a = 0.0f, pw = 1.0f;
      for (int j = 0; j <= D; ++j) {
        a = __fmaf_rn(fabsf(g32[r * D1 + j]), pw, a);
        pw = __fmul_rn(pw, Y);
      }
      const float B = __fmaf_rn(a, kfac, amarg);
      float lo = __fsub_rn(eps32, B), hi = __fadd_rn(eps32, B);
      if (!(a <= FLT_MAX) || !(B <= FLT_MAX)) {
        lo = -INFINITY;   // nothing is certain: every pixel of the row takes the FP64 path
        hi = INFINITY;
      }
      thr[2 * r] = lo;
      thr[2 * r + 1] = hi;
    }
    __syncthreads();
  }

  const double* __restrict__ y64t = J->x64[arity - 1];
  uint64_t* __restrict__ out = J->out;
  constexpr int kG = DS >= 0 ? DS + 1 : kMaxDeg + 1;
  const int nwords = nr * row_words;
  for (int f = threadIdx.x; f < nwords; f += blockDim.x) {
    const int r = f / row_words, w = f - r * row_words;
    const int i0 = w * 64;
    const int nb = min(64, res_last - i0);
    uint64_t word = 0;
    if (hoisted) {
      float g[kG];
#pragma unroll
      for (int j = 0; j < kG; ++j) g[j] = (DS >= 0 || j <= D) ? g32[r * D1 + j] : 0.0f;
      const float lo = thr[2 * r], hi = thr[2 * r + 1];
      uint64_t pending = 0;
      const float* ytab_w = ytab + i0 + w;  // ypad(i0 + b) = i0 + w + b
      const float* y32_w = y32g + i0;
      if (kind == PA_EQ) {
        if (ysmem) eval_word<DS, true, true>(g, D, lo, hi, ytab_w, y32_w, nb, &word, &pending);
        else eval_word<DS, true, false>(g, D, lo, hi, ytab_w, y32_w, nb, &word, &pending);
      } else {
        if (ysmem) eval_word<DS, false, true>(g, D, lo, hi, ytab_w, y32_w, nb, &word, &pending);
        else eval_word<DS, false, false>(g, D, lo, hi, ytab_w, y32_w, nb, &word, &pending);
      }
      while (pending) {
        const int bb = __ffsll((long long)pending) - 1;
        pending &= pending - 1;
        if (exact64(y64t[i0 + bb], g64 + r * D1, D, kind, eps, strict)) word |= (1ull << bb);
      }
    } else {
      for (int bb = 0; bb < nb; ++bb)
        if (general64(J, row0 + r, i0 + bb)) word |= (1ull << bb);
    }
    out[(row0 + r) * (int64_t)row_words + w] = word;
  }
}

cudaError_t probe_kernel_image() {
  cudaFuncAttributes attr;
  return cudaFuncGetAttributes(&attr, plot_kernel<-1>);
}

void launch_plot(const PlotJob* d_jobs, int njobs, int64_t total_tiles, int max_rows_per_tile,
                 int max_degree, int common_degree, int max_res_last, cudaStream_t s) {
  if (total_tiles <= 0) return;
  const int gstride = max_rows_per_tile * (max_degree + 1);
  const int ycap = max_res_last <= kYTabCap ? max_res_last : 0;
  const size_t smem = (size_t)gstride * (sizeof(double) + sizeof(float)) +
                      (size_t)max_rows_per_tile * 2 * sizeof(float) +
                      (size_t)(ycap + ycap / 64 + 1) * sizeof(float);
  const unsigned grid = (unsigned)total_tiles;
#define PA_PLOT(DD)                                                                           \
  do {                                                                                        \
    cudaFuncSetAttribute(plot_kernel<DD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    plot_kernel<DD><<<grid, kPlotThreads, smem, s>>>(d_jobs, njobs, gstride, max_rows_per_tile, ycap);           \
  } while (0)
  switch (common_degree) {
    case 1: PA_PLOT(1); break;
    case 2: PA_PLOT(2); break;
    case 3: PA_PLOT(3); break;
    case 4: PA_PLOT(4); break;
    default: PA_PLOT(-1); break;
  }
#undef PA_PLOT
}

}  // namespace pa
