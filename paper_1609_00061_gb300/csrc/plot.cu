// Plot kernels: the sample-in-center plot of Sec. 3.2 for polynomial relations.
//
// Pixel e is on when f(c_e) is finite and |f(c_e)| <= eps (PA_EQ; f <= eps for
// PA_LE, f < eps for PA_LT; strict makes every test "<").  The decision is
// defined by the IEEE double evaluation fixed in pa.h.  GB300 runs FP64 at a
// small fraction of its FP32 rate, so each pixel is first evaluated in FP32
// against a rigorous bound on |f32 - f64|; only pixels whose FP32 value lies
// within that bound of eps are evaluated again in FP64.  The result is the
// FP64 decision, bit for bit.
//
// Row hoisting: with every port but the last fixed, f is a polynomial
// f = sum_j g_j y^j in the last port y.  The g_j are exactly the inner nested
// sums of the pa.h evaluation order, so computing them once per row in FP64
// (at the start of the block that plots the row) and finishing each pixel with
// sum_j g_j y^j performs the very same IEEE operations as evaluating the pixel
// from scratch.
//
// Error bound for the FP32 pass (u = 2^-24, D the degree, g_j rounded to FP32,
// y32 = fl32(y64), a = sum_j |g_j| |y|^j):
//   |f32 - f64| <= (2D+1) u a   (FP32 evaluation)
//               +  (D+1) u a    (rounding of g_j and y)
//               +  (2D+1) 2^-53 a (FP64 evaluation)
// and a <= a_row = sum_j |g_j| Y^j with Y >= |y| on the whole axis.  The kernel
// uses B_row = (4D + 8) u 1.01 a_row + 2^-21 eps + 1e-30, which also covers the
// rounding of a_row, of eps to FP32 and of the thresholds themselves.
//
// Whole-word pruning (the paper's suggestion of skipping regions whose error
// provably exceeds eps, here per 64-pixel word).  With F the exact row
// polynomial, y_c the word's pixel 32 and h >= the distance from y_c to any
// centre of the word, Taylor's theorem gives for every pixel y of the word
//   |F(y) - F(y_c)| <= h |F'(y_c)| + h^2 / 2 max |F''|,
// max |F''| <= S2 = sum_j j (j-1) |g_j| Yw^(j-2) with Yw = |y_c| + h, and the
// FP32 derivative d_c (Horner) satisfies |d_c - F'(y_c)| <= (2D + 4) u S1,
// S1 = sum_j j |g_j| |y_c|^(j-1).  With T = 1.01 (h (|d_c| + (2D+4) u S1) +
// h^2 S2 / 2) and the pixel bound B_row used three times (f32 vs f64 at y_c,
// f64 vs F at y_c and at y):
//   |f64(y) - f32(y_c)| <= 3 B_row + T,
// so f32(y_c) beyond eps + B_row + 4 B_row + T proves the whole word off (|f|
// for PA_EQ), and for PA_LE / PA_LT f32(y_c) below eps - B_row - 4 B_row - T
// proves it on; only the remaining words are evaluated pixel by pixel.
#include <float.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "expr_eval.cuh"
#include "pa_internal.h"

namespace pa {

// -------------------------------------------------------- nested evaluation
// nest(k, rem) = sum_{e_k = 0}^{rem} nest(k-1, rem - e_k) * x_k^{e_k}, with
// nest(-1, .) the next coefficient in nest order (read through cp).  No
// evaluation recurses at run time: a recursive device function runs on the
// 1 KB default call stack, which an 8-port relation (eight frames) overflows.
template <int K>
__device__ __forceinline__ double nest_t(int rem, const double*& cp, const double* x) {
  if constexpr (K < 0) {
    return *cp++;
  } else {
    double s = 0.0, pw = 1.0;
    for (int e = 0; e <= rem; ++e) {
      const double term = __dmul_rn(nest_t<K - 1>(rem - e, cp, x), pw);
      s = (e == 0) ? term : __dadd_rn(s, term);
      pw = __dmul_rn(pw, x[K]);
    }
    return s;
  }
}

struct NestOut {
  double v;
  const double* cp;  // past the coefficients read
};

// Any depth as a loop over an explicit per-depth state (partial sum, power of
// x_L, exponent, remaining degree): the same products and sums in the same
// order as nest_t, out of line and with few registers, for the deep cases.
__device__ __noinline__ NestOut nest_deep(int k, int rem, const double* cp, const double* x) {
  if (k < 0) return {*cp, cp + 1};
  double s[kMaxDim], pw[kMaxDim];
  int e[kMaxDim], rm[kMaxDim];
  int L = k;
  rm[k] = rem;
  e[k] = 0;
  pw[k] = 1.0;
  s[k] = 0.0;
  for (;;) {
    // open the term e[L] of depth L down to depth 0
    while (L > 0) {
      rm[L - 1] = rm[L] - e[L];
      e[L - 1] = 0;
      pw[L - 1] = 1.0;
      s[L - 1] = 0.0;
      --L;
    }
    double v = *cp++;  // nest(-1, .): the next coefficient
    // close terms upward while depths complete
    for (;;) {
      const double term = __dmul_rn(v, pw[L]);
      s[L] = (e[L] == 0) ? term : __dadd_rn(s[L], term);
      pw[L] = __dmul_rn(pw[L], x[L]);
      if (++e[L] <= rm[L]) break;
      if (L == k) return {s[k], cp};
      v = s[L];
      ++L;
    }
  }
}

__device__ __forceinline__ double nest_rows(int k, int rem, const double*& cp, const double* x) {
  switch (k) {
    case -1: return nest_t<-1>(rem, cp, x);
    case 0: return nest_t<0>(rem, cp, x);
    case 1: return nest_t<1>(rem, cp, x);
    case 2: return nest_t<2>(rem, cp, x);
    default: {
      const NestOut o = nest_deep(k, rem, cp, x);
      cp = o.cp;
      return o.v;
    }
  }
}

// The row polynomial g_0..g_DS of a 2- or 3-port relation at one row, for a
// degree fixed at compile time: the very products and sums of nest_t, in the
// same order, with the powers of the row ports (1, x, x*x, ... by repeated
// multiplication, the same sequence nest_t forms for every sum) computed once
// instead of once per sum, and every sum unrolled, so that the sums of the
// D + 1 blocks proceed side by side rather than one FP64 chain after another.
template <int DS>
__device__ __forceinline__ void row_poly2(const double* __restrict__ cp, double x0, double* g) {
  double p0[DS + 1];
  p0[0] = 1.0;
#pragma unroll
  for (int e = 1; e <= DS; ++e) p0[e] = __dmul_rn(p0[e - 1], x0);
#pragma unroll
  for (int j = 0; j <= DS; ++j) {
    double s0 = __dmul_rn(cp[0], p0[0]);
#pragma unroll
    for (int e = 1; e <= DS - j; ++e) s0 = __dadd_rn(s0, __dmul_rn(cp[e], p0[e]));
    cp += DS - j + 1;
    g[j] = s0;
  }
}

template <int DS>
__device__ __forceinline__ void row_poly3(const double* __restrict__ cp, double x0, double x1,
                                          double* g) {
  double p0[DS + 1], p1[DS + 1];
  p0[0] = 1.0;
  p1[0] = 1.0;
#pragma unroll
  for (int e = 1; e <= DS; ++e) {
    p0[e] = __dmul_rn(p0[e - 1], x0);
    p1[e] = __dmul_rn(p1[e - 1], x1);
  }
#pragma unroll
  for (int j = 0; j <= DS; ++j) {
    double s1 = 0.0;
#pragma unroll
    for (int e1 = 0; e1 <= DS - j; ++e1) {
      double s0 = __dmul_rn(cp[0], p0[0]);
#pragma unroll
      for (int e = 1; e <= DS - j - e1; ++e) s0 = __dadd_rn(s0, __dmul_rn(cp[e], p0[e]));
      cp += DS - j - e1 + 1;
      const double term = __dmul_rn(s0, p1[e1]);
      s1 = (e1 == 0) ? term : __dadd_rn(s1, term);
    }
    g[j] = s1;
  }
}

__device__ __forceinline__ double centre(double lo, double delta, int64_t i) {
  return __dadd_rn(lo, __dmul_rn(__dadd_rn((double)i, 0.5), delta));
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
  int64_t idx[kMaxDim];
  idx[ndim - 1] = i;
  for (int a = ndim - 2; a >= 0; --a) {
    idx[a] = rest % J->res[a];
    rest /= J->res[a];
  }
  double x[kMaxDim];
  for (int p = 0; p < J->arity; ++p) x[p] = centre(J->lo[p], J->delta[p], idx[J->port_axis[p]]);
  const double* cp = J->coeffs;
  return decide64(nest_rows(J->arity - 1, J->degree, cp, x), J->kind, J->eps, J->strict);
}

// --------------------------------------------------------------- plot kernel
// One block plots a tile of rows.  Set-up: the FP32 centres of the last axis
// are staged in shared memory (padded so that consecutive words hit distinct
// banks) and each row's polynomial and thresholds are computed there.  Then
// Taylor tests decide whole spans and words first (each thread a span of
// four words, then its words); the words no test decides are listed, and the
// block evaluates them, a piece of each word per thread, in FP32
// (f = g_0 + g_1 y + ... by fused multiply-adds): |f| below eps - B_row is on,
// above eps + B_row is off, anything else is decided by the exact FP64
// evaluation.
constexpr int kPlotThreads = 256;
static_assert(sizeof(PlotJob) % 4 == 0, "plot descriptors are copied as 32-bit words");
constexpr int kYTabCap = 12288;  // largest last axis whose centres are staged in shared memory

__device__ __forceinline__ int ypad(int i) { return i + (i >> 6); }

// Byte offset of the thresholds in a plot block's shared memory (16-aligned).
__host__ __device__ __forceinline__ size_t plot_thr_offset(int rmax, int gstride) {
  return ((size_t)rmax * gstride * 12 + 15) / 16 * 16;
}

// The FP32 centre of last-axis pixel i.
__device__ __forceinline__ float ycentre32(double ylo, double ydelta, int i) {
  return __double2float_rn(centre(ylo, ydelta, i));
}

// Centre tables, one thread per centre.  The plot launch that follows may
// start as soon as every block of this one has begun.
__global__ void __launch_bounds__(256)
plot_centres_kernel(const CentreTab* __restrict__ tabs, int ntabs, int64_t total) {
  asm volatile("griddepcontrol.launch_dependents;");
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total;
       it += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = ntabs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tabs[mid].item0 <= it) lo = mid; else hi = mid - 1;
    }
    const CentreTab& T = tabs[lo];
    const int i = (int)(it - T.item0);
    T.y32[i] = ycentre32(T.lo, T.delta, i);
  }
}

void launch_plot_centres(const CentreTab* d_tabs, int ntabs, int64_t total_items, cudaStream_t s) {
  if (total_items <= 0) return;
  int64_t blocks = (total_items + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  plot_centres_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_tabs, ntabs, total_items);
}

// Clear the listed ranges with every thread of the grid, eight words per
// thread and step: chunk c covers words [8c, 8c + 8) of the ranges' flat
// index space and may cross from one range into the next.
__device__ __forceinline__ void clear_ranges(const ZeroRange* __restrict__ zr, int nzero,
                                             int64_t zero_words) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = gid; c * 8 < zero_words; c += gstride) {
    int64_t w = c * 8;
    const int64_t wend = min(zero_words, w + 8);
    int lo = 0, hi = nzero - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (zr[mid].w0 <= w) lo = mid; else hi = mid - 1;
    }
    for (int r = lo; w < wend && r < nzero; ++r) {
      const int64_t end = min(wend, zr[r].w0 + zr[r].words);
      for (; w < end; ++w) zr[r].p[w - zr[r].w0] = 0ull;
    }
  }
}

// The 64 pixels of one word in FP32: bit b of *on is set when the pixel is
// certainly on, bit b of *pending when only the FP64 evaluation can decide.
template <int DS, bool EQ, bool YS, bool FULL>
__device__ __forceinline__ void eval_word(const float* g, int D, float lo, float hi,
                                          const float* ytab_w, const float* __restrict__ y32g,
                                          int i0, int nb, uint64_t* on, uint64_t* pending) {
  uint32_t on_lo = 0, on_hi = 0, pe_lo = 0, pe_hi = 0;
#pragma unroll
  for (int bb = 0; bb < 64; ++bb) {
    if (FULL || bb < nb) {
      const float y = YS ? ytab_w[bb] : __ldg(y32g + i0 + bb);
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

template <int DS, bool EQ, bool YS>
__device__ __forceinline__ void eval_word_any(const float* g, int D, float lo, float hi,
                                              const float* ytab_w, const float* y32g, int i0,
                                              int nb, uint64_t* on, uint64_t* pending) {
  if (nb == 64) eval_word<DS, EQ, YS, true>(g, D, lo, hi, ytab_w, y32g, i0, nb, on, pending);
  else eval_word<DS, EQ, YS, false>(g, D, lo, hi, ytab_w, y32g, i0, nb, on, pending);
}

// Eight pixels of a row in FP32 (f = g_0 + g_1 y + ... by fused
// multiply-adds): bit b of the result is set when pixel b is certainly on,
// bit b of *pending when only the FP64 evaluation can decide.  nb8 pixels
// (1..8) exist; y comes from the padded shared table (YS) or global memory.
template <int DS, bool EQ, bool YS>
__device__ __forceinline__ uint32_t eval8(const float* g, int D, float lo, float hi,
                                          const float* yt, const float* __restrict__ yg, int ic,
                                          int nb8, uint32_t* pending) {
  uint32_t on = 0, pe = 0;
#pragma unroll
  for (int bb = 0; bb < 8; ++bb) {
    if (bb < nb8) {
      const float y = YS ? yt[bb] : __ldg(yg + ic + bb);
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
      on |= (uint32_t)c_on << bb;
      pe |= (uint32_t)c_pe << bb;
    }
  }
  *pending = pe;
  return on;
}

template <int DS>
__global__ void __launch_bounds__(kPlotThreads, 3)
plot_kernel(const PlotJob* __restrict__ jobs, int njobs, int ytab_cap, int gstride, int rmax,
            const ZeroRange* __restrict__ zr, int nzero, int64_t zero_words) {
  extern __shared__ __align__(16) unsigned char plot_smem[];
  asm volatile("griddepcontrol.launch_dependents;");
  // [rmax][gstride] FP64 row polynomials, [rmax][gstride] FP32 copies,
  // [rmax] thresholds, then the padded FP32 centre table
  double* g64s = reinterpret_cast<double*>(plot_smem);
  float* g32s = reinterpret_cast<float*>(g64s + (size_t)rmax * gstride);
  float4* thrs = reinterpret_cast<float4*>(plot_smem + plot_thr_offset(rmax, gstride));
  float* ytab = reinterpret_cast<float*>(thrs + rmax);
  // The block's job and a copy of its descriptor in shared memory: every
  // global read of the set-up is one round trip on the block's critical path
  // (the descriptors were just uploaded), so the jobs' first tiles are
  // compared by one thread each instead of a binary search, and the
  // descriptor's fields are read from shared memory afterwards.
  __shared__ PlotJob sJ;
  __shared__ int s_job;
  if (njobs <= (int)blockDim.x) {
    const int below = (threadIdx.x < njobs && jobs[threadIdx.x].tile0 <= (int64_t)blockIdx.x);
    const int n = __syncthreads_count(below);  // tile0 ascends from 0
    if (threadIdx.x == 0) s_job = n - 1;
  } else if (threadIdx.x == 0) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].tile0 <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_job = lo;
  }
  __syncthreads();
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(jobs + s_job);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sJ);
    for (int i = threadIdx.x; i < (int)(sizeof(PlotJob) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const PlotJob* J = &sJ;
  const int D = DS >= 0 ? DS : J->degree;
  const int row_words = (int)J->row_words;
  const int res_last = J->res[J->ndim - 1];
  const int R = J->rows_per_tile;
  const int64_t row0 = ((int64_t)blockIdx.x - J->tile0) * R;
  const int nr = (int)min((int64_t)R, J->nrows - row0);
  const bool hoisted = J->hoisted != 0;
  const bool ysmem = hoisted && res_last <= ytab_cap;
  const int arity = J->arity;
  const double ylo = J->lo[arity - 1], ydelta = J->delta[arity - 1];
  if (hoisted) {
    // set-up: per row (one thread each) the row polynomial g_0..g_D in FP64
    // (the inner nested sums of the pa.h order), its FP32 copy and the row's
    // thresholds eps -+ B_row.  (One thread per (row, j) evaluates every
    // port's centre D + 1 times: slower where the FP64 pipe is the limit, as
    // in the set-up of large 3-D plots.)
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
      int64_t rest = row0 + r;
      int64_t idx[kMaxDim];
      for (int a = J->ndim - 2; a >= 0; --a) {
        idx[a] = rest % J->res[a];
        rest /= J->res[a];
      }
      double x[kMaxDim];
      for (int p = 0; p < arity - 1; ++p)
        x[p] = centre(J->lo[p], J->delta[p], idx[J->port_axis[p]]);
      const double* cp = J->coeffs;
      const float Y = J->ymax;
      float a = 0.0f, pw = 1.0f;
      bool done = false;
      if constexpr (DS >= 0) {
        if (arity == 2 || arity == 3) {
          double gv[DS + 1];
          if (arity == 2) row_poly2<DS>(cp, x[0], gv);
          else row_poly3<DS>(cp, x[0], x[1], gv);
#pragma unroll
          for (int j = 0; j <= DS; ++j) {
            const float g1 = __double2float_rn(gv[j]);
            g64s[r * gstride + j] = gv[j];
            g32s[r * gstride + j] = g1;
            a = __fmaf_rn(fabsf(g1), pw, a);
            pw = __fmul_rn(pw, Y);
          }
          done = true;
        }
      }
      for (int j = 0; !done && j <= D; ++j) {
        const double g = nest_rows(arity - 2, D - j, cp, x);  // cp walks block j
        const float g1 = __double2float_rn(g);
        g64s[r * gstride + j] = g;
        g32s[r * gstride + j] = g1;
        a = __fmaf_rn(fabsf(g1), pw, a);
        pw = __fmul_rn(pw, Y);
      }
      float B = __fmaf_rn(a, J->kfac, J->abs_margin);
      float tlo = __fsub_rn(J->eps32, B), thi = __fadd_rn(J->eps32, B);
      if (!(a <= FLT_MAX) || !(B <= FLT_MAX)) {
        tlo = -INFINITY;  // nothing is certain: every pixel of the row takes the FP64 path
        thi = INFINITY;
        B = INFINITY;
      }
      thrs[r] = make_float4(tlo, thi, B, 0.0f);
    }
  }
  // the centre tables (and any earlier work in the stream) are complete and
  // visible past this point; nothing global is read or written before it but
  // the job descriptors and coefficients
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the later contractions' result buffers that start at zero (each block a
  // share; a block's share is small next to its plot tile)
  if (zero_words > 0) clear_ranges(zr, nzero, zero_words);
  if (hoisted) {
    if (ysmem) {
      // eight loads in flight per thread before the stores (a load-store
      // loop waits out the L2 latency once per element)
      const float* __restrict__ yg = J->y32;
      const int bs = blockDim.x;
      int i = threadIdx.x;
      for (; i + 7 * bs < res_last; i += 8 * bs) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = yg[i + k * bs];
#pragma unroll
        for (int k = 0; k < 8; ++k) ytab[ypad(i + k * bs)] = v[k];
      }
      for (; i < res_last; i += bs) ytab[ypad(i)] = yg[i];
    }
    __syncthreads();
  }
  const int kind = J->kind, strict = J->strict;
  const double eps = J->eps;
  uint64_t* __restrict__ out = J->out;
  // read once: the stores to `out` below could otherwise make the compiler
  // reload these from the job descriptor in every loop
  const float hword = J->hword;
  const float* __restrict__ y32 = J->y32;
  constexpr int kG = DS >= 0 ? DS + 1 : kMaxDeg + 1;
  const int nwords = nr * row_words;
  auto load_g = [&](int r, float* g) {
    const float* gr = g32s + r * gstride;
#pragma unroll
    for (int j = 0; j < kG; ++j) g[j] = (DS >= 0 || j <= D) ? gr[j] : 0.0f;
  };
  // Phase 1: the whole-word test on every full word (see the header); words it
  // cannot decide go to a shared list, so that phase 2 evaluates pixels with
  // every lane busy instead of a few lanes per warp.
  int* list = reinterpret_cast<int*>(ytab + (ysmem ? res_last + res_last / 64 + 1 : 0));
  __shared__ int s_n;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  // Taylor test of the pixels within h of y_c in row r: 1 when every one is
  // certainly off, 2 when every one is certainly on, 0 when undecided
  auto decide_span = [&](int r, float yc, float h) -> int {
    float g[kG];
    load_g(r, g);
    const float4 th = thrs[r];
    const float ya = fabsf(yc), yw = ya + h;
    // Horner for F and F' at y_c; S1 at |y_c| and S2 at |y_c| + h
    float fc = g[D], dc = 0.0f, s1 = 0.0f, s2 = 0.0f;
    for (int j = D - 1; j >= 0; --j) {
      dc = __fmaf_rn(dc, yc, fc);
      fc = __fmaf_rn(fc, yc, g[j]);
    }
    for (int j = D; j >= 1; --j) s1 = __fmaf_rn(s1, ya, (float)j * fabsf(g[j]));
    for (int j = D; j >= 2; --j) s2 = __fmaf_rn(s2, yw, (float)(j * (j - 1)) * fabsf(g[j]));
    const float e1 = (float)(2 * D + 4) * 5.9604645e-8f * s1;  // (2D + 4) 2^-24 S1
    const float taylor = __fmaf_rn(h, fabsf(dc) + e1, 0.5f * h * h * s2) * 1.01f;
    const float margin = __fmaf_rn(4.0f, th.z, taylor);
    if (kind == PA_EQ) return (fabsf(fc) > th.y + margin) ? 1 : 0;
    if (fc > th.y + margin) return 1;
    if (fc < th.x - margin) return 2;
    return 0;
  };
  // Spans of four full words are tested first (centre pixel 128, four times
  // the word's half-width): on a sparse plot most of them are decided at once.
  // Words of undecided spans (and of rows that are not whole spans) are
  // tested one by one; the words no test decides go to phase 2.
  const bool spans = hoisted && (row_words % 4 == 0) && (res_last == row_words * 64);
  const int S = spans ? 4 : 1;
  const int nspans = nwords / S;
  for (int base = 0; base < nspans; base += blockDim.x) {
    const int sp = base + threadIdx.x;
    int span_dec = 0;  // this lane's span decided as a whole (1 off, 2 on)
    int r = 0, w0 = 0;
    if (sp < nspans) {
      r = (sp * S) / row_words;
      w0 = sp * S - r * row_words;
      if (S == 4) {
        const int i0 = w0 * 64;
        const float yc = ysmem ? ytab[ypad(i0 + 128)] : __ldg(y32 + i0 + 128);
        span_dec = decide_span(r, yc, 4.0f * hword);
        if (span_dec) {
          uint64_t* o = out + (row0 + r) * row_words + w0;
          const uint64_t v = span_dec == 1 ? 0ull : ~0ull;
          o[0] = v;
          o[1] = v;
          o[2] = v;
          o[3] = v;
        }
      }
    }
    for (int k = 0; k < S; ++k) {
      bool keep = false;
      if (sp < nspans && !span_dec) {
        keep = true;
        const int w = w0 + k;
        const int i0 = w * 64;
        if (hoisted && res_last - i0 >= 64) {
          const float yc = ysmem ? ytab[i0 + w + 32] : __ldg(y32 + i0 + 32);
          const int dec = decide_span(r, yc, hword);
          if (dec) {
            out[(row0 + r) * row_words + w] = dec == 1 ? 0ull : ~0ull;
            keep = false;
          }
        }
      }
      // warp-aggregated append of the undecided words
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      int off = 0;
      if (lane == 0 && m) off = atomicAdd(&s_n, __popc(m));
      off = __shfl_sync(0xffffffffu, off, 0);
      if (keep) list[off + __popc(m & ((1u << lane) - 1u))] = r * row_words + w0 + k;
    }
  }
  __syncthreads();
  // Phase 2: pixel by pixel.  A block with few undecided words (a curve
  // crossing some of its rows) cuts each into C = 8 pieces of 8 pixels, one
  // per thread, so that they spread over its threads; otherwise each thread
  // takes whole words (C = 1), whose 64 pixels it evaluates with more
  // independent work in flight and one set-up per word.
  const int nlist = s_n;
  const int nthr = (int)blockDim.x;
  const int C = 4 * nlist <= nthr ? 8 : 1;
  const int PC = 64 / C;
  if (C == 1) {
    for (int e = threadIdx.x; e < nlist; e += nthr) {
      const int f = list[e];
      const int r = f / row_words, w = f - r * row_words;
      const int64_t row = row0 + r;
      const int i0 = w * 64;
      const int nb = min(64, res_last - i0);
      uint64_t word = 0;
      if (hoisted) {
        float g[kG];
        load_g(r, g);
        const float4 th = thrs[r];
        const float lo = th.x, hi = th.y;
        uint64_t pending = 0;
        const float* ytab_w = ytab + i0 + w;  // ypad(i0 + b) = i0 + w + b
        if (kind == PA_EQ) {
          if (ysmem) eval_word_any<DS, true, true>(g, D, lo, hi, ytab_w, y32, i0, nb, &word, &pending);
          else eval_word_any<DS, true, false>(g, D, lo, hi, ytab_w, y32, i0, nb, &word, &pending);
        } else {
          if (ysmem) eval_word_any<DS, false, true>(g, D, lo, hi, ytab_w, y32, i0, nb, &word, &pending);
          else eval_word_any<DS, false, false>(g, D, lo, hi, ytab_w, y32, i0, nb, &word, &pending);
        }
        while (pending) {
          const int bb = __ffsll((long long)pending) - 1;
          pending &= pending - 1;
          if (exact64(centre(ylo, ydelta, i0 + bb), g64s + r * gstride, D, kind, eps, strict))
            word |= (1ull << bb);
        }
      } else {
        for (int bb = 0; bb < nb; ++bb)
          if (general64(J, row, i0 + bb)) word |= (1ull << bb);
      }
      out[row * row_words + w] = word;
    }
  }
  for (int e = threadIdx.x; C > 1 && e < nlist * C; e += nthr) {
    const int f = list[e / C], c = e % C;
    const int r = f / row_words, w = f - r * row_words;
    const int64_t row = row0 + r;
    const int ic0 = w * 64 + PC * c;  // first pixel of the piece
    uint64_t bits = 0;
    float g[kG];
    float lo = 0.0f, hi = 0.0f;
    if (hoisted) {
      load_g(r, g);
      const float4 th = thrs[r];
      lo = th.x;
      hi = th.y;
    }
    for (int g8 = 0; g8 < PC / 8; ++g8) {
      const int ic = ic0 + 8 * g8;
      const int nb8 = min(8, res_last - ic);  // <= 0: padding past the row
      if (nb8 <= 0) break;
      uint32_t b8 = 0;
      if (hoisted) {
        uint32_t pending = 0;
        const float* yt = ytab + ic + w;  // ypad(ic + b) = ic + w + b
        if (kind == PA_EQ) {
          if (ysmem) b8 = eval8<DS, true, true>(g, D, lo, hi, yt, y32, ic, nb8, &pending);
          else b8 = eval8<DS, true, false>(g, D, lo, hi, yt, y32, ic, nb8, &pending);
        } else {
          if (ysmem) b8 = eval8<DS, false, true>(g, D, lo, hi, yt, y32, ic, nb8, &pending);
          else b8 = eval8<DS, false, false>(g, D, lo, hi, yt, y32, ic, nb8, &pending);
        }
        while (pending) {
          const int bb = __ffs(pending) - 1;
          pending &= pending - 1;
          if (exact64(centre(ylo, ydelta, ic + bb), g64s + r * gstride, D, kind, eps, strict))
            b8 |= 1u << bb;
        }
      } else {
        for (int bb = 0; bb < nb8; ++bb)
          if (general64(J, row, ic + bb)) b8 |= 1u << bb;
      }
      bits |= (uint64_t)b8 << (8 * g8);
    }
    uint64_t* ow = out + row * row_words + w;
    switch (C) {
      case 1: *ow = bits; break;
      case 2: reinterpret_cast<uint32_t*>(ow)[c] = (uint32_t)bits; break;
      case 4: reinterpret_cast<uint16_t*>(ow)[c] = (uint16_t)bits; break;
      default: reinterpret_cast<uint8_t*>(ow)[c] = (uint8_t)bits; break;
    }
  }
}

// ------------------------------------------------------- corner-rule plots
// The corner rule of pa.h (pa_rule), one thread per output byte (8 pixels of
// the last axis).  For each of the 2^(d-1) corner choices on the leading axes,
// f is evaluated at the lattice points i0 .. i0 + nb of the last axis (9 for a
// full byte); bit j of the masks n / p / q records that lattice point j passes
// the comparison / has a finite value above 0 / below 0.  Pixel b has lattice
// points b and b + 1 on the last axis, so its bit in each pixel mask is
// m | m >> 1.  Bytes past the last pixel of a row are written as 0.  Off by
// default and evaluated in plain FP64 (no FP32 filter): every corner value
// costs one full evaluation, 9/8 per pixel and leading corner choice.
__device__ __forceinline__ double lattice_point(double lo, double delta, int64_t i) {
  return __dadd_rn(lo, __dmul_rn((double)i, delta));
}

__global__ void __launch_bounds__(256)
plot_corner_kernel(const CornerJob* __restrict__ jobs, int njobs, int64_t total_bytes) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total_bytes;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = t >> 3;
    const int byte = (int)(t & 7);
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].word0 <= w) lo = mid; else hi = mid - 1;
    }
    const CornerJob& J = jobs[lo];
    const int64_t lw = w - J.word0;
    const int64_t row = lw / J.row_words;
    const int64_t wi = lw - row * J.row_words;
    const int last = J.ndim - 1;
    int64_t idx[kMaxDim];
    int64_t rest = row;
    for (int a = last - 1; a >= 0; --a) {
      idx[a] = rest % J.res[a];
      rest /= J.res[a];
    }
    const int i0 = (int)(wi * 64) + 8 * byte;
    const int nb = min(8, J.res[last] - i0);  // pixels of this byte (<= 0: padding)
    uint32_t near = 0, pos = 0, neg = 0;  // per pixel, OR over its corners
    for (int m = 0; nb > 0 && m < (1 << last); ++m) {
      double x[kMaxDim];
      for (int p = 0; p < J.arity; ++p) {
        const int a = J.port_axis[p];
        if (a != last) x[p] = lattice_point(J.lo[p], J.delta[p], idx[a] + ((m >> a) & 1));
      }
      uint32_t n = 0, pp = 0, q = 0;  // lattice points 0..nb
      for (int j = 0; j <= nb; ++j) {
        for (int p = 0; p < J.arity; ++p)
          if (J.port_axis[p] == last) x[p] = lattice_point(J.lo[p], J.delta[p], i0 + j);
        double f;
        if (J.prog) {
          f = run_expr(J.prog, J.nops, J.consts, x);
        } else {
          const double* cp = J.coeffs;
          f = nest_rows(J.arity - 1, J.degree, cp, x);
        }
        n |= (decide64(f, J.kind, J.eps, J.strict) ? 1u : 0u) << j;
        pp |= ((isfinite(f) && f > 0.0) ? 1u : 0u) << j;
        q |= ((isfinite(f) && f < 0.0) ? 1u : 0u) << j;
      }
      near |= n | (n >> 1);
      pos |= pp | (pp >> 1);
      neg |= q | (q >> 1);
    }
    uint32_t bits = near | (J.kind == PA_EQ ? (pos & neg) : 0u);
    bits = nb > 0 ? bits & ((1u << nb) - 1u) : 0u;
    reinterpret_cast<uint8_t*>(J.out + lw)[byte] = (uint8_t)bits;
  }
}

void launch_plot_corner(const CornerJob* d_jobs, int njobs, int64_t total_words, cudaStream_t s) {
  if (njobs <= 0 || total_words <= 0) return;
  const int64_t bytes = 8 * total_words;
  int64_t blocks = (bytes + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  plot_corner_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_jobs, njobs, bytes);
}

// Blocks of the plot kernel (of this degree) that the GPU holds at once:
// per SM as the occupancy calculator gives it for 256 threads and a typical
// 16 KB of shared memory (registers are the limit), times the SMs.  Cached;
// 3 x 152 when the device cannot be asked.
int plot_resident_blocks(int common_degree) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 3 * 152;
  }
  const std::pair<int, int> key(dev, common_degree);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  const void* fn;
  switch (common_degree) {
    case 1: fn = reinterpret_cast<const void*>(plot_kernel<1>); break;
    case 2: fn = reinterpret_cast<const void*>(plot_kernel<2>); break;
    case 3: fn = reinterpret_cast<const void*>(plot_kernel<3>); break;
    case 4: fn = reinterpret_cast<const void*>(plot_kernel<4>); break;
    default: fn = reinterpret_cast<const void*>(plot_kernel<-1>); break;
  }
  int sms = 0, per = 0;
  int v = 3 * 152;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kPlotThreads, 16 * 1024) ==
          cudaSuccess &&
      sms > 0 && per > 0)
    v = sms * per;
  else
    cudaGetLastError();
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = v;
  return v;
}

cudaError_t probe_kernel_image() {
  cudaFuncAttributes attr;
  return cudaFuncGetAttributes(&attr, plot_kernel<-1>);
}

void launch_plot(const PlotJob* d_jobs, int njobs, int64_t total_tiles, int max_rows_per_tile,
                 int max_degree, int common_degree, int max_res_last, int64_t max_tile_words,
                 const ZeroRange* d_zero, int nzero, int64_t zero_words, cudaStream_t s) {
  if (total_tiles <= 0) return;
  const int ycap = max_res_last <= kYTabCap ? max_res_last : 0;
  const int gstride = max_degree + 1, rmax = max_rows_per_tile;
  // thresholds, centre table, then the list of undecided words (one int per
  // word of the largest tile)
  const size_t smem = plot_thr_offset(rmax, gstride) + (size_t)rmax * 16 +
                      (size_t)(ycap + ycap / 64 + 1) * sizeof(float) +
                      (size_t)max_tile_words * sizeof(int);
  const unsigned grid = (unsigned)total_tiles;
  // programmatic dependent launch: the blocks may start while the centre
  // tables are being computed and wait for them after their row set-up
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kPlotThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
#define PA_PLOT(DD)                                                                          \
  do {                                                                                       \
    smem_limit(reinterpret_cast<const void*>(plot_kernel<DD>), smem);                        \
    cudaLaunchKernelEx(&cfg, plot_kernel<DD>, d_jobs, njobs, ycap, gstride, rmax, d_zero,    \
                       nzero, zero_words);                                                   \
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
