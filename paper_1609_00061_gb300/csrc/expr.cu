// Plots of expression relations (Sec. 3.2, sample-in-center plot, for
// relations built from the ports with arithmetic and elementary functions,
// as in the examples of Sec. 2.1 and Sec. 2.4).
//
// One thread per pixel, each running the relation's postfix program over a
// small stack in FP64; a warp covers half an output word.  The pixel centre is
// computed as for polynomial relations, lo + ((double)i + 0.5) * delta with
// two IEEE roundings.  (With one thread per 64-pixel word, the paper's
// examples at 125 x 125 pixels gave a few hundred threads, and the FP64
// elementary functions ran one pixel after another on a few SMs.)
#include <math.h>

#include "expr_eval.cuh"
#include "pa_internal.h"

namespace pa {
namespace {

__device__ __forceinline__ double expr_centre(double lo, double delta, int64_t i) {
  return __dadd_rn(lo, __dmul_rn(__dadd_rn((double)i, 0.5), delta));
}

// One warp per 32-pixel half of an output word, one lane per pixel; the
// ballot of the lanes' decisions is the half's 32 bits, stored as one 32-bit
// word (the low half of a little-endian uint64 holds pixels 0..31).  Every
// lane of a warp runs the same program, so the lanes stay converged.
__global__ void __launch_bounds__(256)
plot_expr_kernel(const ExprJob* __restrict__ jobs, int njobs, int64_t total_halves) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t hw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
       hw < total_halves; hw += nwarps) {
    const int64_t w = hw >> 1;
    const int half = (int)(hw & 1);
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (jobs[mid].word0 <= w) lo = mid; else hi = mid - 1;
    }
    const ExprJob& J = jobs[lo];
    const int64_t lw = w - J.word0;
    const int64_t row = lw / J.row_words;
    const int64_t wi = lw - row * J.row_words;
    int64_t idx[kMaxDim];
    int64_t rest = row;
    for (int a = J.ndim - 2; a >= 0; --a) {
      idx[a] = rest % J.res[a];
      rest /= J.res[a];
    }
    const int res_last = J.res[J.ndim - 1];
    const int b = half * 32 + lane;             // bit of the word
    const int i = (int)(wi * 64) + b;            // pixel on the last axis
    bool on = false;
    if (i < res_last) {
      double x[kMaxDim];
      for (int p = 0; p < J.arity; ++p) {
        const int a = J.port_axis[p];
        x[p] = expr_centre(J.lo[p], J.delta[p], a == J.ndim - 1 ? (int64_t)i : idx[a]);
      }
      const double f = run_expr(J.prog, J.nops, J.consts, x);
      if (isfinite(f)) {
        const double d = (J.kind == PA_EQ) ? fabs(f) : f;
        on = (J.strict || J.kind == PA_LT) ? (d < J.eps) : (d <= J.eps);
      }
    }
    const uint32_t bits = __ballot_sync(0xffffffffu, on);
    if (lane == 0) reinterpret_cast<uint32_t*>(J.out + lw)[half] = bits;
  }
}

}  // namespace

void launch_plot_expr(const ExprJob* d_jobs, int njobs, int64_t total_words, cudaStream_t s) {
  if (njobs <= 0 || total_words <= 0) return;
  const int64_t halves = 2 * total_words;
  int64_t blocks = (halves + 7) / 8;  // 8 warps per block
  if (blocks > 152 * 16) blocks = 152 * 16;
  plot_expr_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_jobs, njobs, halves);
}

}  // namespace pa
