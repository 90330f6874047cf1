// Plots of expression relations (Sec. 3.2, sample-in-center plot, for
// relations built from the ports with arithmetic and elementary functions,
// as in the examples of Sec. 2.1 and Sec. 2.4).
//
// One thread per output word: the 64 pixels of the word are evaluated one
// after the other, each by running the relation's postfix program over a
// small stack in FP64.  The pixel centre is computed as for polynomial
// relations, lo + ((double)i + 0.5) * delta with two IEEE roundings.
#include <math.h>

#include "expr_eval.cuh"
#include "pa_internal.h"

namespace pa {
namespace {

__device__ __forceinline__ double expr_centre(double lo, double delta, int64_t i) {
  return __dadd_rn(lo, __dmul_rn(__dadd_rn((double)i, 0.5), delta));
}

__global__ void __launch_bounds__(256)
plot_expr_kernel(const ExprJob* __restrict__ jobs, int njobs, int64_t total_words) {
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total_words;
       w += (int64_t)gridDim.x * blockDim.x) {
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
    const int i0 = (int)(wi * 64);
    const int nb = min(64, res_last - i0);
    double x[kMaxDim];
    for (int p = 0; p < J.arity; ++p)
      if (J.port_axis[p] != J.ndim - 1) x[p] = expr_centre(J.lo[p], J.delta[p], idx[J.port_axis[p]]);
    uint64_t word = 0;
    for (int b = 0; b < nb; ++b) {
      for (int p = 0; p < J.arity; ++p)
        if (J.port_axis[p] == J.ndim - 1) x[p] = expr_centre(J.lo[p], J.delta[p], i0 + b);
      const double f = run_expr(J.prog, J.nops, J.consts, x);
      bool on = false;
      if (isfinite(f)) {
        const double d = (J.kind == PA_EQ) ? fabs(f) : f;
        on = (J.strict || J.kind == PA_LT) ? (d < J.eps) : (d <= J.eps);
      }
      if (on) word |= 1ull << b;
    }
    J.out[lw] = word;
  }
}

}  // namespace

void launch_plot_expr(const ExprJob* d_jobs, int njobs, int64_t total_words, cudaStream_t s) {
  if (njobs <= 0 || total_words <= 0) return;
  int64_t blocks = (total_words + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  plot_expr_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_jobs, njobs, total_words);
}

}  // namespace pa
