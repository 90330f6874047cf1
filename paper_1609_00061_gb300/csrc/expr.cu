// Plots of expression relations (Sec. 3.2, sample-in-center plot, for
// relations built from the ports with arithmetic and elementary functions,
// as in the examples of Sec. 2.1 and Sec. 2.4).
//
// One thread per output word: the 64 pixels of the word are evaluated one
// after the other, each by running the relation's postfix program over a
// small stack in FP64.  The pixel centre is computed as for polynomial
// relations, lo + ((double)i + 0.5) * delta with two IEEE roundings.
#include <math.h>

#include "pa_internal.h"

namespace pa {
namespace {

__device__ __forceinline__ double expr_centre(double lo, double delta, int64_t i) {
  return __dadd_rn(lo, __dmul_rn(__dadd_rn((double)i, 0.5), delta));
}

// f at one point; NaN when the program misbehaves (it was checked on the host)
__device__ double run_expr(const int32_t* __restrict__ prog, int nops,
                           const double* __restrict__ consts, const double* x) {
  double st[PA_EXPR_MAX_STACK];
  int sp = 0;
  for (int k = 0; k < nops; ++k) {
    const int32_t ins = __ldg(prog + k);
    const int op = ins & 0xff;
    const int arg = ins >> 8;
    if (op == PA_X_CONST) {
      st[sp++] = __ldg(consts + arg);
      continue;
    }
    if (op == PA_X_VAR) {
      st[sp++] = x[arg];
      continue;
    }
    if (op >= PA_X_ADD && op <= PA_X_DIV) {
      const double b = st[--sp], a = st[sp - 1];
      double r;
      switch (op) {
        case PA_X_ADD: r = __dadd_rn(a, b); break;
        case PA_X_SUB: r = __dsub_rn(a, b); break;
        case PA_X_MUL: r = __dmul_rn(a, b); break;
        default: r = __ddiv_rn(a, b); break;
      }
      st[sp - 1] = r;
      continue;
    }
    if (op == PA_X_POW) {
      const double b = st[--sp];
      st[sp - 1] = pow(st[sp - 1], b);
      continue;
    }
    const double a = st[sp - 1];
    double r;
    switch (op) {
      case PA_X_NEG: r = -a; break;
      case PA_X_ABS: r = fabs(a); break;
      case PA_X_SQRT: r = __dsqrt_rn(a); break;
      case PA_X_EXP: r = exp(a); break;
      case PA_X_LOG: r = log(a); break;
      case PA_X_SIN: r = sin(a); break;
      case PA_X_COS: r = cos(a); break;
      case PA_X_TAN: r = tan(a); break;
      case PA_X_SINH: r = sinh(a); break;
      case PA_X_COSH: r = cosh(a); break;
      case PA_X_TANH: r = tanh(a); break;
      case PA_X_ATAN: r = atan(a); break;
      case PA_X_POWI: {
        const int n = arg < 0 ? -arg : arg;
        r = 1.0;
        if (n > 0) {
          r = a;
          for (int j = 1; j < n; ++j) r = __dmul_rn(r, a);
        }
        if (arg < 0) r = __ddiv_rn(1.0, r);
        break;
      }
      default: r = __longlong_as_double(0x7ff8000000000000ll); break;
    }
    st[sp - 1] = r;
  }
  return sp == 1 ? st[0] : __longlong_as_double(0x7ff8000000000000ll);
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
