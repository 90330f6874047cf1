// The device interpreter of expression relations (pa.h, pa_expr): one
// program run over a small stack of doubles at one point.  Included by the
// kernels that plot expression relations (each translation unit keeps its own
// copy).
#ifndef PA_EXPR_EVAL_CUH_
#define PA_EXPR_EVAL_CUH_

#include <math.h>
#include <stdint.h>

#include "../../include/pa.h"

namespace pa {
namespace {

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

}  // namespace
}  // namespace pa

#endif  // PA_EXPR_EVAL_CUH_
