/*
 * Pixel-array oracle: a plain, slow, obviously correct CPU statement of what the
 * pixel array method computes (Spivak, Dobson, Kumari, Wu, "Pixel Arrays: a fast
 * and elementary method for solving nonlinear systems", arXiv 1609.00061).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header or
 * table with the CUDA library and must never be called by the product path.
 *
 * Arrays are one byte per pixel (0 or 1), row-major over the array's ports in
 * the order given, last port fastest.  Build flags: -O2 -ffp-contract=off (no
 * fused multiply-add anywhere, so every product and sum is one IEEE-754
 * round-to-nearest-even operation).
 *
 * Functions and the passages they follow:
 *   or_coeff_count / or_coeff_index   -- polynomial format (graded lex order)
 *   or_eval_poly                      -- nested evaluation of a polynomial
 *   or_valid_tolerance                -- a valid tolerance, Sec. 3.2, Eq. (continuity)
 *   or_plot                           -- sample-in-center plot, Sec. 3.2, Definition
 *                                        of the epsilon-tolerance sample-in-center plot
 *   or_eval_expr / or_plot_expr       -- expression relations (Sec. 2.1, Sec. 2.4) and
 *                                        their sample-in-center plot
 *   or_plot_corner, or_valid_tolerance_corner
 *                                     -- the corner-lattice sample rule (not the
 *                                        paper's; an optional mode) and its tolerance
 *   or_gam                            -- Algorithm 1 (generalized array multiplication)
 *   or_contract_pair                  -- Eq. (GAM) for a two-array cluster (Sec. 3.5)
 *   or_contract_count                 -- the same cluster over the counting semiring
 *                                        (Sec. 2.2, footnote on plots)
 *
 * Parity status: every function here is pinned by the tests under tests/
 * (brute force, closed forms, the Appendix A example, no-false-negative points).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_DIM 8

/* ---------------------------------------------------------------- polynomials
 * A polynomial in n variables of total degree <= D has C(n+D, D) coefficients,
 * stored in graded lexicographic order: total degree t = 0, 1, ..., D; within one
 * degree, exponent tuples (e_1, ..., e_n) in descending lexicographic order.
 * For n = 2, D = 2: 1, x1, x2, x1^2, x1 x2, x2^2.
 */
static int64_t binom(int n, int k) {
  int64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

int64_t or_coeff_count(int n, int degree) { return binom(n + degree, degree); }

static int next_tuple_desc(int n, int t, int* e) {
  /* advance e (sum t) to the next tuple in descending lex order; 0 when done */
  /* find the rightmost position i < n-1 with e[i] > 0, decrement it, and put
     the whole remainder of the sum into position i+1, zeros after */
  for (int i = n - 2; i >= 0; --i) {
    if (e[i] > 0) {
      int tail = 0;
      for (int j = i + 1; j < n; ++j) tail += e[j];
      e[i] -= 1;
      tail += 1;
      for (int j = i + 1; j < n; ++j) e[j] = 0;
      e[i + 1] = tail;
      (void)t;
      return 1;
    }
  }
  return 0;
}

/* Position of exponent tuple e in the graded lex order: count every tuple that
 * comes before it by direct enumeration. */
int64_t or_coeff_index(int n, int degree, const int* exps) {
  int64_t idx = 0;
  int tsum = 0;
  for (int i = 0; i < n; ++i) tsum += exps[i];
  if (tsum > degree) return -1;
  for (int t = 0; t <= degree; ++t) {
    int e[OR_MAX_DIM];
    memset(e, 0, sizeof e);
    e[0] = t;
    do {
      int same = (t == tsum);
      for (int i = 0; same && i < n; ++i) same = (e[i] == exps[i]);
      if (same) return idx;
      ++idx;
    } while (n > 1 && next_tuple_desc(n, t, e));
  }
  return -1;
}

/* Coefficient lookup table: tab[mixed-radix (D+1) code of e] = position of e in
 * the graded lex order, filled by direct enumeration of that order. */
static int64_t* build_index_table(int n, int degree) {
  int64_t size = 1;
  for (int i = 0; i < n; ++i) size *= (degree + 1);
  int64_t* tab = (int64_t*)malloc(sizeof(int64_t) * (size_t)size);
  for (int64_t i = 0; i < size; ++i) tab[i] = -1;
  int64_t idx = 0;
  for (int t = 0; t <= degree; ++t) {
    int e[OR_MAX_DIM];
    memset(e, 0, sizeof e);
    e[0] = t;
    do {
      int64_t code = 0;
      for (int i = 0; i < n; ++i) code = code * (degree + 1) + e[i];
      tab[code] = idx++;
    } while (n > 1 && next_tuple_desc(n, t, e));
  }
  return tab;
}

/* Nested evaluation
 *   f = sum_{e_n} ( ... ( sum_{e_1} c_e * x_1^{e_1} ) * x_2^{e_2} ... ) * x_n^{e_n}
 * with e_k running from 0 up to the degree left over by e_{k+1..n}.  Every sum
 * starts from its first term and adds the next one on the right; powers are built
 * by repeated multiplication starting from 1.0 (x^3 = (x*x)*x); the innermost
 * term is coefficient * power, every outer term is inner sum * power. */
static double nest(int k, int n, int degree, int rem, int* e, const double* coeffs,
                   const int64_t* tab, const double* x) {
  if (k < 0) {
    int64_t code = 0;
    for (int i = 0; i < n; ++i) code = code * (degree + 1) + e[i];
    return coeffs[tab[code]];
  }
  double s = 0.0, pw = 1.0;
  for (int ek = 0; ek <= rem; ++ek) {
    e[k] = ek;
    double term = nest(k - 1, n, degree, rem - ek, e, coeffs, tab, x) * pw;
    s = (ek == 0) ? term : s + term;
    pw = pw * x[k];
  }
  e[k] = 0;
  return s;
}

static double eval_with_table(int n, int degree, const double* coeffs, const int64_t* tab,
                              const double* x) {
  int e[OR_MAX_DIM];
  memset(e, 0, sizeof e);
  return nest(n - 1, n, degree, degree, e, coeffs, tab, x);
}

double or_eval_poly(int n, int degree, const double* coeffs, const double* x) {
  int64_t* tab = build_index_table(n, degree);
  double f = eval_with_table(n, degree, coeffs, tab, x);
  free(tab);
  return f;
}

/* ---------------------------------------------------------- valid tolerance
 * Sec. 3.2: epsilon is valid for f on a pack when points closer than the pixel
 * radius have values closer than epsilon (Eq. continuity).  The paper gives no
 * recipe.  For a polynomial, the mean value theorem in the l-infinity metric
 * gives |f(x) - f(c)| <= sum_p S_p * delta_p / 2 for x in the pixel centred at c,
 * where S_p bounds |df/dx_p| on the box:
 *   S_p = sum_e |c_e| * e_p * M_p^(e_p - 1) * prod_{q != p} M_q^(e_q),
 *   M_q = max(|lo_q|, |hi_q|),  delta_p = (hi_p - lo_p) / res_p.
 * The result is scaled by (1 + 2^-30) so that rounding in f(c) cannot turn a
 * pixel holding an exact solution off.  Fixed order: ports p ascending, monomials
 * in graded lex order, factors multiplied left to right as written above.
 * `width` is the fraction of delta_p that a point of the pixel can lie from the
 * sample point along port p: 1/2 for the centre, 1 for a corner (or_plot_corner). */
static double tolerance(int n, int degree, const double* coeffs, const double* lo,
                        const double* hi, const int* res, double width) {
  double M[OR_MAX_DIM];
  for (int q = 0; q < n; ++q) {
    double a = fabs(lo[q]), b = fabs(hi[q]);
    M[q] = (a > b) ? a : b;
  }
  double total = 0.0;
  for (int p = 0; p < n; ++p) {
    double Sp = 0.0;
    for (int t = 0; t <= degree; ++t) {
      int e[OR_MAX_DIM];
      memset(e, 0, sizeof e);
      e[0] = t;
      do {
        if (e[p] > 0) {
          int64_t ci = or_coeff_index(n, degree, e);
          double term = fabs(coeffs[ci]);
          term = term * (double)e[p];
          double pw = 1.0;
          for (int k = 0; k < e[p] - 1; ++k) pw = pw * M[p];
          term = term * pw;
          for (int q = 0; q < n; ++q) {
            if (q == p) continue;
            double pq = 1.0;
            for (int k = 0; k < e[q]; ++k) pq = pq * M[q];
            term = term * pq;
          }
          Sp = Sp + term;
        }
      } while (n > 1 && next_tuple_desc(n, t, e));
    }
    double delta = (hi[p] - lo[p]) / (double)res[p];
    total = total + Sp * (delta * width);
  }
  return total * (1.0 + 0x1p-30);
}

double or_valid_tolerance(int n, int degree, const double* coeffs, const double* lo,
                          const double* hi, const int* res) {
  return tolerance(n, degree, coeffs, lo, hi, res, 0.5);
}

/* The same bound for the corner-lattice plot: every point of a pixel lies within
 * delta_p of each of its corners along port p, so the full width is used. */
double or_valid_tolerance_corner(int n, int degree, const double* coeffs, const double* lo,
                                 const double* hi, const int* res) {
  return tolerance(n, degree, coeffs, lo, hi, res, 1.0);
}

/* --------------------------------------------------------------------- plot
 * Sec. 3.2, sample-in-center plot: entry e is on iff the error at the pixel
 * centre c_e achieves epsilon (Sec. 3.2, definition of the N-error set).  Pixel e covers, along port p, the
 * half-open interval [lo + delta*i, lo + delta*(i+1)) with 0-based index i
 * (Eq. Pixel_def), so the centre coordinate is lo + (i + 1/2) * delta, computed
 * as: delta = (hi - lo) / res; t = (double)i + 0.5; x = lo + t * delta.
 * With S = {0} (kind 0) the error set at c is {|f(c)|}; with S = (-inf, 0]
 * (kind 1) it reaches down to max(f(c), 0); with S = (-inf, 0) (kind 2) it is the
 * open ray above max(f(c), 0).  "Achieves epsilon" then reads
 *   kind 0: |f(c)| <= eps;  kind 1: f(c) <= eps;  kind 2: f(c) < eps.
 * strict != 0 replaces every <= by < (the Appendix A sample code uses a strict
 * test).  A value that is undefined (NaN) or infinite turns the pixel off
 * (Sec. 2.4, the butterfly example). */
static int decide(double f, int kind, double eps, int strict) {
  if (!isfinite(f)) return 0;
  if (kind == 0) {
    double d = fabs(f);
    return strict ? (d < eps) : (d <= eps);
  }
  if (kind == 1) return strict ? (f < eps) : (f <= eps);
  return f < eps;
}

int or_plot(int n, int degree, const double* coeffs, int kind, double eps, int strict,
            const double* lo, const double* hi, const int* res, uint8_t* out) {
  if (n < 1 || n > OR_MAX_DIM) return -1;
  int64_t total = 1;
  for (int p = 0; p < n; ++p) total *= res[p];
  double delta[OR_MAX_DIM];
  for (int p = 0; p < n; ++p) delta[p] = (hi[p] - lo[p]) / (double)res[p];
  int64_t* tab = build_index_table(n, degree);
#pragma omp parallel for schedule(static)
  for (int64_t flat = 0; flat < total; ++flat) {
    int64_t rest = flat;
    double x[OR_MAX_DIM];
    for (int p = n - 1; p >= 0; --p) {
      int64_t i = rest % res[p];
      rest /= res[p];
      double t = (double)i + 0.5;
      x[p] = lo[p] + t * delta[p];
    }
    double f = eval_with_table(n, degree, coeffs, tab, x);
    out[flat] = (uint8_t)decide(f, kind, eps, strict);
  }
  free(tab);
  return 0;
}

/* ------------------------------------------------------------- expressions
 * A relation given as an expression of its ports (the paper's examples in
 * Sec. 2.1 and Sec. 2.4 use |.|, cos, ln, tan, cosh, exp and reciprocals).
 * The expression is a postfix program: instruction k is op | (arg << 8) with
 * a signed arg; op 0 pushes consts[arg], op 1 pushes the coordinate of port
 * arg, ops 2..5 and 19 pop b then a and push a+b, a-b, a*b, a/b, pow(a, b);
 * ops 6..17 replace the top a by -a, |a|, sqrt, exp, ln, sin, cos, tan, sinh,
 * cosh, tanh, atan (C library); op 18 replaces a by a^arg for an integer arg:
 * a multiplied by itself |arg| - 1 times left to right, then 1 / that when
 * arg < 0, and 1 when arg = 0.
 * *mag (when mag is not NULL) receives the largest magnitude of any value
 * the program pushes: rounding differences between math libraries scale with
 * it, which is what the parity tests' tolerance at the threshold uses. */
double or_eval_expr(int nops, const int* ops, const double* consts, const double* x,
                    double* mag) {
  double st[64];
  int sp = 0;
  double m = 0.0;
  for (int k = 0; k < nops; ++k) {
    int op = ops[k] & 0xff;
    int arg = ops[k] >> 8;
    double a, b, r;
    if (op == 0) {
      r = consts[arg];
    } else if (op == 1) {
      r = x[arg];
    } else if ((op >= 2 && op <= 5) || op == 19) {
      b = st[--sp];
      a = st[--sp];
      if (op == 2) r = a + b;
      else if (op == 3) r = a - b;
      else if (op == 4) r = a * b;
      else if (op == 5) r = a / b;
      else r = pow(a, b);
    } else {
      a = st[--sp];
      switch (op) {
        case 6: r = -a; break;
        case 7: r = fabs(a); break;
        case 8: r = sqrt(a); break;
        case 9: r = exp(a); break;
        case 10: r = log(a); break;
        case 11: r = sin(a); break;
        case 12: r = cos(a); break;
        case 13: r = tan(a); break;
        case 14: r = sinh(a); break;
        case 15: r = cosh(a); break;
        case 16: r = tanh(a); break;
        case 17: r = atan(a); break;
        case 18: {
          int n = arg < 0 ? -arg : arg;
          r = 1.0;
          if (n > 0) {
            r = a;
            for (int j = 1; j < n; ++j) r = r * a;
          }
          if (arg < 0) r = 1.0 / r;
          break;
        }
        default: r = NAN; break;
      }
    }
    st[sp++] = r;
    if (fabs(r) > m || r != r) m = (r != r) ? INFINITY : fmax(m, fabs(r));
  }
  if (mag) *mag = m;
  return sp == 1 ? st[0] : NAN;
}

/* Sample-in-center plot of an expression relation over its ports (same pixel
 * centres and decision as or_plot). */
int or_plot_expr(int n, int nops, const int* ops, const double* consts, int kind, double eps,
                 int strict, const double* lo, const double* hi, const int* res, uint8_t* out) {
  if (n < 1 || n > OR_MAX_DIM || nops < 1) return -1;
  int64_t total = 1;
  for (int p = 0; p < n; ++p) total *= res[p];
  double delta[OR_MAX_DIM];
  for (int p = 0; p < n; ++p) delta[p] = (hi[p] - lo[p]) / (double)res[p];
#pragma omp parallel for schedule(static)
  for (int64_t flat = 0; flat < total; ++flat) {
    int64_t rest = flat;
    double x[OR_MAX_DIM];
    for (int p = n - 1; p >= 0; --p) {
      int64_t i = rest % res[p];
      rest /= res[p];
      double t = (double)i + 0.5;
      x[p] = lo[p] + t * delta[p];
    }
    double f = or_eval_expr(nops, ops, consts, x, NULL);
    out[flat] = (uint8_t)decide(f, kind, eps, strict);
  }
  return 0;
}

/* ---------------------------------------------------------- corner lattice
 * An alternative sample rule, off by default (the paper's rule is the centre
 * rule of or_plot): f is sampled on the lattice of grid corners.  Variable k has
 * the res_k + 1 lattice coordinates lo_k + (double)i * delta_k, i = 0..res_k,
 * delta_k = (hi_k - lo_k) / res_k (one product and one sum, each rounded), and
 * pixel e has the 2^nv corners that take index e_k or e_k + 1 on each variable.
 * Ports read variables through port_var (a variable on two ports reads one
 * coordinate on both: the corners are those of the pixel over the distinct
 * variables).  Pixel e is on iff some corner value c with finite f(c) achieves
 * eps under the same comparison as or_plot, or, for kind 0, the finite corner
 * values include one above 0 and one below 0 (f changes sign in the pixel).
 * Corners with a non-finite value take part in neither test.  With
 * eps >= or_valid_tolerance_corner every pixel holding a solution is on:
 * |f(c) - f(x)| <= sum_p S_p * delta_p for any corner c of x's pixel.
 * The relation is a polynomial (nops == 0: degree, coeffs) or an expression
 * program (nops > 0: ops, consts, as in or_eval_expr).  lo, hi, res and the
 * output axes are over the nv distinct variables, last variable fastest. */
int or_plot_corner(int nports, const int* port_var, int nv, int degree, const double* coeffs,
                   int nops, const int* ops, const double* consts, int kind, double eps,
                   int strict, const double* lo, const double* hi, const int* res,
                   uint8_t* out) {
  if (nports < 1 || nports > OR_MAX_DIM || nv < 1 || nv > OR_MAX_DIM) return -1;
  for (int p = 0; p < nports; ++p)
    if (port_var[p] < 0 || port_var[p] >= nv) return -1;
  int64_t total = 1;
  for (int k = 0; k < nv; ++k) total *= res[k];
  double delta[OR_MAX_DIM];
  for (int k = 0; k < nv; ++k) delta[k] = (hi[k] - lo[k]) / (double)res[k];
  int64_t* tab = nops > 0 ? NULL : build_index_table(nports, degree);
#pragma omp parallel for schedule(static)
  for (int64_t flat = 0; flat < total; ++flat) {
    int64_t idx[OR_MAX_DIM];
    int64_t rest = flat;
    for (int k = nv - 1; k >= 0; --k) {
      idx[k] = rest % res[k];
      rest /= res[k];
    }
    int on = 0, pos = 0, neg = 0;
    for (int m = 0; m < (1 << nv); ++m) {
      double coord[OR_MAX_DIM], x[OR_MAX_DIM];
      for (int k = 0; k < nv; ++k) {
        int64_t i = idx[k] + ((m >> k) & 1);
        coord[k] = lo[k] + (double)i * delta[k];
      }
      for (int p = 0; p < nports; ++p) x[p] = coord[port_var[p]];
      double f = nops > 0 ? or_eval_expr(nops, ops, consts, x, NULL)
                          : eval_with_table(nports, degree, coeffs, tab, x);
      if (!isfinite(f)) continue;
      if (decide(f, kind, eps, strict)) on = 1;
      if (f > 0.0) pos = 1;
      if (f < 0.0) neg = 1;
    }
    out[flat] = (uint8_t)(on || (kind == 0 && pos && neg));
  }
  free(tab);
  return 0;
}

/* ------------------------------------------------------------- Algorithm 1
 * Generalized array multiplication for a wiring diagram with links
 * Lambda = {0..nlinks-1}: for every link entry e in Entr(Lambda), the product of
 * A_i(Entr^i(e)) over the inner packs is OR-ed into A'(Entr'(e)).  Port j of
 * array i is wired to link port_links[off_i + j]; the outer pack's ports are
 * wired to out_links.  Entr^i(e) reads the link value of every port.  Loops run
 * over every entry of Entr(Lambda) exactly as the algorithm states (tiny grids). */
int or_gam(int nlinks, const int* link_res, int narr, const int* ndims,
           const int* port_links, const uint8_t* const* arrays, int nout,
           const int* out_links, uint8_t* out) {
  int64_t out_size = 1;
  for (int j = 0; j < nout; ++j) out_size *= link_res[out_links[j]];
  memset(out, 0, (size_t)out_size);
  int64_t total = 1;
  for (int l = 0; l < nlinks; ++l) total *= link_res[l];
  int e[64];
  if (nlinks > 64) return -1;
  for (int64_t flat = 0; flat < total; ++flat) {
    int64_t rest = flat;
    for (int l = nlinks - 1; l >= 0; --l) {
      e[l] = (int)(rest % link_res[l]);
      rest /= link_res[l];
    }
    uint8_t a = 1;
    int off = 0;
    for (int i = 0; i < narr; ++i) {
      int64_t idx = 0;
      for (int j = 0; j < ndims[i]; ++j) {
        int l = port_links[off + j];
        idx = idx * link_res[l] + e[l];
      }
      a = a & arrays[i][idx];
      off += ndims[i];
    }
    int64_t oidx = 0;
    for (int j = 0; j < nout; ++j) oidx = oidx * link_res[out_links[j]] + e[out_links[j]];
    out[oidx] = out[oidx] | a;
  }
  return 0;
}

/* ------------------------------------------------------- pairwise contraction
 * One node of a cluster tree with two children (Sec. 3.5): arrays X and Y over
 * variables xvars / yvars (a variable may repeat inside one array: the array is
 * then read on its diagonal), output over the distinct variables keep[].  Every
 * variable of X or Y that is not kept is summed out, so by Eq. (GAM)
 *   out(e') = OR over the values of the summed variables of X(e_X) AND Y(e_Y).
 * One loop per output entry over all values of the summed variables; it stops at
 * the first true product since OR cannot become false again.  vres[v] is the
 * resolution of variable v. */
int or_contract_pair(int nx, const int* xvars, const uint8_t* X, int ny, const int* yvars,
                     const uint8_t* Y, int nkeep, const int* keep, const int* vres,
                     uint8_t* out) {
  /* local variable list: the kept variables, then every other variable of X or Y */
  int vlist[3 * OR_MAX_DIM], nv = 0;
  for (int k = 0; k < nkeep; ++k) vlist[nv++] = keep[k];
  for (int s = 0; s < nx + ny; ++s) {
    int v = (s < nx) ? xvars[s] : yvars[s - nx];
    int seen = 0;
    for (int k = 0; k < nv; ++k) seen |= (vlist[k] == v);
    if (!seen) vlist[nv++] = v;
  }
  int nsum = nv - nkeep;
  /* stride of each local variable inside X and Y (a repeated variable adds the
     strides of all its ports, which reads the diagonal) */
  int64_t xs[3 * OR_MAX_DIM], ys[3 * OR_MAX_DIM], r[3 * OR_MAX_DIM];
  for (int k = 0; k < nv; ++k) {
    xs[k] = 0;
    ys[k] = 0;
    r[k] = vres[vlist[k]];
  }
  int64_t st = 1;
  for (int j = nx - 1; j >= 0; --j) {
    for (int k = 0; k < nv; ++k)
      if (vlist[k] == xvars[j]) xs[k] += st;
    st *= vres[xvars[j]];
  }
  st = 1;
  for (int j = ny - 1; j >= 0; --j) {
    for (int k = 0; k < nv; ++k)
      if (vlist[k] == yvars[j]) ys[k] += st;
    st *= vres[yvars[j]];
  }
  int64_t out_size = 1;
  for (int k = 0; k < nkeep; ++k) out_size *= r[k];
  int64_t sum_size = 1;
  for (int k = nkeep; k < nv; ++k) sum_size *= r[k];
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t o = 0; o < out_size; ++o) {
    int64_t rest = o, xi = 0, yi = 0;
    for (int k = nkeep - 1; k >= 0; --k) {
      int64_t v = rest % r[k];
      rest /= r[k];
      xi += xs[k] * v;
      yi += ys[k] * v;
    }
    int64_t cnt[3 * OR_MAX_DIM];
    for (int k = 0; k < nsum; ++k) cnt[k] = 0;
    uint8_t acc = 0;
    for (int64_t s = 0; s < sum_size; ++s) {
      acc = X[xi] && Y[yi];  /* Y is read only where X is on */
      if (acc) break;
      /* next value of the summed variables, last one fastest */
      for (int k = nsum - 1; k >= 0; --k) {
        int kk = nkeep + k;
        cnt[k] += 1;
        xi += xs[kk];
        yi += ys[kk];
        if (cnt[k] < r[kk]) break;
        xi -= xs[kk] * r[kk];
        yi -= ys[kk] * r[kk];
        cnt[k] = 0;
      }
    }
    out[o] = acc;
  }
  return 0;
}

/* The same cluster over the counting semiring (Sec. 2.2, footnote on plots:
 * arrays with values in the natural numbers count solutions): out(e') is the
 * sum over every value of the variables not kept of X(e_X) * Y(e_Y), each
 * product 0 or 1.  A plain loop over the kept entries and, inside, over every
 * value of the summed variables. */
int or_contract_count(int nx, const int* xvars, const uint8_t* X, int ny, const int* yvars,
                      const uint8_t* Y, int nkeep, const int* keep, const int* vres,
                      uint64_t* out) {
  int vlist[3 * OR_MAX_DIM], nv = 0;
  for (int k = 0; k < nkeep; ++k) vlist[nv++] = keep[k];
  for (int s = 0; s < nx + ny; ++s) {
    int v = (s < nx) ? xvars[s] : yvars[s - nx];
    int seen = 0;
    for (int k = 0; k < nv; ++k) seen |= (vlist[k] == v);
    if (!seen) vlist[nv++] = v;
  }
  int64_t xs[3 * OR_MAX_DIM], ys[3 * OR_MAX_DIM], r[3 * OR_MAX_DIM];
  for (int k = 0; k < nv; ++k) {
    xs[k] = 0;
    ys[k] = 0;
    r[k] = vres[vlist[k]];
  }
  int64_t st = 1;
  for (int j = nx - 1; j >= 0; --j) {
    for (int k = 0; k < nv; ++k)
      if (vlist[k] == xvars[j]) xs[k] += st;
    st *= vres[xvars[j]];
  }
  st = 1;
  for (int j = ny - 1; j >= 0; --j) {
    for (int k = 0; k < nv; ++k)
      if (vlist[k] == yvars[j]) ys[k] += st;
    st *= vres[yvars[j]];
  }
  int64_t out_size = 1;
  for (int k = 0; k < nkeep; ++k) out_size *= r[k];
  int64_t sum_size = 1;
  for (int k = nkeep; k < nv; ++k) sum_size *= r[k];
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t o = 0; o < out_size; ++o) {
    int64_t rest = o, base_x = 0, base_y = 0;
    for (int k = nkeep - 1; k >= 0; --k) {
      int64_t v = rest % r[k];
      rest /= r[k];
      base_x += xs[k] * v;
      base_y += ys[k] * v;
    }
    uint64_t total = 0;
    for (int64_t s = 0; s < sum_size; ++s) {
      /* decode s into the summed variables' values, last one fastest */
      int64_t rs = s, xi = base_x, yi = base_y;
      for (int k = nv - 1; k >= nkeep; --k) {
        int64_t v = rs % r[k];
        rs /= r[k];
        xi += xs[k] * v;
        yi += ys[k] * v;
      }
      total += (uint64_t)X[xi] * (uint64_t)Y[yi];
    }
    out[o] = total;
  }
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads the loops above may use from now on (timing the oracle on one core
 * and on all of them). */
void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
