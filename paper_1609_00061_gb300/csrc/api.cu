// C interface of the pixel array engine (include/pa.h): argument checks, the
// context and its workspace, and the executor that turns a join plan into
// kernel launches.
//
// The executor runs every call twice: a sizing pass that only adds up the
// workspace it needs (no CUDA calls), then the real pass.  All work of a call is
// stream-ordered on the caller's stream, so workspace regions are never read
// after the call's last kernel.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pa_internal.h"
#include "planner.h"

struct pa_ctx {
  int device = 0;
  size_t cap = 0;
  char* arena = nullptr;
  size_t arena_size = 0;
  char* h_stage = nullptr;  // pinned staging for descriptor uploads
  size_t h_stage_size = 0;
  cudaEvent_t stage_done = nullptr;
  bool stage_pending = false;
  std::string err;
  // kernel timing (pa_profile_enable)
  int* d_err = nullptr;  // device error word written by bounded waits
  unsigned long long* d_stat = nullptr;  // words OR-ed by contractions (timing mode)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec {
    std::string name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  size_t ev_used = 0;
};

namespace pa {
namespace {

constexpr size_t kAlign = 256;

struct Fail {
  pa_status st;
};

pa_status set_err(pa_ctx* ctx, pa_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

#define PA_CHECK_ARG(cond, msg) \
  do {                          \
    if (!(cond)) throw Fail{set_err(ctx, PA_ERR_INVALID_ARG, msg)}; \
  } while (0)

// ------------------------------------------------------------ executor
struct Exec {
  pa_ctx* ctx;
  cudaStream_t s;
  bool dry;
  size_t used = 0;
  pa_stats st{};

  Exec(pa_ctx* c, cudaStream_t st_, bool dry_) : ctx(c), s(st_), dry(dry_) {}

  void* alloc(size_t bytes) {
    const size_t off = (used + kAlign - 1) / kAlign * kAlign;
    used = off + std::max<size_t>(bytes, 8);
    if (dry) return reinterpret_cast<void*>(static_cast<uintptr_t>(kAlign + off));
    return ctx->arena + off;
  }
  uint64_t* alloc_words(int64_t n) { return static_cast<uint64_t*>(alloc((size_t)n * 8)); }

  void check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
      throw Fail{set_err(ctx, PA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e))};
    }
  }
  cudaEvent_t next_event() {
    if (ctx->ev_used == ctx->ev_pool.size()) {
      cudaEvent_t e;
      check(cudaEventCreate(&e), "cudaEventCreate");
      ctx->ev_pool.push_back(e);
    }
    return ctx->ev_pool[ctx->ev_used++];
  }
  // bracket the next launch with events when timing is on
  void before(const char* what) {
    if (dry || !ctx->prof) return;
    pa_ctx::Rec r;
    r.name = what;
    r.a = next_event();
    r.b = next_event();
    check(cudaEventRecord(r.a, s), "cudaEventRecord");
    ctx->recs.push_back(r);
  }
  void launched(const char* what) {
    st.n_launches++;
    if (dry) return;
    check(cudaGetLastError(), what);
    if (ctx->prof && !ctx->recs.empty()) check(cudaEventRecord(ctx->recs.back().b, s), "cudaEventRecord");
  }
  void memset0(uint64_t* p, int64_t words) {
    if (words <= 0) return;
    before("memset");
    if (!dry) check(cudaMemsetAsync(p, 0, (size_t)words * 8, s), "cudaMemsetAsync");
    launched("memset");
  }
  // Copy a host blob to a fresh workspace region through the pinned stage.
  void* upload(const std::vector<char>& blob) {
    void* d = alloc(blob.size());
    if (dry || blob.empty()) return d;
    if (ctx->stage_pending) {
      check(cudaEventSynchronize(ctx->stage_done), "cudaEventSynchronize");
      ctx->stage_pending = false;
    }
    if (ctx->h_stage_size < blob.size()) {
      if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
      ctx->h_stage = nullptr;
      ctx->h_stage_size = 0;
      size_t sz = std::max<size_t>(blob.size(), 1 << 16);
      check(cudaMallocHost(reinterpret_cast<void**>(&ctx->h_stage), sz), "cudaMallocHost");
      ctx->h_stage_size = sz;
    }
    memcpy(ctx->h_stage, blob.data(), blob.size());
    check(cudaMemcpyAsync(d, ctx->h_stage, blob.size(), cudaMemcpyHostToDevice, s),
          "cudaMemcpyAsync");
    check(cudaEventRecord(ctx->stage_done, s), "cudaEventRecord");
    ctx->stage_pending = true;
    return d;
  }
};

template <class T>
size_t blob_put(std::vector<char>& blob, const T* data, size_t n) {
  size_t off = (blob.size() + 15) / 16 * 16;
  blob.resize(off + sizeof(T) * n);
  if (n) memcpy(blob.data() + off, data, sizeof(T) * n);
  return off;
}

// ------------------------------------------------------------ bit arrays
BitArr from_pa(const pa_array& a) {
  BitArr b;
  b.w = a.words;
  b.ndim = a.ndim;
  b.inner = a.ndim > 0 ? 1 : 0;
  for (int i = 0; i < a.ndim; ++i) {
    b.vars[i] = a.vars[i];
    b.res[i] = a.res[i];
  }
  return b;
}

int axis_of(const BitArr& a, int v) {
  for (int i = 0; i < a.ndim; ++i)
    if (a.vars[i] == v) return i;
  return -1;
}

// Same bits at the same word positions?
bool same_layout(const BitArr& x, const BitArr& y) {
  if (x.ndim != y.ndim) return false;
  for (int i = 0; i < x.ndim; ++i)
    if (x.vars[i] != y.vars[i] || x.res[i] != y.res[i]) return false;
  if (x.inner == y.inner) return true;
  const BitArr& small = (x.inner < y.inner) ? x : y;
  return small.inner >= 1 && small.rowlen() % 64 == 0;
}

// out <- in with axes matched by variable; input axes missing from out are
// OR-reduced, output axes missing from in are broadcast.
void reshape(Exec& ex, const BitArr& in, const BitArr& out) {
  ReshapeDesc d;
  memset(&d, 0, sizeof d);
  d.in = in.w;
  d.out = out.w;
  d.out_nrows = out.nrows();
  d.out_row_words = out.row_words();
  d.out_rowlen = out.rowlen();
  d.out_ndim = out.ndim;
  d.out_inner = out.inner;
  d.in_row_words = in.row_words();
  const int in_outer = in.ndim - in.inner;
  auto strides = [&](int ia, int64_t& rs, int64_t& cs) {
    rs = 0;
    cs = 0;
    if (ia < in_outer) {
      rs = 1;
      for (int b = ia + 1; b < in_outer; ++b) rs *= in.res[b];
    } else {
      cs = 1;
      for (int b = ia + 1; b < in.ndim; ++b) cs *= in.res[b];
    }
  };
  for (int a = 0; a < out.ndim; ++a) {
    d.out_res[a] = out.res[a];
    const int ia = axis_of(in, out.vars[a]);
    if (ia >= 0) strides(ia, d.row_stride[a], d.col_stride[a]);
  }
  for (int ia = 0; ia < in.ndim; ++ia) {
    if (axis_of(out, in.vars[ia]) >= 0) continue;
    const int q = d.nred++;
    d.red_res[q] = in.res[ia];
    strides(ia, d.red_row_stride[q], d.red_col_stride[q]);
  }
  // word mode: identical inner axes, nothing reduced or broadcast inside a row
  bool wm = (out.inner == in.inner) && out.inner > 0;
  for (int j = 0; wm && j < out.inner; ++j) {
    const int oa = out.ndim - out.inner + j, ia = in.ndim - in.inner + j;
    wm = (out.vars[oa] == in.vars[ia]) && (out.res[oa] == in.res[ia]);
  }
  for (int q = 0; wm && q < d.nred; ++q) wm = (d.red_col_stride[q] == 0);
  d.word_mode = wm ? 1 : 0;
  ex.st.n_reshapes++;
  ex.before("reshape_kernel");
  if (!ex.dry) launch_reshape(d, ex.s);
  ex.launched("reshape_kernel");
}

// Bring `x` into layout `want` (vars/res/inner of want; want.w ignored).  Returns
// x itself when the layouts already agree.
BitArr conform(Exec& ex, const BitArr& x, BitArr want) {
  if (same_layout(x, want)) {
    want.w = x.w;
    return want;
  }
  want.w = ex.alloc_words(want.words());
  reshape(ex, x, want);
  return want;
}

BitArr make_arr(const std::vector<int>& vars, const std::vector<int64_t>& vres, int inner) {
  BitArr a;
  a.ndim = (int)vars.size();
  a.inner = inner;
  for (int i = 0; i < a.ndim; ++i) {
    a.vars[i] = vars[i];
    a.res[i] = vres[vars[i]];
  }
  return a;
}

bool has(const std::vector<int>& v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); }

// One two-array cluster (Eq. GAM on X and Y, outer pack `keep`).  When `target`
// is given (non-null words) and the result lands in its layout, the result is
// written there directly.
// Contractions prepared by join() and launched together by flush_rowor().
struct PendingRowOr {
  std::vector<RowOrDesc> d;
};

void flush_rowor(Exec& ex, PendingRowOr& pend) {
  // one launch per tile width, at most kRowOrMaxBatch contractions each
  std::vector<int> done(pend.d.size(), 0);
  for (size_t i = 0; i < pend.d.size(); ++i) {
    if (done[i]) continue;
    std::vector<RowOrDesc> group;
    for (size_t j = i; j < pend.d.size() && (int)group.size() < kRowOrMaxBatch; ++j)
      if (!done[j] && pend.d[j].Nt == pend.d[i].Nt) {
        group.push_back(pend.d[j]);
        done[j] = 1;
      }
    ex.before("rowor_kernel");
    if (!ex.dry) ex.check(launch_rowor(group.data(), (int)group.size(), ex.s), "rowor_kernel");
    ex.launched("rowor_kernel");
  }
  pend.d.clear();
}

BitArr join(Exec& ex, const BitArr& X, const BitArr& Y, const std::vector<int>& keep,
            const std::vector<int64_t>& vres, const BitArr* target,
            PendingRowOr* pend = nullptr, int64_t target_ctas = 152) {
  std::vector<int> xv(X.vars, X.vars + X.ndim), yv(Y.vars, Y.vars + Y.ndim);
  double cost = 1.0;
  {
    std::vector<int> u = xv;
    for (int v : yv)
      if (!has(u, v)) u.push_back(v);
    for (int v : u) cost *= (double)vres[v];
  }
  ex.st.pixel_ops_dense += cost;
  ex.st.n_joins++;

  auto classify = [&](const std::vector<int>& av, const std::vector<int>& bv,
                      std::vector<int>& batch, std::vector<int>& M, std::vector<int>& K,
                      std::vector<int>& N) {
    batch.clear(); M.clear(); K.clear(); N.clear();
    for (int v : av) {
      const bool inb = has(bv, v), kept = has(keep, v);
      if (inb && kept) batch.push_back(v);
      else if (!inb && kept) M.push_back(v);
      else if (inb && !kept) K.push_back(v);
    }
    for (int v : bv)
      if (!has(av, v) && has(keep, v)) N.push_back(v);
  };

  std::vector<int> batch, M, K, N;
  classify(xv, yv, batch, M, K, N);

  // Hadamard: every kept variable is in both arrays and nothing is summed
  // between them (only private variables are reduced)
  if (K.empty() && M.empty() && N.empty()) {
    bool use_target = target && target->w && target->ndim == (int)keep.size();
    for (int i = 0; use_target && i < target->ndim; ++i) use_target = has(keep, target->vars[i]);
    BitArr want = use_target ? *target : make_arr(keep, vres, keep.empty() ? 0 : 1);
    BitArr xa = conform(ex, X, make_arr(std::vector<int>(want.vars, want.vars + want.ndim), vres, want.inner));
    BitArr ya = conform(ex, Y, make_arr(std::vector<int>(want.vars, want.vars + want.ndim), vres, want.inner));
    BitArr out = want;
    if (!out.w) out.w = ex.alloc_words(out.words());
    ex.before("and_kernel");
    if (!ex.dry) launch_and(xa.w, ya.w, out.w, out.words(), ex.s);
    ex.launched("and_kernel");
    return out;
  }

  // choose which side is A (rows) and which is B (packed columns): the one with
  // fewer reshaped bits, then the wider packed side as B
  struct Choice {
    bool swap;
    std::vector<int> batch, M, K, N;
    double reshape_bits;
    double nbits;
  };
  auto evaluate = [&](bool swap) {
    Choice c;
    c.swap = swap;
    const BitArr& A = swap ? Y : X;
    const BitArr& B = swap ? X : Y;
    std::vector<int> av(A.vars, A.vars + A.ndim), bv(B.vars, B.vars + B.ndim);
    classify(av, bv, c.batch, c.M, c.K, c.N);
    std::vector<int> a_axes = c.batch, b_axes = c.batch, c_axes = c.batch;
    a_axes.insert(a_axes.end(), c.M.begin(), c.M.end());
    a_axes.insert(a_axes.end(), c.K.begin(), c.K.end());
    b_axes.insert(b_axes.end(), c.K.begin(), c.K.end());
    b_axes.insert(b_axes.end(), c.N.begin(), c.N.end());
    c_axes.insert(c_axes.end(), c.M.begin(), c.M.end());
    c_axes.insert(c_axes.end(), c.N.begin(), c.N.end());
    c.reshape_bits = 0;
    BitArr wa = make_arr(a_axes, vres, (int)c.K.size());
    BitArr wb = make_arr(b_axes, vres, (int)c.N.size());
    if (!same_layout(A, wa)) c.reshape_bits += (double)A.bits();
    if (!same_layout(B, wb)) c.reshape_bits += (double)B.bits();
    double nb = 1;
    for (int v : c.N) nb *= (double)vres[v];
    c.nbits = nb;
    return c;
  };
  Choice c0 = evaluate(false), c1 = evaluate(true);
  const Choice& ch = (c1.reshape_bits < c0.reshape_bits ||
                      (c1.reshape_bits == c0.reshape_bits && c1.nbits > c0.nbits)) ? c1 : c0;
  const BitArr& A = ch.swap ? Y : X;
  const BitArr& B = ch.swap ? X : Y;
  std::vector<int> a_axes = ch.batch, b_axes = ch.batch, c_axes = ch.batch;
  a_axes.insert(a_axes.end(), ch.M.begin(), ch.M.end());
  a_axes.insert(a_axes.end(), ch.K.begin(), ch.K.end());
  b_axes.insert(b_axes.end(), ch.K.begin(), ch.K.end());
  b_axes.insert(b_axes.end(), ch.N.begin(), ch.N.end());
  c_axes.insert(c_axes.end(), ch.M.begin(), ch.M.end());
  c_axes.insert(c_axes.end(), ch.N.begin(), ch.N.end());
  BitArr Am = conform(ex, A, make_arr(a_axes, vres, (int)ch.K.size()));
  BitArr Bm = conform(ex, B, make_arr(b_axes, vres, (int)ch.N.size()));
  BitArr C = make_arr(c_axes, vres, (int)ch.N.size());
  if (target && target->w && same_layout(C, *target)) C.w = target->w;
  else C.w = ex.alloc_words(C.words());

  RowOrDesc d;
  memset(&d, 0, sizeof d);
  d.A = Am.w;
  d.B = Bm.w;
  d.C = C.w;
  d.nbatch = 1;
  for (int v : ch.batch) d.nbatch *= vres[v];
  d.M = 1;
  for (int v : ch.M) d.M *= vres[v];
  d.K = 1;
  for (int v : ch.K) d.K *= vres[v];
  d.Nw = Bm.row_words();
  d.a_row_words = Am.row_words();
  d.err = ex.ctx->d_err;
  d.stat = ex.ctx->prof ? ex.ctx->d_stat : nullptr;
  rowor_plan(d, target_ctas);
  if (d.atomic) ex.memset0(C.w, C.words());
  if (pend) {
    pend->d.push_back(d);
  } else {
    PendingRowOr one;
    one.d.push_back(d);
    flush_rowor(ex, one);
  }
  ex.st.peak_words = std::max<int64_t>(ex.st.peak_words, C.words());
  return C;
}

// ------------------------------------------------------------ validation
void check_axes(pa_ctx* ctx, int32_t nvars, const pa_axis* axes) {
  PA_CHECK_ARG(nvars >= 0 && (nvars == 0 || axes), "axes: null pointer or negative nvars");
  for (int v = 0; v < nvars; ++v) {
    PA_CHECK_ARG(axes[v].res >= 2, "axis resolution must be >= 2");
    PA_CHECK_ARG(isfinite(axes[v].lo) && isfinite(axes[v].hi) && axes[v].lo < axes[v].hi,
                 "axis range must be finite with lo < hi");
  }
}

void check_relation(pa_ctx* ctx, const pa_relation& r, int32_t nvars) {
  PA_CHECK_ARG(r.arity >= 1 && r.arity <= PA_MAX_DIM, "relation arity must be in 1..8");
  PA_CHECK_ARG(r.degree >= 0 && r.degree <= PA_MAX_DEGREE, "relation degree must be in 0..16");
  PA_CHECK_ARG(r.coeffs != nullptr, "relation coefficients: null pointer");
  PA_CHECK_ARG(r.kind == PA_EQ || r.kind == PA_LE || r.kind == PA_LT, "relation kind");
  PA_CHECK_ARG(!isnan(r.eps) && r.eps < INFINITY, "relation eps must be a number");
  for (int p = 0; p < r.arity; ++p)
    PA_CHECK_ARG(r.vars[p] >= 0 && r.vars[p] < nvars, "relation variable out of range");
  const int64_t nc = coeff_count(r.arity, r.degree);
  for (int64_t i = 0; i < nc; ++i)
    PA_CHECK_ARG(isfinite(r.coeffs[i]), "relation coefficients must be finite");
}

std::vector<int> distinct_vars(const pa_relation& r) {
  std::vector<int> d;
  for (int p = 0; p < r.arity; ++p)
    if (!has(d, r.vars[p])) d.push_back(r.vars[p]);
  return d;
}

double relation_eps(const pa_relation& r, const pa_axis* axes) {
  if (r.eps >= 0) return r.eps;
  double lo[kMaxDim], hi[kMaxDim];
  int32_t res[kMaxDim];
  for (int p = 0; p < r.arity; ++p) {
    lo[p] = axes[r.vars[p]].lo;
    hi[p] = axes[r.vars[p]].hi;
    res[p] = axes[r.vars[p]].res;
  }
  return valid_tolerance(r.arity, r.degree, r.coeffs, lo, hi, res);
}

void check_array(pa_ctx* ctx, const pa_array* a, const char* name) {
  PA_CHECK_ARG(a != nullptr, std::string(name) + ": null pointer");
  PA_CHECK_ARG(a->words != nullptr, std::string(name) + ": null words");
  PA_CHECK_ARG(a->ndim >= 0 && a->ndim <= PA_MAX_DIM, std::string(name) + ": ndim in 0..8");
  for (int i = 0; i < a->ndim; ++i) {
    PA_CHECK_ARG(a->res[i] >= 1, std::string(name) + ": res >= 1");
    for (int j = 0; j < i; ++j)
      PA_CHECK_ARG(a->vars[i] != a->vars[j], std::string(name) + ": repeated variable");
  }
}

// ------------------------------------------------------------ plotting
// Plot all relations into fresh workspace arrays (or into `direct_out`, when
// given, for a single relation): one preparation launch (row polynomials,
// thresholds, FP32 centre tables) and one plot launch for all of them.
std::vector<BitArr> plot_all(Exec& ex, int32_t nvars, const pa_axis* axes, int32_t nrel,
                             const pa_relation* rels, int strict, const BitArr* direct_out) {
  (void)nvars;
  std::vector<BitArr> plots;
  std::vector<PlotJob> jobs(nrel);
  std::vector<char> blob;
  std::vector<size_t> coeff_off(nrel);
  int64_t tiles = 0, prep_items = 0;
  int max_rows = 1, max_deg = 0, common_deg = rels[0].degree, max_res_last = 1;
  for (int i = 0; i < nrel; ++i) {
    const pa_relation& r = rels[i];
    std::vector<int> dv = distinct_vars(r);
    BitArr a;
    a.ndim = (int)dv.size();
    a.inner = 1;
    for (int k = 0; k < a.ndim; ++k) {
      a.vars[k] = dv[k];
      a.res[k] = axes[dv[k]].res;
    }
    a.w = direct_out ? direct_out->w : ex.alloc_words(a.words());
    plots.push_back(a);
    // coefficients in nest order
    std::vector<int64_t> ord = nest_order(r.arity, r.degree);
    std::vector<double> nc(ord.size());
    for (size_t k = 0; k < ord.size(); ++k) nc[k] = r.coeffs[ord[k]];
    coeff_off[i] = blob_put(blob, nc.data(), nc.size());

    PlotJob& J = jobs[i];
    memset(&J, 0, sizeof J);
    J.out = a.w;
    J.arity = r.arity;
    J.degree = r.degree;
    J.kind = r.kind;
    J.strict = strict;
    J.ndim = a.ndim;
    for (int k = 0; k < a.ndim; ++k) J.res[k] = (int32_t)a.res[k];
    for (int p = 0; p < r.arity; ++p) {
      const pa_axis& ax = axes[r.vars[p]];
      J.port_axis[p] = axis_of(a, r.vars[p]);
      J.lo[p] = ax.lo;
      J.delta[p] = (ax.hi - ax.lo) / (double)ax.res;
    }
    J.hoisted = (a.ndim == r.arity) ? 1 : 0;
    J.nrows = a.nrows();
    J.row_words = a.row_words();
    const int64_t res_last = a.res[a.ndim - 1];
    const int D1 = r.degree + 1;
    if (J.hoisted) {
      J.g64 = static_cast<double*>(ex.alloc((size_t)J.nrows * D1 * 8));
      J.g32 = static_cast<float*>(ex.alloc((size_t)J.nrows * D1 * 4));
      J.thr = static_cast<float*>(ex.alloc((size_t)J.nrows * 2 * 4));
      J.y32 = static_cast<float*>(ex.alloc((size_t)res_last * 4));
      J.prep0 = prep_items;
      prep_items += J.nrows + res_last;
    }
    {
      const pa_axis& ax = axes[r.vars[r.arity - 1]];
      J.ymax = (float)(fmax(fabs(ax.lo), fabs(ax.hi)) * (1.0 + 0x1p-20));
      // coefficients with e_last = j form block j of the nest order; its size is
      // the number of monomials of arity-1 variables of degree <= D - j
      int32_t off = 0;
      for (int j = 0; j <= r.degree; ++j) {
        J.block_off[j] = off;
        off += (int32_t)coeff_count(r.arity - 1, r.degree - j);
      }
    }
    J.rows_per_tile = (int32_t)std::max<int64_t>(1, std::min<int64_t>(64, 512 / J.row_words));
    J.tile0 = tiles;
    tiles += (J.nrows + J.rows_per_tile - 1) / J.rows_per_tile;
    max_rows = std::max(max_rows, J.rows_per_tile);
    max_deg = std::max(max_deg, r.degree);
    max_res_last = std::max(max_res_last, (int)res_last);
    if (r.degree != common_deg) common_deg = -1;
    const double eps = relation_eps(r, axes);
    J.eps = eps;
    J.eps32 = (float)eps;
    J.kfac = (float)((4.0 * r.degree + 8.0) * 0x1p-24 * 1.01);
    J.abs_margin = (float)(0x1p-21 * (double)J.eps32 + 1e-30);
    if (!isfinite(J.eps32)) {
      // eps beyond FP32 range: disable the filter, every pixel takes the FP64 path
      J.eps32 = 0.0f;
      J.kfac = INFINITY;
    }
    ex.st.pixels_plotted += (double)a.bits();
    ex.st.n_plots++;
  }
  // prep items are assigned to jobs by binary search on prep0: give the jobs
  // without preparation work the offset of the next one so the search skips them
  for (int i = nrel - 1; i >= 0; --i)
    if (!jobs[i].hoisted) jobs[i].prep0 = (i + 1 < nrel) ? jobs[i + 1].prep0 : prep_items;
  if (tiles > 0x7fffffffLL) throw Fail{set_err(ex.ctx, PA_ERR_TOO_LARGE, "plot grid too large")};
  const size_t jobs_off = blob_put(blob, jobs.data(), jobs.size());
  char* dblob = nullptr;
  if (ex.dry) {
    dblob = static_cast<char*>(ex.alloc(blob.size()));
  } else {
    // patch device coefficient pointers, then upload
    // (the device address of the blob is known only after allocation)
    const size_t off = (ex.used + kAlign - 1) / kAlign * kAlign;
    char* base = ex.ctx->arena + off;
    PlotJob* hj = reinterpret_cast<PlotJob*>(blob.data() + jobs_off);
    for (int i = 0; i < nrel; ++i)
      hj[i].coeffs = reinterpret_cast<const double*>(base + coeff_off[i]);
    dblob = static_cast<char*>(ex.upload(blob));
  }
  const PlotJob* djobs = reinterpret_cast<const PlotJob*>(dblob + jobs_off);
  if (prep_items > 0) {
    ex.before("plot_prep_kernel");
    if (!ex.dry) launch_plot_prep(djobs, nrel, prep_items, ex.s);
    ex.launched("plot_prep_kernel");
  }
  ex.before("plot_kernel");
  if (!ex.dry) launch_plot(djobs, nrel, tiles, max_rows, max_deg, common_deg, max_res_last, ex.s);
  ex.launched("plot_kernel");
  return plots;
}

// --------------------------------------------------------- solve (one pass)
struct SolveArgs {
  int32_t nvars;
  const pa_axis* axes;
  int32_t nrel;
  const pa_relation* rels;
  std::vector<int> exposed;
  int strict;
  int order;
  const int32_t* pairs;
  const pa_array* out;
};

void solve_pass(Exec& ex, const SolveArgs& a) {
  std::vector<int64_t> vres(a.nvars);
  std::vector<double> vresd(a.nvars);
  for (int v = 0; v < a.nvars; ++v) {
    vres[v] = a.axes[v].res;
    vresd[v] = a.axes[v].res;
  }
  std::vector<std::vector<int>> rv;
  for (int i = 0; i < a.nrel; ++i) rv.push_back(distinct_vars(a.rels[i]));
  Plan plan = plan_joins(a.nvars, vresd, rv, a.exposed, a.order, a.pairs);
  BitArr target = from_pa(*a.out);

  std::vector<BitArr> slots = plot_all(ex, a.nvars, a.axes, a.nrel, a.rels, a.strict, nullptr);
  // Joins whose inputs are ready at the same time (same depth in the cluster
  // tree) are independent: their contractions share one launch.
  const int nj = (int)plan.joins.size();
  std::vector<int> level(a.nrel + nj, 0);
  int max_level = 0;
  for (int t = 0; t < nj; ++t) {
    const Join& jn = plan.joins[t];
    level[a.nrel + t] = 1 + std::max(level[jn.a], level[jn.b]);
    max_level = std::max(max_level, level[a.nrel + t]);
  }
  slots.resize(a.nrel + nj);
  PendingRowOr pend;
  for (int lv = 1; lv <= max_level; ++lv) {
    int n_in_level = 0;
    for (int t = 0; t < nj; ++t) n_in_level += (level[a.nrel + t] == lv);
    const int64_t target_ctas = std::max<int64_t>(1, 152 / std::max(1, n_in_level));
    for (int t = 0; t < nj; ++t) {
      if (level[a.nrel + t] != lv) continue;
      const Join& jn = plan.joins[t];
      const bool last = (t + 1 == nj);
      slots[a.nrel + t] = join(ex, slots[jn.a], slots[jn.b], jn.keep, vres,
                               last ? &target : nullptr, &pend, target_ctas);
    }
    flush_rowor(ex, pend);
  }
  const BitArr& root = slots[plan.root];
  if (root.w != target.w) reshape(ex, root, target);
}

pa_status ensure_arena(pa_ctx* ctx, size_t need) {
  if (need <= ctx->arena_size) return PA_OK;
  if (ctx->cap && need > ctx->cap) {
    return set_err(ctx, PA_ERR_OOM, "workspace of " + std::to_string(need) +
                                        " bytes exceeds the context's cap");
  }
  if (ctx->stage_pending) {
    cudaEventSynchronize(ctx->stage_done);
    ctx->stage_pending = false;
  }
  if (ctx->arena) {
    cudaDeviceSynchronize();  // the old arena may still be in use by queued work
    cudaFree(ctx->arena);
    ctx->arena = nullptr;
    ctx->arena_size = 0;
  }
  size_t sz = need + need / 4 + (1 << 20);
  if (ctx->cap && sz > ctx->cap) sz = ctx->cap;
  if (cudaMalloc(reinterpret_cast<void**>(&ctx->arena), sz) != cudaSuccess) {
    cudaGetLastError();
    ctx->arena = nullptr;
    return set_err(ctx, PA_ERR_OOM, "cudaMalloc of the workspace failed");
  }
  ctx->arena_size = sz;
  return PA_OK;
}

template <class F>
pa_status run_two_pass(pa_ctx* ctx, cudaStream_t s, pa_stats* stats, F&& body) {
  try {
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, PA_ERR_CUDA, "cudaSetDevice failed");
    }
    Exec dry(ctx, s, true);
    body(dry);
    pa_status st = ensure_arena(ctx, dry.used);
    if (st != PA_OK) return st;
    Exec ex(ctx, s, false);
    body(ex);
    ex.st.workspace_bytes = (int64_t)ex.used;
    if (stats) *stats = ex.st;
    return PA_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

}  // namespace
}  // namespace pa

using namespace pa;

// ================================================================ C ABI
extern "C" {

pa_status pa_create(pa_ctx** out, int device, size_t workspace_cap) {
  if (!out) return PA_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
    cudaGetLastError();
    return PA_ERR_CUDA;
  }
  if (device < 0 || device >= n) return PA_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return PA_ERR_CUDA;
  if (probe_kernel_image() != cudaSuccess) {
    cudaGetLastError();
    return PA_ERR_CUDA;
  }
  pa_ctx* ctx = new pa_ctx();
  ctx->device = device;
  ctx->cap = workspace_cap;
  if (cudaEventCreateWithFlags(&ctx->stage_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&ctx->d_err), sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&ctx->d_stat), sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(ctx->d_stat, 0, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->stage_done) cudaEventDestroy(ctx->stage_done);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_stat) cudaFree(ctx->d_stat);
    delete ctx;
    return PA_ERR_CUDA;
  }
  *out = ctx;
  return PA_OK;
}

void pa_destroy(pa_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stage_pending) cudaEventSynchronize(ctx->stage_done);
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->d_stat) cudaFree(ctx->d_stat);
  if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
  if (ctx->stage_done) cudaEventDestroy(ctx->stage_done);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
}

const char* pa_last_error(const pa_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

pa_status pa_profile_enable(pa_ctx* ctx, int32_t on) {
  if (!ctx) return PA_ERR_INVALID_ARG;
  ctx->prof = on != 0;
  return PA_OK;
}

pa_status pa_profile_read(pa_ctx* ctx, int32_t max_kernels, char* names, int64_t* launches,
                          double* total_ms, int32_t* nkernels) {
  if (!ctx || max_kernels < 0 || (max_kernels > 0 && (!names || !launches || !total_ms)) ||
      !nkernels)
    return PA_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  std::vector<std::string> seen;
  std::vector<int64_t> cnt;
  std::vector<double> tot;
  for (const auto& r : ctx->recs) {
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return set_err(ctx, PA_ERR_CUDA, cudaGetErrorString(e));
    float ms = 0.0f;
    e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) return set_err(ctx, PA_ERR_CUDA, cudaGetErrorString(e));
    size_t k = std::find(seen.begin(), seen.end(), r.name) - seen.begin();
    if (k == seen.size()) {
      seen.push_back(r.name);
      cnt.push_back(0);
      tot.push_back(0.0);
    }
    cnt[k] += 1;
    tot[k] += ms;
  }
  ctx->recs.clear();
  ctx->ev_used = 0;
  unsigned long long words = 0;
  cudaError_t e2 = cudaMemcpy(&words, ctx->d_stat, sizeof words, cudaMemcpyDeviceToHost);
  if (e2 != cudaSuccess) return set_err(ctx, PA_ERR_CUDA, cudaGetErrorString(e2));
  cudaMemset(ctx->d_stat, 0, sizeof words);
  seen.push_back("words_or");  // not a kernel: 64-bit words OR-ed by the contractions
  cnt.push_back((int64_t)words);
  tot.push_back(0.0);
  *nkernels = (int32_t)seen.size();
  for (int k = 0; k < (int)seen.size() && k < max_kernels; ++k) {
    snprintf(names + 32 * k, 32, "%s", seen[k].c_str());
    launches[k] = cnt[k];
    total_ms[k] = tot[k];
  }
  return PA_OK;
}

pa_status pa_sync(pa_ctx* ctx, void* stream) {
  if (!ctx) return PA_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return set_err(ctx, PA_ERR_CUDA, cudaGetErrorString(e));
  int err = 0;
  e = cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return set_err(ctx, PA_ERR_CUDA, cudaGetErrorString(e));
  if (err) {
    cudaMemset(ctx->d_err, 0, sizeof(int));
    return set_err(ctx, PA_ERR_TIMEOUT, "a bounded device wait ran out (shared-memory tile load)");
  }
  return PA_OK;
}

int64_t pa_array_words(int32_t ndim, const int32_t* res) {
  if (ndim < 0 || ndim > PA_MAX_DIM || (ndim > 0 && !res)) return -1;
  if (ndim == 0) return 1;
  int64_t rows = 1;
  for (int i = 0; i < ndim - 1; ++i) {
    if (res[i] < 1) return -1;
    rows *= res[i];
  }
  if (res[ndim - 1] < 1) return -1;
  return rows * ((res[ndim - 1] + 63) / 64);
}

pa_status pa_valid_tolerance(const pa_relation* rel, const pa_axis* axes, int32_t nvars,
                             double* eps_out) {
  pa_ctx* ctx = nullptr;
  try {
    PA_CHECK_ARG(rel && eps_out, "null pointer");
    check_axes(ctx, nvars, axes);
    check_relation(ctx, *rel, nvars);
    pa_relation r = *rel;
    r.eps = -1.0;
    *eps_out = relation_eps(r, axes);
    return PA_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

pa_status pa_plot(pa_ctx* ctx, const pa_relation* rel, const pa_axis* axes, int32_t nvars,
                  int32_t strict, pa_array* out, void* stream) {
  if (!ctx) return PA_ERR_INVALID_ARG;
  try {
    PA_CHECK_ARG(rel != nullptr, "rel: null pointer");
    check_axes(ctx, nvars, axes);
    check_relation(ctx, *rel, nvars);
    check_array(ctx, out, "out");
    std::vector<int> dv = distinct_vars(*rel);
    PA_CHECK_ARG(out->ndim == (int)dv.size(), "out: ndim must equal the relation's distinct variables");
    for (int i = 0; i < out->ndim; ++i) {
      PA_CHECK_ARG(out->vars[i] == dv[i], "out: vars must be the relation's variables in order");
      PA_CHECK_ARG(out->res[i] == axes[dv[i]].res, "out: res must match the axes");
    }
  } catch (const Fail& f) {
    return f.st;
  }
  BitArr target = from_pa(*out);
  return run_two_pass(ctx, static_cast<cudaStream_t>(stream), nullptr, [&](Exec& ex) {
    plot_all(ex, nvars, axes, 1, rel, strict ? 1 : 0, &target);
  });
}

pa_status pa_contract(pa_ctx* ctx, const pa_array* A, const pa_array* B, int32_t nkeep,
                      const int32_t* keep, pa_array* out, void* stream) {
  if (!ctx) return PA_ERR_INVALID_ARG;
  std::vector<int> kv;
  std::vector<int64_t> vres;
  try {
    check_array(ctx, A, "A");
    check_array(ctx, B, "B");
    check_array(ctx, out, "out");
    PA_CHECK_ARG(nkeep >= 0 && nkeep <= PA_MAX_DIM && (nkeep == 0 || keep), "keep");
    PA_CHECK_ARG(out->ndim == nkeep, "out: ndim must equal nkeep");
    int maxv = 0;
    for (int i = 0; i < A->ndim; ++i) maxv = std::max(maxv, A->vars[i]);
    for (int i = 0; i < B->ndim; ++i) maxv = std::max(maxv, B->vars[i]);
    for (int i = 0; i < A->ndim; ++i) PA_CHECK_ARG(A->vars[i] >= 0, "A: negative variable id");
    for (int i = 0; i < B->ndim; ++i) PA_CHECK_ARG(B->vars[i] >= 0, "B: negative variable id");
    vres.assign(maxv + 1, 0);
    for (int i = 0; i < A->ndim; ++i) vres[A->vars[i]] = A->res[i];
    for (int i = 0; i < B->ndim; ++i) {
      const int v = B->vars[i];
      PA_CHECK_ARG(vres[v] == 0 || vres[v] == B->res[i], "A and B disagree on a resolution");
      vres[v] = B->res[i];
    }
    for (int i = 0; i < nkeep; ++i) {
      const int v = keep[i];
      PA_CHECK_ARG(v >= 0 && v <= maxv && vres[v] > 0, "keep: variable not in A or B");
      PA_CHECK_ARG(out->vars[i] == v && out->res[i] == vres[v], "out: vars/res must match keep");
      for (int j = 0; j < i; ++j) PA_CHECK_ARG(keep[j] != v, "keep: repeated variable");
      kv.push_back(v);
    }
    PA_CHECK_ARG(out->words != A->words && out->words != B->words, "out must not alias A or B");
  } catch (const Fail& f) {
    return f.st;
  }
  BitArr a = from_pa(*A), b = from_pa(*B), target = from_pa(*out);
  return run_two_pass(ctx, static_cast<cudaStream_t>(stream), nullptr, [&](Exec& ex) {
    BitArr r = join(ex, a, b, kv, vres, &target);
    if (r.w != target.w) reshape(ex, r, target);
  });
}

pa_status pa_solve_network(pa_ctx* ctx, int32_t nvars, const pa_axis* axes, int32_t nrel,
                           const pa_relation* rels, int32_t nexposed, const int32_t* exposed,
                           const pa_options* opts, pa_array* out, pa_stats* stats,
                           void* stream) {
  if (!ctx) return PA_ERR_INVALID_ARG;
  SolveArgs a;
  try {
    check_axes(ctx, nvars, axes);
    PA_CHECK_ARG(nrel >= 1 && rels, "at least one relation");
    for (int i = 0; i < nrel; ++i) check_relation(ctx, rels[i], nvars);
    PA_CHECK_ARG(nexposed >= 0 && nexposed <= PA_MAX_DIM && (nexposed == 0 || exposed),
                 "exposed: 0..8 variables");
    check_array(ctx, out, "out");
    PA_CHECK_ARG(out->ndim == nexposed, "out: ndim must equal nexposed");
    for (int i = 0; i < nexposed; ++i) {
      PA_CHECK_ARG(exposed[i] >= 0 && exposed[i] < nvars, "exposed: variable out of range");
      for (int j = 0; j < i; ++j) PA_CHECK_ARG(exposed[j] != exposed[i], "exposed: repeated");
      PA_CHECK_ARG(out->vars[i] == exposed[i] && out->res[i] == axes[exposed[i]].res,
                   "out: vars/res must match the exposed variables");
      a.exposed.push_back(exposed[i]);
    }
    a.order = opts ? opts->order : PA_ORDER_GREEDY;
    PA_CHECK_ARG(a.order == PA_ORDER_GREEDY || a.order == PA_ORDER_GIVEN || a.order == PA_ORDER_LEFT,
                 "opts: unknown order");
    a.pairs = nullptr;
    if (a.order == PA_ORDER_GIVEN) {
      PA_CHECK_ARG(plan_valid_given(nrel, opts->npairs, opts->pairs),
                   "opts: pairs must be nrel-1 joins of distinct live slots");
      a.pairs = opts->pairs;
    }
    a.strict = (opts && opts->strict) ? 1 : 0;
  } catch (const Fail& f) {
    return f.st;
  }
  a.nvars = nvars;
  a.axes = axes;
  a.nrel = nrel;
  a.rels = rels;
  a.out = out;
  return run_two_pass(ctx, static_cast<cudaStream_t>(stream), stats,
                      [&](Exec& ex) { solve_pass(ex, a); });
}

pa_status pa_plan_order(int32_t nvars, const pa_axis* axes, int32_t nrel, const pa_relation* rels,
                        int32_t nexposed, const int32_t* exposed, int32_t order,
                        int32_t* pairs_out, double* pixel_ops_out, int64_t* peak_bits_out) {
  pa_ctx* ctx = nullptr;
  try {
    check_axes(ctx, nvars, axes);
    PA_CHECK_ARG(nrel >= 1 && rels && (nexposed == 0 || exposed), "null pointer");
    PA_CHECK_ARG(order == PA_ORDER_GREEDY || order == PA_ORDER_LEFT, "order");
    for (int i = 0; i < nrel; ++i) check_relation(ctx, rels[i], nvars);
    std::vector<double> vres(nvars);
    for (int v = 0; v < nvars; ++v) vres[v] = axes[v].res;
    std::vector<std::vector<int>> rv;
    for (int i = 0; i < nrel; ++i) rv.push_back(distinct_vars(rels[i]));
    std::vector<int> ex(exposed, exposed + nexposed);
    Plan p = plan_joins(nvars, vres, rv, ex, order, nullptr);
    for (size_t t = 0; t < p.joins.size(); ++t) {
      if (pairs_out) {
        pairs_out[2 * t] = p.joins[t].a;
        pairs_out[2 * t + 1] = p.joins[t].b;
      }
    }
    if (pixel_ops_out) *pixel_ops_out = p.pixel_ops;
    if (peak_bits_out) *peak_bits_out = (int64_t)p.peak_bits;
    return PA_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

pa_status pa_tree_cost(int32_t nlinks, const double* link_res, int32_t npacks,
                       const int32_t* pack_nports, const int32_t* pack_links, int32_t nouter,
                       const int32_t* outer_links, int32_t njoins, const int32_t* join_nchildren,
                       const int32_t* join_children, double* serial_cost, double* parallel_cost) {
  if (!link_res || !pack_nports || !pack_links || (nouter && !outer_links) ||
      (njoins && (!join_nchildren || !join_children)))
    return PA_ERR_INVALID_ARG;
  return tree_cost(nlinks, link_res, npacks, pack_nports, pack_links, nouter, outer_links, njoins,
                   join_nchildren, join_children, serial_cost, parallel_cost);
}

}  // extern "C"
