// C interface of the pixel array engine (include/pa.h): argument checks, the
// context and its workspace, and the builder that turns join plans into a
// launch program.
//
// Every call is built twice: a sizing pass that only adds up the workspace and
// the descriptor blob it needs (no CUDA calls), then the real pass, which
// fills the blob with device addresses and records the launches.  The blob is
// copied to the device in one transfer and the launches run in order on the
// caller's stream.  A planned batch (pa_batch_create) keeps its program and its
// own memory and replays the whole sequence as one CUDA graph.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <thread>
#include <vector>

#include "mlp.h"
#include "pa_internal.h"
#include "planner.h"

namespace pa {
namespace {
struct Memo;
}
}  // namespace pa

struct pa_ctx {
  int device = 0;
  size_t cap = 0;
  char* arena = nullptr;
  size_t arena_size = 0;
  // pinned staging for descriptor uploads: a ring of slots, so that a call
  // waits only for the upload kNStage calls back (the host may run that many
  // calls ahead of the device)
  static constexpr int kNStage = 4;
  char* h_stage[kNStage] = {};
  size_t h_stage_size[kNStage] = {};
  cudaEvent_t stage_done[kNStage] = {};
  bool stage_pending[kNStage] = {};
  int stage_next = 0;
  std::string err;
  int* d_err = nullptr;                  // device error word written by bounded waits
  unsigned long long* d_stat = nullptr;  // words OR-ed by contractions (timing mode)
  // kernel timing (pa_profile_enable)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec {
    std::string name;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  size_t ev_used = 0;
  // contraction path (pa_set_contract_path) and the rates its automatic
  // choice compares (defaults measured on a GB300; pa_autotune re-measures)
  int path = PA_PATH_AUTO;
  double rate_or = 2.0e5;      // row-OR: B words OR-ed per microsecond, A 2 % dense
  double rate_or_dense = 9.0e5;  // the same, A 16 % dense
  double rate_mma = 4.4e8;     // tensor path (with operand expansion): multiply-adds per microsecond
  std::unordered_map<uint64_t, double> dens_cache;  // relation key -> estimated plot density
  std::unordered_map<uint64_t, double> obs_dens;    // subtree key -> density measured by pa_join_log
  std::unordered_map<uint64_t, double> obs_time;    // subtree key -> join microseconds measured by pa_join_log
  // the last pa_solve_network program, relaunched without planning when the
  // next call's arguments and planning state are the same byte for byte
  uint64_t plan_epoch = 0;  // changes with every setting or measurement that steers planning
  pa::Memo* memo = nullptr;
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

bool has(const std::vector<int>& v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); }

// ------------------------------------------------------------ program
enum OpKind { OP_PLOT, OP_MEMSET, OP_RESHAPE, OP_ROWOR, OP_UNPACK,
              OP_MMA, OP_CENTRES, OP_PLOT_EXPR, OP_PLOT_CORNER, OP_PERMUTE, OP_EWISE };

struct Op {
  OpKind kind;
  size_t off0 = 0, off1 = 0, off2 = 0;  // blob offsets (plot jobs; rowor descs, maps, cta0)
  int n = 0;                            // plot jobs / rowor problems
  int64_t count = 0;                    // prep items / plot tiles / rowor grid / words / rows
  int64_t m = 0, nw = 0;                // outer / dot: M and words per row
  int i0 = 0, i1 = 0, i2 = 0, i3 = 0;   // plot: rows/tile, max degree, common degree, max res
  size_t smem = 0;                      // rowor dynamic shared memory
  int64_t zw = 0;                       // plot: words of the ranges it clears (off1, nw ranges)
  uint64_t* p = nullptr;                // memset / and output
  const uint64_t* a = nullptr;
  const uint64_t* b = nullptr;
  int join = -1;                        // join this op belongs to (join logging)
};

const char* op_name(const Op& op) {
  switch (op.kind) {
    case OP_PLOT: return "plot_kernel";
    case OP_CENTRES: return "plot_centres_kernel";
    case OP_PLOT_EXPR: return "plot_expr_kernel";
    case OP_PLOT_CORNER: return "plot_corner_kernel";
    case OP_PERMUTE: return "permute_u32_kernel";
    case OP_EWISE: return "ewise_kernel";
    case OP_MEMSET: return "memset";
    case OP_RESHAPE:
      return op.i0 == kRsTranspose ? "reshape_transpose_kernel"
             : (op.i0 == kRsWords32 || op.i0 == kRsWords64) ? "reshape_words_kernel"
                                                            : "reshape_kernel";
    case OP_UNPACK: return "unpack_kernels";
    case OP_MMA: return "mma_bool_kernel";
    default: return "rowor_kernel";
  }
}

// A planned call kept for reuse: its key (arguments and planning state), its
// launch list, its descriptor blob (coefficients included) and its statistics.
struct Memo {
  std::vector<char> key;
  std::vector<Op> ops;
  std::vector<char> blob;
  pa_stats st{};
  // the launches captured as one CUDA graph on the second call with the key
  // (the descriptor upload stays a copy of its own before each launch)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool capture_failed = false;
  ~Memo() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

// Builds the workspace layout, the descriptor blob and the launch list of a call.
struct Builder {
  pa_ctx* ctx;
  bool dry;
  char* base = nullptr;     // device memory the layout lives in (null in the sizing pass)
  size_t used = 0;          // bytes of `base` in use
  size_t blob_cap = 0;      // bytes reserved for the blob at the start of `base`
  std::vector<char> blob;   // host image of the descriptor blob
  std::vector<Op> ops;
  pa_stats st{};
  int* d_err = nullptr;
  unsigned long long* d_stat = nullptr;
  std::vector<RowOrDesc> pend;  // contractions waiting for one shared launch
  std::vector<MmaDesc> pend_mma;  // tensor-core contractions waiting for one launch
  // Inside one tree level of build_networks: reshapes wait for one launch per
  // kind, and the level's other ops for after them (they read the reshapes'
  // results), so independent joins share launches.
  bool defer = false;
  std::vector<ReshapeDesc> pend_rs;
  std::vector<EwJob> pend_ew;
  std::vector<Op> pend_ops;
  void emit(const Op& op) { (defer ? pend_ops : ops).push_back(op); }

  Builder(pa_ctx* c, bool dry_, char* base_, size_t blob_cap_)
      : ctx(c), dry(dry_), base(base_), used(blob_cap_), blob_cap(blob_cap_) {}

  void* alloc(size_t bytes) {
    const size_t off = (used + kAlign - 1) / kAlign * kAlign;
    used = off + std::max<size_t>(bytes, 8);
    if (dry) return reinterpret_cast<void*>(static_cast<uintptr_t>(kAlign + off));
    return base + off;
  }
  uint64_t* alloc_words(int64_t n) { return static_cast<uint64_t*>(alloc((size_t)n * 8)); }

  template <class T>
  size_t put(const T* data, size_t n, size_t align = 16) {
    const size_t off = (blob.size() + align - 1) / align * align;
    blob.resize(off + sizeof(T) * n);
    if (n) memcpy(blob.data() + off, data, sizeof(T) * n);
    return off;
  }
  // device address of a blob offset (fake in the sizing pass)
  char* dev(size_t off) const {
    if (dry) return reinterpret_cast<char*>(static_cast<uintptr_t>(64 + off));
    return base + off;
  }
  void fail(pa_status st, const std::string& msg) { throw Fail{set_err(ctx, st, msg)}; }
};

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

// Output words per step of output axis a (a non-last inner axis needs a
// row length that is a multiple of 64 beyond it, which the callers check).
int64_t out_word_stride(const BitArr& out, int a) {
  const int outer = out.ndim - out.inner;
  int64_t st = 1;
  if (a < outer) {
    for (int b = a + 1; b < outer; ++b) st *= out.res[b];
    return st * out.row_words();
  }
  for (int b = a + 1; b < out.ndim; ++b) st *= out.res[b];
  return st / 64;
}

// Pick the fastest reshape kernel whose preconditions hold (strides of `d`
// already filled in).  Words: the last output axis L is the input's last axis
// and its runs start on word boundaries.  Transpose: L steps by input rows or
// by whole input words, the input's last axis J is kept, both packed axes
// start on word boundaries, nothing is reduced.
void choose_reshape_mode(ReshapeDesc& d, const BitArr& in, const BitArr& out) {
  d.mode = kReshapeBits;
  d.row_any = 0;
  if (d.nred > 0) {
    // every packed input axis reduced: OR whole rows instead of single bits
    bool all_inner_reduced = in.inner > 0;
    for (int a = 0; a < out.ndim && all_inner_reduced; ++a) all_inner_reduced = d.col_stride[a] == 0;
    if (all_inner_reduced) {
      int n = 0;
      for (int q = 0; q < d.nred; ++q) {
        if (d.red_col_stride[q] != 0) continue;
        d.red_res[n] = d.red_res[q];
        d.red_row_stride[n] = d.red_row_stride[q];
        d.red_col_stride[n] = 0;
        ++n;
      }
      d.nred = n;
      d.row_any = 1;
      return;
    }
  }
  if (out.ndim == 0 || out.inner == 0 || in.ndim == 0) return;
  const int L = out.ndim - 1;
  const int64_t R = out.res[L];
  const bool l_aligned = (R % 64 == 0) || out.inner == 1;
  if (!l_aligned) return;
  if (d.col_stride[L] == 1 && (R % 64 == 0 || (in.inner == 1 && out.inner == 1))) {
    bool ok = true;
    for (int a = 0; a < L && ok; ++a) ok = (d.col_stride[a] % 64 == 0);
    for (int q = 0; q < d.nred && ok; ++q) ok = (d.red_col_stride[q] % 64 == 0);
    if (ok) {
      d.mode = kReshapeWords;
      d.nu = out.ndim;
      for (int a = 0; a < L; ++a) {
        d.u_res[a] = out.res[a];
        d.u_in[a] = d.row_stride[a] * d.in_row_words + d.col_stride[a] / 64;
      }
      d.u_res[L] = (R + 63) / 64;
      d.u_in[L] = 1;
      for (int q = 0; q < d.nred; ++q)
        d.red_in_w[q] = d.red_row_stride[q] * d.in_row_words + d.red_col_stride[q] / 64;
      return;
    }
  }
  if (d.nred != 0) return;
  // L steps by whole input rows, or by whole words inside a row
  const bool l_row = d.row_stride[L] > 0 && d.col_stride[L] == 0;
  const bool l_col = d.row_stride[L] == 0 && d.col_stride[L] > 0 && d.col_stride[L] % 64 == 0;
  if (!l_row && !l_col) return;
  int J = -1;
  for (int a = 0; a < L; ++a)
    if (d.col_stride[a] == 1) J = a;
  if (J < 0) return;
  const int64_t Q = out.res[J];
  if (!(in.inner == 1 || Q % 64 == 0)) return;
  for (int a = 0; a < L; ++a)
    if (a != J && d.col_stride[a] % 64 != 0) return;
  d.mode = kReshapeTranspose;
  d.nu = 0;
  d.n_other = 1;
  for (int a = 0; a < L; ++a) {
    if (a == J) continue;
    d.u_res[d.nu] = out.res[a];
    d.u_in[d.nu] = d.row_stride[a] * d.in_row_words + d.col_stride[a] / 64;
    d.u_out[d.nu] = out_word_stride(out, a);
    d.n_other *= out.res[a];
    d.nu++;
  }
  d.tQ = Q;
  d.tR = R;
  d.t_in_L = d.row_stride[L] * d.in_row_words + d.col_stride[L] / 64;
  d.t_out_J = out_word_stride(out, J);
}

void flush_reshapes(Builder& bd);

// The waiting outer / dot / Hadamard clusters as one launch (job table and
// block offsets in the blob).
void flush_ew(Builder& bd) {
  std::vector<EwJob> jobs;
  std::vector<int64_t> cta0(1, 0);
  for (const EwJob& j : bd.pend_ew) {
    const int64_t nb = ewise_blocks(j);
    if (nb <= 0) continue;
    jobs.push_back(j);
    cta0.push_back(cta0.back() + nb);
  }
  bd.pend_ew.clear();
  if (jobs.empty()) return;
  if (cta0.back() > 0x7fffffffLL) bd.fail(PA_ERR_TOO_LARGE, "cluster grid too large");
  Op op;
  op.kind = OP_EWISE;
  op.off0 = bd.put(jobs.data(), jobs.size(), 64);
  op.off1 = bd.put(cta0.data(), cta0.size(), 16);
  op.n = (int)jobs.size();
  op.count = cta0.back();
  bd.ops.push_back(op);
}

void add_ew(Builder& bd, const EwJob& j) {
  bd.pend_ew.push_back(j);
  if (!bd.defer) flush_ew(bd);
}

// out <- in with axes matched by variable; input axes missing from out are
// OR-reduced, output axes missing from in are broadcast.
void reshape(Builder& bd, const BitArr& in, const BitArr& out) {
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
  choose_reshape_mode(d, in, out);
  bd.st.n_reshapes++;
  bd.pend_rs.push_back(d);
  if (!bd.defer) flush_reshapes(bd);
}

// The waiting reshapes as one launch per kernel kind (descriptor table and
// block offsets in the blob).
void flush_reshapes(Builder& bd) {
  for (int kind = 0; kind < 4; ++kind) {
    std::vector<ReshapeDesc> group;
    std::vector<int64_t> cta0(1, 0);
    for (const ReshapeDesc& d : bd.pend_rs) {
      if (reshape_kind(d) != kind) continue;
      const int64_t nb = reshape_blocks(d);
      if (nb <= 0) continue;
      group.push_back(d);
      cta0.push_back(cta0.back() + nb);
    }
    if (group.empty()) continue;
    if (cta0.back() > 0x7fffffffLL) bd.fail(PA_ERR_TOO_LARGE, "reshape grid too large");
    Op op;
    op.kind = OP_RESHAPE;
    op.off0 = bd.put(group.data(), group.size(), 64);
    op.off1 = bd.put(cta0.data(), cta0.size(), 16);
    op.n = (int)group.size();
    op.count = cta0.back();
    op.i0 = kind;
    bd.ops.push_back(op);
  }
  bd.pend_rs.clear();
}

// Bring `x` into layout `want` (vars/res/inner of want; want.w ignored).  Returns
// x itself when the layouts already agree.
BitArr conform(Builder& bd, const BitArr& x, BitArr want) {
  if (same_layout(x, want)) {
    want.w = x.w;
    return want;
  }
  want.w = bd.alloc_words(want.words());
  reshape(bd, x, want);
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

// The waiting tensor-core contractions as one launch.
void flush_mma(Builder& bd) {
  if (bd.pend_mma.empty()) return;
  const size_t n = bd.pend_mma.size();
  std::vector<CUtensorMap> maps(2 * n);
  std::vector<int64_t> cta0(n + 1, 0);
  for (size_t p = 0; p < n; ++p) {
    if (bd.dry) memset(&maps[2 * p], 0, 2 * sizeof(CUtensorMap));
    else if (mma_encode_maps(bd.pend_mma[p], &maps[2 * p]) != cudaSuccess)
      bd.fail(PA_ERR_CUDA, "cuTensorMapEncodeTiled failed (tensor-core path)");
    cta0[p + 1] = cta0[p] + mma_ctas(bd.pend_mma[p]);
  }
  // one launch per operand kind expands every problem's operands, then one
  // launch contracts them all
  Op up;
  up.kind = OP_UNPACK;
  up.off0 = bd.put(bd.pend_mma.data(), n, 64);
  up.n = (int)n;
  for (const MmaDesc& d : bd.pend_mma) {
    up.m = std::max<int64_t>(up.m, unpack_blocks_a(d));
    up.nw = std::max<int64_t>(up.nw, unpack_blocks_b(d));
  }
  if (n > 65535) bd.fail(PA_ERR_TOO_LARGE, "more than 65535 tensor-core problems in one level");
  bd.ops.push_back(up);
  Op op;
  op.kind = OP_MMA;
  op.off0 = up.off0;
  op.off1 = bd.put(maps.data(), maps.size(), 128);
  op.off2 = bd.put(cta0.data(), cta0.size(), 16);
  op.n = (int)n;
  op.count = cta0.back();
  if (op.count > 0x7fffffffLL) bd.fail(PA_ERR_TOO_LARGE, "contraction grid too large");
  bd.ops.push_back(op);
  bd.pend_mma.clear();
}

void flush_rowor_only(Builder& bd);

// The waiting contractions as launches: one per tile width, one for the
// tensor-core path.
void flush_rowor(Builder& bd) {
  flush_rowor_only(bd);
  flush_mma(bd);
}

// End of one tree level: its reshapes, then the ops that read them, then the
// contraction launches.
void flush_level(Builder& bd) {
  flush_reshapes(bd);
  bd.ops.insert(bd.ops.end(), bd.pend_ops.begin(), bd.pend_ops.end());
  bd.pend_ops.clear();
  flush_ew(bd);
  flush_rowor(bd);
}

void flush_rowor_only(Builder& bd) {
  std::vector<int> done(bd.pend.size(), 0);
  for (size_t i = 0; i < bd.pend.size(); ++i) {
    if (done[i]) continue;
    std::vector<RowOrDesc> group;
    for (size_t j = i; j < bd.pend.size(); ++j)
      if (!done[j] && bd.pend[j].Nt == bd.pend[i].Nt) {
        group.push_back(bd.pend[j]);
        done[j] = 1;
      }
    std::vector<CUtensorMap> maps(group.size());
    std::vector<int64_t> cta0(group.size() + 1, 0);
    size_t smem = 0;
    for (size_t p = 0; p < group.size(); ++p) {
      if (bd.dry) memset(&maps[p], 0, sizeof(CUtensorMap));
      else if (rowor_encode_map(group[p], &maps[p]) != cudaSuccess)
        bd.fail(PA_ERR_CUDA, "cuTensorMapEncodeTiled failed");
      cta0[p + 1] = cta0[p] + rowor_ctas(group[p]);
      smem = std::max(smem, rowor_smem_bytes(group[p]));
    }
    Op op;
    op.kind = OP_ROWOR;
    op.off0 = bd.put(group.data(), group.size(), 64);
    op.off1 = bd.put(maps.data(), maps.size(), 128);
    op.off2 = bd.put(cta0.data(), cta0.size(), 16);
    op.n = (int)group.size();
    op.count = cta0.back();
    op.smem = smem;
    op.i0 = group[0].Nt;
    if (op.count > 0x7fffffffLL) bd.fail(PA_ERR_TOO_LARGE, "contraction grid too large");
    bd.ops.push_back(op);
  }
  bd.pend.clear();
}

// Shape of one two-array cluster (Eq. GAM on X and Y, outer pack `keep`):
// either a Hadamard product (nothing summed between X and Y) or a matrix form
// A[batch][M][K] x B[batch][K][N] -> C[batch][M][N] with A and B chosen so that
// fewer bits need reshaping, then the wider packed side as B.
struct JoinShape {
  bool hadamard = false;
  bool outer = false;           // nothing summed: C[batch][M][N] = A[batch][M] AND B[batch][N]
  bool dot = false;             // nothing kept from B alone: C[batch][M] = OR_K A AND B[batch][K]
  bool swap = false;            // A = Y, B = X
  std::vector<int> a_axes, b_axes, c_axes;
  int kinner = 0, ninner = 0;   // number of K and N axes
  int64_t nbatch = 1, M = 1, K = 1;
  double nbits = 1.0;           // N (bits per output row)
  double reshape_bits = 0.0;    // bits of operands that need a reshape
  double cost = 1.0;            // r^Lambda of the cluster (naive cost, Sec. 3.5)
  double result_bits = 1.0;
  double private_a = 1.0, private_b = 1.0;  // sizes of the axes reduced away
};

JoinShape analyze_join(const BitArr& X, const BitArr& Y, const std::vector<int>& keep,
                       const std::vector<int64_t>& vres) {
  JoinShape js;
  std::vector<int> xv(X.vars, X.vars + X.ndim), yv(Y.vars, Y.vars + Y.ndim);
  {
    std::vector<int> u = xv;
    for (int v : yv)
      if (!has(u, v)) u.push_back(v);
    for (int v : u) js.cost *= (double)vres[v];
  }
  for (int v : keep) js.result_bits *= (double)vres[v];
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
  if (K.empty() && M.empty() && N.empty()) {
    js.hadamard = true;
    for (int v : xv)
      if (!has(keep, v)) js.private_a *= (double)vres[v];
    for (int v : yv)
      if (!has(keep, v)) js.private_b *= (double)vres[v];
    return js;
  }
  struct Choice {
    std::vector<int> batch, M, K, N;
    double reshape_bits = 0, nbits = 1;
  };
  auto evaluate = [&](bool swap) {
    Choice c;
    const BitArr& A = swap ? Y : X;
    const BitArr& B = swap ? X : Y;
    std::vector<int> av(A.vars, A.vars + A.ndim), bv(B.vars, B.vars + B.ndim);
    classify(av, bv, c.batch, c.M, c.K, c.N);
    std::vector<int> a_axes = c.batch, b_axes = c.batch;
    a_axes.insert(a_axes.end(), c.M.begin(), c.M.end());
    a_axes.insert(a_axes.end(), c.K.begin(), c.K.end());
    b_axes.insert(b_axes.end(), c.K.begin(), c.K.end());
    b_axes.insert(b_axes.end(), c.N.begin(), c.N.end());
    // a K-free cluster reads A as one flat bit vector over (batch, M); an
    // N-free one reads B as one packed row of K bits per batch value
    const int a_inner = c.K.empty() ? (int)a_axes.size() : (int)c.K.size();
    const int b_inner = (c.N.empty() && !c.K.empty()) ? (int)c.K.size() : (int)c.N.size();
    if (!same_layout(A, make_arr(a_axes, vres, a_inner))) c.reshape_bits += (double)A.bits();
    if (!same_layout(B, make_arr(b_axes, vres, b_inner))) c.reshape_bits += (double)B.bits();
    for (int v : c.N) c.nbits *= (double)vres[v];
    return c;
  };
  Choice c0 = evaluate(false), c1 = evaluate(true);
  js.outer = K.empty();
  if (js.outer && (c0.N.empty() != c1.N.empty()))
    js.swap = c0.N.empty();  // keep packed result rows: the side with N axes is B
  else if (c1.reshape_bits != c0.reshape_bits)
    js.swap = c1.reshape_bits < c0.reshape_bits;
  else if (c0.N.empty() != c1.N.empty())
    js.swap = c0.N.empty();
  else
    js.swap = c1.nbits > c0.nbits;
  const Choice& ch = js.swap ? c1 : c0;
  js.a_axes = js.b_axes = js.c_axes = ch.batch;
  js.a_axes.insert(js.a_axes.end(), ch.M.begin(), ch.M.end());
  js.a_axes.insert(js.a_axes.end(), ch.K.begin(), ch.K.end());
  js.b_axes.insert(js.b_axes.end(), ch.K.begin(), ch.K.end());
  js.b_axes.insert(js.b_axes.end(), ch.N.begin(), ch.N.end());
  js.c_axes.insert(js.c_axes.end(), ch.M.begin(), ch.M.end());
  js.c_axes.insert(js.c_axes.end(), ch.N.begin(), ch.N.end());
  js.kinner = (int)ch.K.size();
  js.ninner = (int)ch.N.size();
  js.dot = !js.outer && ch.N.empty();
  for (int v : ch.batch) js.nbatch *= vres[v];
  for (int v : ch.M) js.M *= vres[v];
  for (int v : ch.K) js.K *= vres[v];
  js.nbits = ch.nbits;
  js.reshape_bits = ch.reshape_bits;
  const BitArr& A = js.swap ? Y : X;
  const BitArr& B = js.swap ? X : Y;
  for (int i = 0; i < A.ndim; ++i)
    if (!has(js.a_axes, A.vars[i])) js.private_a *= (double)A.res[i];
  for (int i = 0; i < B.ndim; ++i)
    if (!has(js.b_axes, B.vars[i])) js.private_b *= (double)B.res[i];
  return js;
}

// Layout of a join's result before any final reshape.
BitArr join_result_layout(const JoinShape& js, const std::vector<int>& keep,
                          const std::vector<int64_t>& vres) {
  if (js.hadamard) return make_arr(keep, vres, keep.empty() ? 0 : 1);
  if (js.dot) return make_arr(js.c_axes, vres, (int)js.c_axes.size());
  return make_arr(js.c_axes, vres, js.ninner);
}

// One two-array cluster.  When `target` is given and the result lands in its
// layout, the result is written there.  Row-OR contractions wait in bd.pend
// for flush_rowor.
void join_features(const JoinShape& js, double rx, double ry, float* f, double* rho_out);
double or_density(double rho, double n);

// Tensor-core path or row-OR for a matrix-form cluster?  Forced by
// pa_set_contract_path, else the faster by the context's measured rates: the
// row-OR is costed as (set bits of A) x (words per B row) word ORs at the rate
// measured on random operands (runs of set bits make it faster than that)
// plus a fixed cost per (row, K chunk, tile) unit; the tensor path as every
// multiply-add of its padded 128 x BN x 128 tiles (its rate includes the
// expansion of both operands; tile pairs it skips because one operand's tile
// is empty are not credited, so the estimate errs towards the row-OR).  `ra`
// is A's estimated density (< 0: unknown).
constexpr double kRowOrUnitsPerUs = 3.0e3;

// Estimated microseconds of a matrix-form cluster on the row-OR path when A
// has density `dens`: its word ORs at the context's measured rate (log-linear
// in the density between the two measured points) plus every (row, K chunk,
// tile) unit's fixed bookkeeping, about 200 warp instructions (ncu, chain
// joins) at half the issue rate of 152 SMs x 4 schedulers x 2 GHz, some 3e9
// units per second.
double rowor_cost_us(const pa_ctx* ctx, const JoinShape& js, double dens) {
  const double M = (double)js.M, N = js.nbits, K = (double)js.K, nb = (double)js.nbatch;
  const double r0 = ctx ? ctx->rate_or : 2.0e5, r1 = ctx ? ctx->rate_or_dense : 9.0e5;
  const double f = std::min(1.0, std::max(0.0, log(std::max(dens, 1e-12) / 0.02) / log(8.0)));
  const double rate_or = r0 * pow(r1 / r0, f);
  RowOrDesc rd;
  memset(&rd, 0, sizeof rd);
  rd.nbatch = js.nbatch;
  rd.M = js.M;
  rd.K = js.K;
  rd.Nw = (int64_t)ceil(N / 64);
  rd.a_row_words = (js.K + 63) / 64;
  rowor_plan(rd, 152);
  const double units = nb * M * (double)rd.k_chunks * (double)rd.n_tiles;
  return dens * M * K * nb * ceil(N / 64) / rate_or + units / kRowOrUnitsPerUs;
}

// Bytes per microsecond the two expansion kernels write together (measured
// on 2048 x 2048 operands of a GB300: 8.4 MB in 12 us).
constexpr double kExpandBytesPerUs = 7.0e5;

bool use_mma(const pa_ctx* ctx, const JoinShape& js, double ra) {
  // no context (pa_solve_network_static): the row-OR, which needs no byte copies
  if (!ctx || ctx->path == PA_PATH_ROWOR || tensor_map_encoder() == nullptr) return false;
  const double M = (double)js.M, N = js.nbits, K = (double)js.K, nb = (double)js.nbatch;
  if (nb * M >= 2147483647.0 || N >= 2147483647.0 || nb >= 2147483647.0) return false;
  if (nb * (M + N) * (ceil(K / 128) * 128) > 4e9) return false;  // byte copies of the operands
  if (ctx->path == PA_PATH_MMA) return true;
  const double BN = N <= 64 ? 64 : N <= 128 ? 128 : 256;
  const double macs = nb * ceil(M / 128) * 128 * ceil(N / BN) * BN * ceil(K / 128) * 128;
  if (macs < 134217728.0) return false;  // small clusters: the row-OR's launch is cheaper
  const double dens = ra >= 0 ? ra : 0.05;
  const double t_or = rowor_cost_us(ctx, js, dens);
  // rate_mma is measured on a 2048^3 product, expansion of both operands
  // included (2 x 2048^2 bytes for 2048^3 multiply-adds); a cluster whose
  // operands are larger relative to its products (few rows and columns,
  // many summed values) pays the bytes beyond that share at the expansion
  // kernels' rate
  const double bytes = nb * (M + N) * (ceil(K / 128) * 128);
  const double extra = std::max(0.0, bytes - macs * (2.0 / 2048.0));
  const double t_mma = macs / ctx->rate_mma + extra / kExpandBytesPerUs;
  return t_mma < t_or;
}

// The occupancy bitmaps of a tensor-core problem (one bit per 128 x 128 tile
// of each operand), cleared before its expansion kernels set them.
void add_occupancy(Builder& bd, MmaDesc& md) {
  const int64_t w32 = mma_occ_words(md);
  const int64_t w64 = (w32 + 1) / 2;
  uint32_t* occ = static_cast<uint32_t*>(bd.alloc((size_t)w64 * 8));
  md.occ_a = occ;
  md.occ_b = occ + md.nbatch * md.m_tiles * md.kb_words;
  Op op;
  op.kind = OP_MEMSET;
  op.p = reinterpret_cast<uint64_t*>(occ);
  op.count = w64;
  bd.emit(op);
}

// rx, ry: estimated densities of X and Y (< 0: unknown); *rho_out receives the
// estimated density of the result when both are known.
BitArr join(Builder& bd, const BitArr& X, const BitArr& Y, const std::vector<int>& keep,
            const std::vector<int64_t>& vres, const BitArr* target, int64_t target_ctas,
            double rx = -1.0, double ry = -1.0, double* rho_out = nullptr) {
  const JoinShape js = analyze_join(X, Y, keep, vres);
  bd.st.pixel_ops_dense += js.cost;
  bd.st.n_joins++;
  double ra = -1.0;
  if (rx >= 0 && ry >= 0) {
    float f[PA_FEATURES];
    join_features(js, rx, ry, f, rho_out);
    ra = or_density(js.swap ? ry : rx, js.private_a);
  }

  if (js.hadamard) {
    bool use_target = target && target->w && target->ndim == (int)keep.size();
    for (int i = 0; use_target && i < target->ndim; ++i) use_target = has(keep, target->vars[i]);
    BitArr want = use_target ? *target : make_arr(keep, vres, keep.empty() ? 0 : 1);
    std::vector<int> wv(want.vars, want.vars + want.ndim);
    BitArr xa = conform(bd, X, make_arr(wv, vres, want.inner));
    BitArr ya = conform(bd, Y, make_arr(wv, vres, want.inner));
    BitArr out = want;
    if (!out.w) out.w = bd.alloc_words(out.words());
    add_ew(bd, EwJob{xa.w, ya.w, out.w, out.words(), 1, 1, kEwAnd});
    return out;
  }

  const BitArr& A = js.swap ? Y : X;
  const BitArr& B = js.swap ? X : Y;
  if (js.outer) {
    BitArr Am = conform(bd, A, make_arr(js.a_axes, vres, (int)js.a_axes.size()));
    BitArr Bm = conform(bd, B, make_arr(js.b_axes, vres, js.ninner));
    BitArr C = make_arr(js.c_axes, vres, js.ninner);
    if (target && target->w && same_layout(C, *target)) C.w = target->w;
    else C.w = bd.alloc_words(C.words());
    add_ew(bd, EwJob{Am.w, Bm.w, C.w, js.nbatch * js.M, js.M, Bm.row_words(), kEwOuter});
    bd.st.peak_words = std::max<int64_t>(bd.st.peak_words, C.words());
    return C;
  }
  if (js.dot) {
    BitArr Am = conform(bd, A, make_arr(js.a_axes, vres, js.kinner));
    BitArr Bm = conform(bd, B, make_arr(js.b_axes, vres, js.kinner));
    BitArr C = make_arr(js.c_axes, vres, (int)js.c_axes.size());
    if (target && target->w && same_layout(C, *target)) C.w = target->w;
    else C.w = bd.alloc_words(C.words());
    const int64_t rows = js.nbatch * js.M, kw = Am.row_words();
    if (kw > 16) {
      // long rows OR their bits into a cleared C
      Op z;
      z.kind = OP_MEMSET;
      z.p = C.w;
      z.count = (rows + 63) / 64;
      bd.emit(z);
    }
    add_ew(bd, EwJob{Am.w, Bm.w, C.w, rows, js.M, kw, kw > 16 ? kEwDotWide : kEwDot});
    bd.st.peak_words = std::max<int64_t>(bd.st.peak_words, C.words());
    return C;
  }
  BitArr Am = conform(bd, A, make_arr(js.a_axes, vres, js.kinner));
  BitArr Bm = conform(bd, B, make_arr(js.b_axes, vres, js.ninner));
  BitArr C = make_arr(js.c_axes, vres, js.ninner);
  if (target && target->w && same_layout(C, *target)) C.w = target->w;
  else C.w = bd.alloc_words(C.words());

  if (use_mma(bd.ctx, js, ra)) {
    MmaDesc md;
    memset(&md, 0, sizeof md);
    md.A = Am.w;
    md.B = Bm.w;
    md.C = C.w;
    md.M = js.M;
    md.N = (int64_t)js.nbits;
    md.K = js.K;
    md.a_row_words = Am.row_words();
    md.nbatch = js.nbatch;
    md.err = bd.d_err;
    mma_plan(md);
    md.Ab = static_cast<uint8_t*>(bd.alloc((size_t)(md.nbatch * md.M * md.Kp)));
    md.Bb = static_cast<uint8_t*>(bd.alloc((size_t)(md.nbatch * md.N * md.Kp)));
    add_occupancy(bd, md);
    if (md.ksplit > 1) {
      // the CTAs of one tile OR their partial results into C
      Op z;
      z.kind = OP_MEMSET;
      z.p = C.w;
      z.count = C.words();
      bd.emit(z);
    }
    bd.pend_mma.push_back(md);
    bd.st.mma_macs += (double)js.nbatch * (double)js.M * js.nbits * (double)js.K;
    bd.st.n_mma++;
    bd.st.peak_words = std::max<int64_t>(bd.st.peak_words, C.words());
    return C;
  }
  RowOrDesc d;
  memset(&d, 0, sizeof d);
  d.A = Am.w;
  d.B = Bm.w;
  d.C = C.w;
  d.nbatch = js.nbatch;
  d.M = js.M;
  d.K = js.K;
  d.Nw = Bm.row_words();
  d.a_row_words = Am.row_words();
  d.err = bd.d_err;
  d.stat = bd.d_stat;
  if (d.M > 0x7fffffffLL || d.K > 0x7fffffffLL)
    bd.fail(PA_ERR_TOO_LARGE, "contraction with more than 2^31 rows");
  rowor_plan(d, target_ctas);
  if (d.atomic) {
    Op op;
    op.kind = OP_MEMSET;
    op.p = C.w;
    op.count = C.words();
    bd.emit(op);
  }
  bd.pend.push_back(d);
  bd.st.peak_words = std::max<int64_t>(bd.st.peak_words, C.words());
  return C;
}

// One cluster over the counting semiring (the paper's footnote on other
// semi-rings, Sec. 2.2): out(e') = sum over the summed variables of
// A(e_A) * B(e_B), the number of latent pixel tuples behind each output
// pixel.  On the tensor cores with the > 0 threshold left out: the operands
// are 0/1, so every sum is an integer <= K, exact in FP32 up to 2^24.
// Supported when every summed variable is shared by A and B (no axis private
// to one operand) and both keep a variable of their own or a shared one.
void join_count(Builder& bd, const BitArr& X, const BitArr& Y, const std::vector<int>& keep,
                const std::vector<int64_t>& vres, uint32_t* out) {
  const JoinShape js = analyze_join(X, Y, keep, vres);
  if (js.hadamard || js.outer || js.dot)
    bd.fail(PA_ERR_UNSUPPORTED, "counting: A and B must share a summed variable and B must keep "
                                "a variable A does not have");
  if (js.private_a != 1.0 || js.private_b != 1.0)
    bd.fail(PA_ERR_UNSUPPORTED, "counting: every summed variable must be shared by A and B");
  if (js.K > (1 << 24)) bd.fail(PA_ERR_UNSUPPORTED, "counting: more than 2^24 summed values");
  if (tensor_map_encoder() == nullptr) bd.fail(PA_ERR_UNSUPPORTED, "counting needs the tensor maps");
  const double M = (double)js.M, N = js.nbits, nb = (double)js.nbatch;
  if (nb * M >= 2147483647.0 || N >= 2147483647.0 ||
      nb * (M + N) * (ceil((double)js.K / 128) * 128) > 4e9)
    bd.fail(PA_ERR_TOO_LARGE, "counting: operands too large for the tensor-core expansion");
  bd.st.pixel_ops_dense += js.cost;
  bd.st.n_joins++;
  const BitArr& A = js.swap ? Y : X;
  const BitArr& B = js.swap ? X : Y;
  BitArr Am = conform(bd, A, make_arr(js.a_axes, vres, js.kinner));
  BitArr Bm = conform(bd, B, make_arr(js.b_axes, vres, js.ninner));
  // the sums come out row-major over c_axes (batch, M, N); keep may order them
  // otherwise
  const bool natural = (js.c_axes == keep);
  const int64_t total = (int64_t)(nb * M * N);
  uint32_t* sums = natural ? out : static_cast<uint32_t*>(bd.alloc((size_t)total * 4));
  MmaDesc md;
  memset(&md, 0, sizeof md);
  md.A = Am.w;
  md.B = Bm.w;
  md.C = nullptr;
  md.counts = sums;
  md.M = js.M;
  md.N = (int64_t)js.nbits;
  md.K = js.K;
  md.a_row_words = Am.row_words();
  md.nbatch = js.nbatch;
  md.err = bd.d_err;
  mma_plan(md);
  md.Ab = static_cast<uint8_t*>(bd.alloc((size_t)(md.nbatch * md.M * md.Kp)));
  md.Bb = static_cast<uint8_t*>(bd.alloc((size_t)(md.nbatch * md.N * md.Kp)));
  add_occupancy(bd, md);
  bd.pend_mma.push_back(md);
  bd.st.mma_macs += nb * M * N * (double)js.K;
  bd.st.n_mma++;
  flush_mma(bd);
  if (!natural) {
    const int nd = (int)keep.size();
    std::vector<int64_t> ext(nd), stride(nd);
    for (int a = 0; a < nd; ++a) {
      ext[a] = vres[keep[a]];
      int64_t st = 1;
      bool after = false;
      for (int v : js.c_axes) {
        if (after) st *= vres[v];
        if (v == keep[a]) after = true;
      }
      stride[a] = st;
    }
    Op op;
    op.kind = OP_PERMUTE;
    op.a = reinterpret_cast<const uint64_t*>(sums);
    op.p = reinterpret_cast<uint64_t*>(out);
    op.n = nd;
    op.off0 = bd.put(ext.data(), ext.size(), 16);
    op.off1 = bd.put(stride.data(), stride.size(), 16);
    op.count = total;
    bd.ops.push_back(op);
  }
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

// An expression's program: valid instructions and arguments, a stack that
// never underflows or exceeds PA_EXPR_MAX_STACK and ends with one value.
void check_expr(pa_ctx* ctx, const pa_expr& e, int arity) {
  PA_CHECK_ARG(e.nops >= 1 && e.nops <= PA_EXPR_MAX_OPS && e.ops, "expression: 1..256 instructions");
  PA_CHECK_ARG(e.nconsts >= 0 && e.nconsts <= PA_EXPR_MAX_OPS && (e.nconsts == 0 || e.consts),
               "expression: 0..256 constants");
  for (int i = 0; i < e.nconsts; ++i)
    PA_CHECK_ARG(!isnan(e.consts[i]), "expression: constants must not be NaN");
  int sp = 0;
  for (int k = 0; k < e.nops; ++k) {
    const int op = e.ops[k] & 0xff, arg = e.ops[k] >> 8;
    PA_CHECK_ARG(op <= PA_X_POW, "expression: unknown instruction");
    if (op == PA_X_CONST) PA_CHECK_ARG(arg >= 0 && arg < e.nconsts, "expression: constant index");
    if (op == PA_X_VAR) PA_CHECK_ARG(arg >= 0 && arg < arity, "expression: port index");
    if (op == PA_X_POWI) PA_CHECK_ARG(arg >= -64 && arg <= 64, "expression: integer power in -64..64");
    const int pops = (op == PA_X_CONST || op == PA_X_VAR) ? 0
                     : ((op >= PA_X_ADD && op <= PA_X_DIV) || op == PA_X_POW) ? 2 : 1;
    PA_CHECK_ARG(sp >= pops, "expression: stack underflow");
    sp += 1 - pops;
    PA_CHECK_ARG(sp <= PA_EXPR_MAX_STACK, "expression: more than 16 stack values");
  }
  PA_CHECK_ARG(sp == 1, "expression: must leave exactly one value");
}

void check_relation(pa_ctx* ctx, const pa_relation& r, int32_t nvars) {
  PA_CHECK_ARG(r.arity >= 1 && r.arity <= PA_MAX_DIM, "relation arity must be in 1..8");
  PA_CHECK_ARG(r.rule == PA_RULE_CENTER || r.rule == PA_RULE_CORNER, "relation rule");
  if (r.expr) {
    check_expr(ctx, *r.expr, r.arity);
    PA_CHECK_ARG(r.kind == PA_EQ || r.kind == PA_LE || r.kind == PA_LT, "relation kind");
    PA_CHECK_ARG(r.eps >= 0 && r.eps < INFINITY, "expression relation: eps must be >= 0 and finite");
    for (int p = 0; p < r.arity; ++p)
      PA_CHECK_ARG(r.vars[p] >= 0 && r.vars[p] < nvars, "relation variable out of range");
    return;
  }
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
  if (r.eps >= 0 || r.expr) return r.eps;
  double lo[kMaxDim], hi[kMaxDim];
  int32_t res[kMaxDim];
  for (int p = 0; p < r.arity; ++p) {
    lo[p] = axes[r.vars[p]].lo;
    hi[p] = axes[r.vars[p]].hi;
    res[p] = axes[r.vars[p]].res;
  }
  return valid_tolerance(r.arity, r.degree, r.coeffs, lo, hi, res,
                         r.rule == PA_RULE_CORNER ? 1.0 : 0.5);
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
// One relation to plot: the relation, the axes of its system, where to put it.
struct PlotReq {
  const pa_relation* rel;
  const pa_axis* axes;
  int strict;
  uint64_t* direct;  // plot straight into this array (pa_plot), else workspace
};

std::vector<BitArr> plot_poly(Builder& bd, const std::vector<PlotReq>& reqs);

// The relations plotted by the corner rule (pa.h, pa_rule), polynomial or
// expression, in one launch; their arrays are appended to `plots` at `at`.
void plot_corner(Builder& bd, const std::vector<PlotReq>& reqs, const std::vector<size_t>& at,
                 std::vector<BitArr>& plots) {
  std::vector<CornerJob> jobs;
  std::vector<size_t> a_off, b_off;  // program and constants, or coefficients
  int64_t words = 0;
  for (size_t k = 0; k < reqs.size(); ++k) {
    const pa_relation& r = *reqs[k].rel;
    const pa_axis* axes = reqs[k].axes;
    const std::vector<int> dv = distinct_vars(r);
    BitArr a;
    a.ndim = (int)dv.size();
    a.inner = 1;
    for (int d = 0; d < a.ndim; ++d) {
      a.vars[d] = dv[d];
      a.res[d] = axes[dv[d]].res;
    }
    a.w = reqs[k].direct ? reqs[k].direct : bd.alloc_words(a.words());
    plots[at[k]] = a;
    CornerJob J;
    memset(&J, 0, sizeof J);
    J.out = a.w;
    J.arity = r.arity;
    J.degree = r.degree;
    J.kind = r.kind;
    J.strict = reqs[k].strict;
    J.eps = relation_eps(r, axes);
    J.ndim = a.ndim;
    for (int d = 0; d < a.ndim; ++d) J.res[d] = (int32_t)a.res[d];
    for (int p = 0; p < r.arity; ++p) {
      const pa_axis& ax = axes[r.vars[p]];
      J.port_axis[p] = axis_of(a, r.vars[p]);
      J.lo[p] = ax.lo;
      J.delta[p] = (ax.hi - ax.lo) / (double)ax.res;
    }
    J.nrows = a.nrows();
    J.row_words = a.row_words();
    J.word0 = words;
    words += a.words();
    if (r.expr) {
      J.nops = r.expr->nops;
      a_off.push_back(bd.put(r.expr->ops, (size_t)r.expr->nops));
      b_off.push_back(bd.put(r.expr->consts, (size_t)r.expr->nconsts));
    } else {
      std::vector<int64_t> ord = nest_order(r.arity, r.degree);
      std::vector<double> nc(ord.size());
      for (size_t c = 0; c < ord.size(); ++c) nc[c] = r.coeffs[ord[c]];
      a_off.push_back(0);
      b_off.push_back(bd.put(nc.data(), nc.size()));
    }
    jobs.push_back(J);
    bd.st.pixels_plotted += (double)a.bits();
    bd.st.n_plots++;
  }
  for (size_t k = 0; k < jobs.size(); ++k) {
    if (reqs[k].rel->expr) {
      jobs[k].prog = reinterpret_cast<const int32_t*>(bd.dev(a_off[k]));
      jobs[k].consts = reinterpret_cast<const double*>(bd.dev(b_off[k]));
    } else {
      jobs[k].coeffs = reinterpret_cast<const double*>(bd.dev(b_off[k]));
    }
  }
  Op op;
  op.kind = OP_PLOT_CORNER;
  op.off0 = bd.put(jobs.data(), jobs.size(), 64);
  op.n = (int)jobs.size();
  op.count = words;
  bd.ops.push_back(op);
}

// Every requested plot: the corner-rule relations and the expression relations
// in one launch each (first, so that the polynomial plot launch stays right
// before the contractions), the polynomial ones in the two launches of
// plot_poly.  Arrays come back in the order of `reqs`.
std::vector<BitArr> plot_all(Builder& bd, const std::vector<PlotReq>& reqs) {
  std::vector<BitArr> plots(reqs.size());
  std::vector<PlotReq> poly, corner;
  std::vector<size_t> poly_at, corner_at;
  std::vector<ExprJob> ejobs;
  std::vector<size_t> prog_off, const_off;
  int64_t words = 0;
  for (size_t i = 0; i < reqs.size(); ++i) {
    const pa_relation& r = *reqs[i].rel;
    if (r.rule == PA_RULE_CORNER) {
      corner.push_back(reqs[i]);
      corner_at.push_back(i);
      continue;
    }
    if (!r.expr) {
      poly.push_back(reqs[i]);
      poly_at.push_back(i);
      continue;
    }
    const pa_axis* axes = reqs[i].axes;
    const std::vector<int> dv = distinct_vars(r);
    BitArr a;
    a.ndim = (int)dv.size();
    a.inner = 1;
    for (int k = 0; k < a.ndim; ++k) {
      a.vars[k] = dv[k];
      a.res[k] = axes[dv[k]].res;
    }
    a.w = reqs[i].direct ? reqs[i].direct : bd.alloc_words(a.words());
    plots[i] = a;
    ExprJob J;
    memset(&J, 0, sizeof J);
    J.out = a.w;
    J.arity = r.arity;
    J.kind = r.kind;
    J.strict = reqs[i].strict;
    J.eps = r.eps;
    J.ndim = a.ndim;
    for (int k = 0; k < a.ndim; ++k) J.res[k] = (int32_t)a.res[k];
    for (int p = 0; p < r.arity; ++p) {
      const pa_axis& ax = axes[r.vars[p]];
      J.port_axis[p] = axis_of(a, r.vars[p]);
      J.lo[p] = ax.lo;
      J.delta[p] = (ax.hi - ax.lo) / (double)ax.res;
    }
    J.nops = r.expr->nops;
    J.nrows = a.nrows();
    J.row_words = a.row_words();
    J.word0 = words;
    words += a.words();
    prog_off.push_back(bd.put(r.expr->ops, (size_t)r.expr->nops));
    const_off.push_back(bd.put(r.expr->consts, (size_t)r.expr->nconsts));
    ejobs.push_back(J);
    bd.st.pixels_plotted += (double)a.bits();
    bd.st.n_plots++;
  }
  if (!corner.empty()) plot_corner(bd, corner, corner_at, plots);
  if (!ejobs.empty()) {
    for (size_t k = 0; k < ejobs.size(); ++k) {
      ejobs[k].prog = reinterpret_cast<const int32_t*>(bd.dev(prog_off[k]));
      ejobs[k].consts = reinterpret_cast<const double*>(bd.dev(const_off[k]));
    }
    Op op;
    op.kind = OP_PLOT_EXPR;
    op.off0 = bd.put(ejobs.data(), ejobs.size(), 64);
    op.n = (int)ejobs.size();
    op.count = words;
    bd.ops.push_back(op);
  }
  if (!poly.empty()) {
    const std::vector<BitArr> pp = plot_poly(bd, poly);
    for (size_t k = 0; k < pp.size(); ++k) plots[poly_at[k]] = pp[k];
  }
  return plots;
}

// The polynomial relations' plots in two launches: the FP32 centre tables of
// the last ports (once per distinct axis, not once per block), then the plot
// itself.
std::vector<BitArr> plot_poly(Builder& bd, const std::vector<PlotReq>& reqs) {
  const int nrel = (int)reqs.size();
  std::vector<BitArr> plots;
  std::vector<PlotJob> jobs(nrel);
  std::vector<size_t> coeff_off(nrel);
  // Words per block: the plots' words spread over the blocks the GPU holds
  // at once (so that no second wave of blocks waits for the first), between
  // 256 (enough words to carry a block's set-up: row polynomials, centre
  // table copy) and 2048.
  int64_t tile_words = 2048;
  {
    int64_t words = 0;
    int common = reqs[0].rel->degree;
    for (const PlotReq& q : reqs) {
      const std::vector<int> dv = distinct_vars(*q.rel);
      int64_t nrows = 1;
      for (size_t k = 0; k + 1 < dv.size(); ++k) nrows *= q.axes[dv[k]].res;
      words += nrows * ((q.axes[dv.back()].res + 63) / 64);
      if (q.rel->degree != common) common = -1;
    }
    const int64_t slots = plot_resident_blocks(common >= 1 && common <= 4 ? common : -1);
    tile_words = std::min<int64_t>(2048, std::max<int64_t>(256, (words + slots - 1) / slots));
  }
  int64_t tiles = 0, max_tile_words = 1, ycen = 0;
  std::vector<CentreTab> tabs;  // one per distinct last-port axis of the hoisted jobs
  int max_rows = 1, max_deg = 0, common_deg = reqs[0].rel->degree, max_res_last = 1;
  for (int i = 0; i < nrel; ++i) {
    const pa_relation& r = *reqs[i].rel;
    const pa_axis* axes = reqs[i].axes;
    std::vector<int> dv = distinct_vars(r);
    BitArr a;
    a.ndim = (int)dv.size();
    a.inner = 1;
    for (int k = 0; k < a.ndim; ++k) {
      a.vars[k] = dv[k];
      a.res[k] = axes[dv[k]].res;
    }
    a.w = reqs[i].direct ? reqs[i].direct : bd.alloc_words(a.words());
    plots.push_back(a);
    // coefficients in nest order
    std::vector<int64_t> ord = nest_order(r.arity, r.degree);
    std::vector<double> nc(ord.size());
    for (size_t k = 0; k < ord.size(); ++k) nc[k] = r.coeffs[ord[k]];
    coeff_off[i] = bd.put(nc.data(), nc.size());

    PlotJob& J = jobs[i];
    memset(&J, 0, sizeof J);
    J.out = a.w;
    J.arity = r.arity;
    J.degree = r.degree;
    J.kind = r.kind;
    J.strict = reqs[i].strict;
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
    if (J.hoisted) {
      const int a = r.arity - 1;
      const CentreTab* t = nullptr;
      for (const CentreTab& c : tabs)
        if (c.lo == J.lo[a] && c.delta == J.delta[a] && c.res == res_last) t = &c;
      if (!t) {
        CentreTab c;
        c.y32 = reinterpret_cast<float*>(bd.alloc_words((res_last + 1) / 2));
        c.lo = J.lo[a];
        c.delta = J.delta[a];
        c.item0 = ycen;
        c.res = res_last;
        ycen += res_last;
        tabs.push_back(c);
        t = &tabs.back();
      }
      J.y32 = t->y32;
    }
    {
      const pa_axis& ax = axes[r.vars[r.arity - 1]];
      J.ymax = (float)(fmax(fabs(ax.lo), fabs(ax.hi)) * (1.0 + 0x1p-20));
      J.hword = (float)(32.0 * ((ax.hi - ax.lo) / (double)ax.res) * 1.01);
      // coefficients with e_last = j form block j of the nest order; its size is
      // the number of monomials of arity-1 variables of degree <= D - j
      int32_t off = 0;
      for (int j = 0; j <= r.degree; ++j) {
        J.block_off[j] = off;
        off += (int32_t)coeff_count(r.arity - 1, r.degree - j);
      }
    }
    J.rows_per_tile = (int32_t)std::max<int64_t>(
        1, std::min<int64_t>(256, (tile_words + J.row_words - 1) / J.row_words));
    J.tile0 = tiles;
    tiles += (J.nrows + J.rows_per_tile - 1) / J.rows_per_tile;
    max_rows = std::max(max_rows, J.rows_per_tile);
    max_tile_words = std::max<int64_t>(max_tile_words, (int64_t)J.rows_per_tile * J.row_words);
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
    bd.st.pixels_plotted += (double)a.bits();
    bd.st.n_plots++;
  }
  if (tiles > 0x7fffffffLL) bd.fail(PA_ERR_TOO_LARGE, "plot grid too large");
  for (int i = 0; i < nrel; ++i)
    jobs[i].coeffs = reinterpret_cast<const double*>(bd.dev(coeff_off[i]));
  const size_t jobs_off = bd.put(jobs.data(), jobs.size(), 64);
  if (ycen > 0) {
    Op cop;
    cop.kind = OP_CENTRES;
    cop.off0 = bd.put(tabs.data(), tabs.size(), 64);
    cop.n = (int)tabs.size();
    cop.count = ycen;
    bd.ops.push_back(cop);
  }
  Op op;
  op.kind = OP_PLOT;
  op.off0 = jobs_off;
  op.n = nrel;
  op.count = tiles;
  op.i0 = max_rows;
  op.i1 = max_deg;
  op.i2 = common_deg;
  op.i3 = max_res_last;
  op.m = max_tile_words;
  bd.ops.push_back(op);
  return plots;
}

// ------------------------------------------------------- networks
struct Network {
  int32_t nvars;
  const pa_axis* axes;
  int32_t nrel;
  const pa_relation* rels;
  std::vector<int> exposed;
  int strict;
  int order;
  const int32_t* pairs;
  BitArr target;
  std::vector<int32_t> own_pairs;  // orders chosen by the learned planner
  std::vector<double> dens_cache;  // estimated plot densities (both passes of a call share them)
  std::vector<uint64_t> slot_keys;  // per slot: key of the relations and kept variables below it
  Plan plan;                        // the join order, planned once for both passes of a call
  bool planned = false;
};

// Run f(i) for i in [0, n) on up to `threads` host threads (contiguous
// shares; f must not touch shared state).
template <class F>
void parallel_for(size_t n, size_t min_per_thread, F&& f) {
  const size_t hw = std::max<unsigned>(1u, std::thread::hardware_concurrency());
  const size_t nt = std::min<size_t>(std::min<size_t>(hw, 32), (n + min_per_thread - 1) /
                                                                   std::max<size_t>(1, min_per_thread));
  if (nt <= 1) {
    for (size_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> pool;
  for (size_t t = 0; t < nt; ++t)
    pool.emplace_back([&, t]() {
      for (size_t i = n * t / nt; i < n * (t + 1) / nt; ++i) f(i);
    });
  for (auto& th : pool) th.join();
}

// The join order of every network not planned yet, in parallel (planning
// reads only the network's own shapes).
void plan_networks(std::vector<Network>& nets) {
  std::vector<size_t> todo;
  bool heavy = false;
  for (size_t k = 0; k < nets.size(); ++k)
    if (!nets[k].planned) {
      todo.push_back(k);
      heavy = heavy || nets[k].order == PA_ORDER_OPTIMAL;
    }
  parallel_for(todo.size(), heavy ? 1 : 256, [&](size_t i) {
    Network& n = nets[todo[i]];
    std::vector<double> vresd(n.nvars);
    for (int v = 0; v < n.nvars; ++v) vresd[v] = n.axes[v].res;
    std::vector<std::vector<int>> rv;
    for (int r = 0; r < n.nrel; ++r) {
      std::vector<int> d;
      for (int p = 0; p < n.rels[r].arity; ++p)
        if (std::find(d.begin(), d.end(), n.rels[r].vars[p]) == d.end()) d.push_back(n.rels[r].vars[p]);
      rv.push_back(d);
    }
    n.plan = plan_joins(n.nvars, vresd, rv, n.exposed, n.order, n.pairs);
    n.planned = true;
  });
}

std::vector<double> plot_densities(const Network& n, pa_ctx* ctx);
uint64_t relation_key(const pa_relation& r, const pa_axis* axes);
uint64_t mix64(uint64_t z);

// Key of a join's result: its two operands' keys (in either order) and the
// variables it keeps.
uint64_t subtree_key(uint64_t ka, uint64_t kb, const std::vector<int>& keep) {
  uint64_t h = mix64(std::min(ka, kb) ^ 0x5bd1e995ull) ^ (std::max(ka, kb) * 0x9E3779B97F4A7C15ull);
  for (int v : keep) h = mix64(h ^ (uint64_t)(uint32_t)v);
  return h;
}

// Clear every memset target of the program in the plot launch that opens it
// instead of in memsets of their own: a memset between two launches ends
// their programmatic overlap and costs a launch.  Valid because every memset
// target is a result buffer that no op before its contraction touches (the
// workspace is handed out once per call, and the output array is written only
// by the program's last joins), and every contraction waits for the plot
// launch to complete.
void fold_memsets(Builder& bd) {
  size_t plot_at = bd.ops.size();
  for (size_t i = 0; i < bd.ops.size() && plot_at == bd.ops.size(); ++i)
    if (bd.ops[i].kind == OP_PLOT) plot_at = i;
  if (plot_at == bd.ops.size()) return;
  std::vector<ZeroRange> zr;
  int64_t total = 0;
  std::vector<Op> kept;
  for (size_t i = 0; i < bd.ops.size(); ++i) {
    const Op& op = bd.ops[i];
    if (op.kind == OP_MEMSET && i > plot_at) {
      zr.push_back({op.p, op.count, total});
      total += op.count;
    } else {
      kept.push_back(op);
    }
  }
  if (zr.empty()) return;
  if (zr.size() > 0x7fffffff) bd.fail(PA_ERR_TOO_LARGE, "too many result buffers to clear");
  bd.ops.swap(kept);
  Op& pop = bd.ops[plot_at];
  pop.off1 = bd.put(zr.data(), zr.size(), 64);
  pop.nw = (int64_t)zr.size();
  pop.zw = total;
}

// Plots of all networks in one launch pair, then their joins level by level:
// the joins of one level of every network's cluster tree are independent and
// share one contraction launch per tile width.
void build_networks(Builder& bd, std::vector<Network>& nets, bool one_join_per_launch = false,
                    std::vector<BitArr>* join_results = nullptr) {
  std::vector<PlotReq> reqs;
  for (auto& n : nets)
    for (int i = 0; i < n.nrel; ++i) reqs.push_back({&n.rels[i], n.axes, n.strict, nullptr});
  std::vector<BitArr> plots = plot_all(bd, reqs);
  plan_networks(nets);

  struct State {
    Plan plan;
    std::vector<int64_t> vres;
    std::vector<BitArr> slots;
    std::vector<int> level;
    std::vector<double> dens;  // estimated slot densities (empty: not needed)
  };
  std::vector<State> S(nets.size());
  int max_level = 0;
  size_t pidx = 0;
  for (size_t k = 0; k < nets.size(); ++k) {
    Network& n = nets[k];
    State& s = S[k];
    s.vres.resize(n.nvars);
    std::vector<double> vresd(n.nvars);
    for (int v = 0; v < n.nvars; ++v) {
      s.vres[v] = n.axes[v].res;
      vresd[v] = n.axes[v].res;
    }
    s.plan = n.plan;
    for (int i = 0; i < n.nrel; ++i) s.slots.push_back(plots[pidx++]);
    const int nj = (int)s.plan.joins.size();
    s.slots.resize(n.nrel + nj);
    s.level.assign(n.nrel + nj, 0);
    bool large = false;
    for (int t = 0; t < nj; ++t) {
      const Join& jn = s.plan.joins[t];
      s.level[n.nrel + t] = 1 + std::max(s.level[jn.a], s.level[jn.b]);
      max_level = std::max(max_level, s.level[n.nrel + t]);
      large = large || jn.cost >= 134217728.0;
    }
    // the automatic path choice weighs densities, estimated only where a
    // cluster is large enough for the tensor-core path to be considered
    if (large && bd.ctx && bd.ctx->path == PA_PATH_AUTO) {
      if (n.dens_cache.empty()) n.dens_cache = plot_densities(n, bd.ctx);
      s.dens = n.dens_cache;
      s.dens.resize(n.nrel + nj, -1.0);
    }
    if (bd.ctx && (!s.dens.empty() || join_results)) {
      n.slot_keys.assign(n.nrel + nj, 0);
      for (int i = 0; i < n.nrel; ++i) n.slot_keys[i] = relation_key(n.rels[i], n.axes);
      for (int t = 0; t < nj; ++t) {
        const Join& jn = s.plan.joins[t];
        n.slot_keys[n.nrel + t] = subtree_key(n.slot_keys[jn.a], n.slot_keys[jn.b], jn.keep);
      }
    }
  }
  for (int lv = 1; lv <= max_level; ++lv) {
    int n_in_level = 0;
    for (size_t k = 0; k < nets.size(); ++k)
      for (size_t t = 0; t < S[k].plan.joins.size(); ++t)
        n_in_level += (S[k].level[nets[k].nrel + t] == lv);
    // The row-OR joins of a level share one launch; each gets a share of one
    // wave of 152 CTAs in proportion to its estimated time, so a large join
    // among many small ones is split over many CTAs instead of setting the
    // launch's length alone.
    std::map<std::pair<size_t, int>, int64_t> target_of;
    {
      std::vector<std::pair<std::pair<size_t, int>, double>> work;
      double total = 0.0;
      for (size_t k = 0; k < nets.size(); ++k) {
        const State& s = S[k];
        const int nrel = nets[k].nrel;
        for (int t = 0; t < (int)s.plan.joins.size(); ++t) {
          if (s.level[nrel + t] != lv) continue;
          const Join& jn = s.plan.joins[t];
          const JoinShape js = analyze_join(s.slots[jn.a], s.slots[jn.b], jn.keep, s.vres);
          double w = 0.0;
          if (!js.hadamard && !js.outer && !js.dot) {
            double ra = 0.05;
            if (!s.dens.empty() && s.dens[jn.a] >= 0 && s.dens[jn.b] >= 0)
              ra = or_density(js.swap ? s.dens[jn.b] : s.dens[jn.a], js.private_a);
            w = rowor_cost_us(bd.ctx, js, ra);
          }
          work.push_back({{k, t}, w});
          total += w;
        }
      }
      for (const auto& e : work)
        target_of[e.first] =
            total > 0 ? std::max<int64_t>(1, (int64_t)(152.0 * e.second / total)) : 1;
    }
    bd.defer = !one_join_per_launch;
    for (size_t k = 0; k < nets.size(); ++k) {
      State& s = S[k];
      const int nrel = nets[k].nrel, nj = (int)s.plan.joins.size();
      for (int t = 0; t < nj; ++t) {
        if (s.level[nrel + t] != lv) continue;
        const Join& jn = s.plan.joins[t];
        const bool last = (t + 1 == nj);
        const size_t first_op = bd.ops.size();
        const bool dn = !s.dens.empty();
        s.slots[nrel + t] = join(bd, s.slots[jn.a], s.slots[jn.b], jn.keep, s.vres,
                                 last ? &nets[k].target : nullptr,
                                 one_join_per_launch ? 152 : target_of[{k, t}],
                                 dn ? s.dens[jn.a] : -1.0, dn ? s.dens[jn.b] : -1.0,
                                 dn ? &s.dens[nrel + t] : nullptr);
        if (dn) {
          // a density measured by pa_join_log beats the independence estimate
          auto it = bd.ctx->obs_dens.find(nets[k].slot_keys[nrel + t]);
          if (it != bd.ctx->obs_dens.end()) s.dens[nrel + t] = it->second;
        }
        if (one_join_per_launch) {
          flush_rowor(bd);
          for (size_t q = first_op; q < bd.ops.size(); ++q) bd.ops[q].join = t;
          if (join_results) join_results->push_back(s.slots[nrel + t]);
        }
      }
    }
    flush_level(bd);
    bd.defer = false;
  }
  // the final reshapes into the callers' arrays: one launch per kind for all
  // systems
  bd.defer = !one_join_per_launch;
  for (size_t k = 0; k < nets.size(); ++k) {
    const BitArr& root = S[k].slots[S[k].plan.root];
    if (root.w != nets[k].target.w) reshape(bd, root, nets[k].target);
  }
  flush_level(bd);
  bd.defer = false;
  if (!one_join_per_launch) fold_memsets(bd);
}

// ------------------------------------------------------------ running
cudaEvent_t next_event(pa_ctx* ctx) {
  if (ctx->ev_used == ctx->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) throw Fail{set_err(ctx, PA_ERR_CUDA, "cudaEventCreate")};
    ctx->ev_pool.push_back(e);
  }
  return ctx->ev_pool[ctx->ev_used++];
}

void check_cuda(pa_ctx* ctx, cudaError_t e, const char* what) {
  if (e != cudaSuccess)
    throw Fail{set_err(ctx, PA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e))};
}

// Launch the ops of a program whose blob lives at device address `blob`.
void run_ops(pa_ctx* ctx, const std::vector<Op>& ops, char* blob, cudaStream_t s, bool timing) {
  for (const Op& op : ops) {
    pa_ctx::Rec rec;
    if (timing) {
      rec.name = op_name(op);
      rec.a = next_event(ctx);
      rec.b = next_event(ctx);
      check_cuda(ctx, cudaEventRecord(rec.a, s), "cudaEventRecord");
    }
    switch (op.kind) {
      case OP_PLOT:
        launch_plot(reinterpret_cast<const PlotJob*>(blob + op.off0), op.n, op.count, op.i0,
                    op.i1, op.i2, op.i3, op.m, reinterpret_cast<const ZeroRange*>(blob + op.off1),
                    (int)op.nw, op.zw, s);
        break;
      case OP_EWISE:
        launch_ewise(reinterpret_cast<const EwJob*>(blob + op.off0),
                     reinterpret_cast<const int64_t*>(blob + op.off1), op.n, op.count, s);
        break;
      case OP_PERMUTE:
        launch_permute_u32(reinterpret_cast<const uint32_t*>(op.a), reinterpret_cast<uint32_t*>(op.p),
                           op.n, reinterpret_cast<const int64_t*>(blob + op.off0),
                           reinterpret_cast<const int64_t*>(blob + op.off1), op.count, s);
        break;
      case OP_PLOT_EXPR:
        launch_plot_expr(reinterpret_cast<const ExprJob*>(blob + op.off0), op.n, op.count, s);
        break;
      case OP_PLOT_CORNER:
        launch_plot_corner(reinterpret_cast<const CornerJob*>(blob + op.off0), op.n, op.count, s);
        break;
      case OP_CENTRES:
        launch_plot_centres(reinterpret_cast<const CentreTab*>(blob + op.off0), op.n, op.count, s);
        break;
      case OP_MEMSET:
        check_cuda(ctx, cudaMemsetAsync(op.p, 0, (size_t)op.count * 8, s), "cudaMemsetAsync");
        break;
      case OP_RESHAPE:
        launch_reshape(reinterpret_cast<const ReshapeDesc*>(blob + op.off0),
                       reinterpret_cast<const int64_t*>(blob + op.off1), op.n, op.i0, op.count, s);
        break;
      case OP_UNPACK:
        launch_unpack(reinterpret_cast<const MmaDesc*>(blob + op.off0), op.n, op.m, op.nw, s);
        break;
      case OP_MMA:
        check_cuda(ctx,
                   launch_mma(reinterpret_cast<const MmaDesc*>(blob + op.off0),
                              reinterpret_cast<const CUtensorMap*>(blob + op.off1),
                              reinterpret_cast<const int64_t*>(blob + op.off2), op.n, op.count, s),
                   "mma_bool_kernel");
        break;
      case OP_ROWOR:
        check_cuda(ctx,
                   launch_rowor(reinterpret_cast<const RowOrDesc*>(blob + op.off0),
                                reinterpret_cast<const CUtensorMap*>(blob + op.off1),
                                reinterpret_cast<const int64_t*>(blob + op.off2), op.n, op.count,
                                op.smem, op.i0, s),
                   "rowor_kernel");
        break;
    }
    check_cuda(ctx, cudaGetLastError(), op_name(op));
    if (timing) {
      check_cuda(ctx, cudaEventRecord(rec.b, s), "cudaEventRecord");
      ctx->recs.push_back(rec);
    }
  }
}

pa_status ensure_arena(pa_ctx* ctx, size_t need) {
  if (need <= ctx->arena_size) return PA_OK;
  if (ctx->cap && need > ctx->cap) {
    return set_err(ctx, PA_ERR_OOM, "workspace of " + std::to_string(need) +
                                        " bytes exceeds the context's cap");
  }
  for (int i = 0; i < pa_ctx::kNStage; ++i)
    if (ctx->stage_pending[i]) {
      cudaEventSynchronize(ctx->stage_done[i]);
      ctx->stage_pending[i] = false;
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

// Copy the blob into the arena through the pinned stage, on the stream.
void upload_blob(pa_ctx* ctx, const std::vector<char>& blob, cudaStream_t s) {
  if (blob.empty()) return;
  const int i = ctx->stage_next;
  ctx->stage_next = (i + 1) % pa_ctx::kNStage;
  if (ctx->stage_pending[i]) {
    check_cuda(ctx, cudaEventSynchronize(ctx->stage_done[i]), "cudaEventSynchronize");
    ctx->stage_pending[i] = false;
  }
  if (ctx->h_stage_size[i] < blob.size()) {
    if (ctx->h_stage[i]) cudaFreeHost(ctx->h_stage[i]);
    ctx->h_stage[i] = nullptr;
    ctx->h_stage_size[i] = 0;
    const size_t sz = std::max<size_t>(blob.size() * 2, 1 << 16);
    check_cuda(ctx, cudaMallocHost(reinterpret_cast<void**>(&ctx->h_stage[i]), sz),
               "cudaMallocHost");
    ctx->h_stage_size[i] = sz;
  }
  memcpy(ctx->h_stage[i], blob.data(), blob.size());
  check_cuda(ctx,
             cudaMemcpyAsync(ctx->arena, ctx->h_stage[i], blob.size(), cudaMemcpyHostToDevice, s),
             "cudaMemcpyAsync");
  check_cuda(ctx, cudaEventRecord(ctx->stage_done[i], s), "cudaEventRecord");
  ctx->stage_pending[i] = true;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Size, build and run one call on the context's arena.
template <class F>
pa_status run_call(pa_ctx* ctx, cudaStream_t s, pa_stats* stats, F&& body,
                   std::vector<char>* memo_key = nullptr) {
  try {
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, PA_ERR_CUDA, "cudaSetDevice failed");
    }
    Builder dry(ctx, true, nullptr, 0);
    body(dry);
    const size_t blob_cap = round_up(dry.blob.size() + 64, kAlign);
    const size_t need = dry.used + blob_cap + kAlign;
    pa_status st = ensure_arena(ctx, need);
    if (st != PA_OK) return st;
    Builder bd(ctx, false, ctx->arena, blob_cap);
    bd.d_err = ctx->d_err;
    bd.d_stat = ctx->prof ? ctx->d_stat : nullptr;
    body(bd);
    if (bd.blob.size() > blob_cap) return set_err(ctx, PA_ERR_CUDA, "internal: blob grew");
    upload_blob(ctx, bd.blob, s);
    run_ops(ctx, bd.ops, ctx->arena, s, ctx->prof);
    bd.st.workspace_bytes = (int64_t)bd.used;
    bd.st.n_launches = (int32_t)bd.ops.size();
    if (stats) *stats = bd.st;
    if (memo_key) {
      // a new program: the old one's graph goes with it (an executable graph
      // still running is freed when it completes)
      delete ctx->memo;
      ctx->memo = new Memo();
      Memo& m = *ctx->memo;
      m.key.swap(*memo_key);
      m.ops = std::move(bd.ops);
      m.blob = std::move(bd.blob);
      m.st = bd.st;
    }
    return PA_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

template <class T>
void put_val(std::vector<char>& k, const T& v) {
  const char* p = reinterpret_cast<const char*>(&v);
  k.insert(k.end(), p, p + sizeof v);
}
void put_bytes(std::vector<char>& k, const void* p, size_t n) {
  const char* c = static_cast<const char*>(p);
  k.insert(k.end(), c, c + n);
}

// Everything a validated pa_solve_network call's program depends on: each
// argument by value (coefficients included), the stream, and the context
// state that steers planning or is written into the program.
std::vector<char> solve_key(pa_ctx* ctx, int32_t nvars, const pa_axis* axes, int32_t nrel,
                            const pa_relation* rels, int32_t nexposed, const int32_t* exposed,
                            const pa_options* opts, const pa_array* out, void* stream) {
  std::vector<char> k;
  k.reserve(512);
  put_val(k, ctx->plan_epoch);
  put_val(k, reinterpret_cast<uintptr_t>(ctx->arena));
  put_val(k, ctx->prof);
  put_val(k, reinterpret_cast<uintptr_t>(stream));
  put_val(k, nvars);
  for (int i = 0; i < nvars; ++i) {
    put_val(k, axes[i].lo);
    put_val(k, axes[i].hi);
    put_val(k, axes[i].res);
  }
  put_val(k, nrel);
  for (int i = 0; i < nrel; ++i) {
    const pa_relation& r = rels[i];
    put_val(k, r.arity);
    put_bytes(k, r.vars, sizeof(int32_t) * r.arity);
    put_val(k, r.degree);
    put_val(k, r.kind);
    put_val(k, r.eps);
    put_val(k, r.rule);
    if (r.expr) {
      put_val(k, r.expr->nops);
      put_bytes(k, r.expr->ops, sizeof(int32_t) * r.expr->nops);
      put_val(k, r.expr->nconsts);
      put_bytes(k, r.expr->consts, sizeof(double) * r.expr->nconsts);
    } else {
      put_val(k, (int32_t)-1);
      put_bytes(k, r.coeffs, sizeof(double) * coeff_count(r.arity, r.degree));
    }
  }
  put_val(k, nexposed);
  put_bytes(k, exposed, sizeof(int32_t) * nexposed);
  put_val(k, opts ? opts->strict : 0);
  put_val(k, opts ? opts->order : 0);
  if (opts && opts->order == PA_ORDER_GIVEN) {
    put_val(k, opts->npairs);
    put_bytes(k, opts->pairs, sizeof(int32_t) * 2 * opts->npairs);
  }
  put_val(k, reinterpret_cast<uintptr_t>(out->words));
  return k;
}

// Relaunch the kept program.  Its blob is uploaded again like any call's: the
// coefficients are host inputs of every call, and another call may have
// replaced the blob region of the arena since.
pa_status run_memo(pa_ctx* ctx, cudaStream_t s, pa_stats* stats) {
  try {
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
      cudaGetLastError();
      return set_err(ctx, PA_ERR_CUDA, "cudaSetDevice failed");
    }
    Memo& m = *ctx->memo;
    upload_blob(ctx, m.blob, s);
    if (ctx->prof || m.capture_failed) {
      // per-launch timing needs the launches one by one
      run_ops(ctx, m.ops, ctx->arena, s, ctx->prof);
    } else {
      if (!m.exec) {
        // capture the launches once, on a stream of their own
        cudaStream_t cs = nullptr;
        bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
          try {
            run_ops(ctx, m.ops, ctx->arena, cs, false);
          } catch (const Fail&) {
            ok = false;
          }
          cudaGraph_t g = nullptr;
          ok = (cudaStreamEndCapture(cs, &g) == cudaSuccess) && ok;
          m.graph = g;
          ok = ok && g && cudaGraphInstantiate(&m.exec, g, 0) == cudaSuccess;
        }
        if (cs) cudaStreamDestroy(cs);
        if (!ok) {
          cudaGetLastError();
          if (m.exec) cudaGraphExecDestroy(m.exec);
          m.exec = nullptr;
          m.capture_failed = true;
          run_ops(ctx, m.ops, ctx->arena, s, false);
          if (stats) *stats = m.st;
          return PA_OK;
        }
      }
      check_cuda(ctx, cudaGraphLaunch(m.exec, s), "cudaGraphLaunch");
    }
    if (stats) *stats = m.st;
    return PA_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

// Validate one network and turn it into a Network record.
void check_network(pa_ctx* ctx, int32_t nvars, const pa_axis* axes, int32_t nrel,
                   const pa_relation* rels, int32_t nexposed, const int32_t* exposed,
                   const pa_options* opts, pa_array* out, Network& n) {
  check_axes(ctx, nvars, axes);
  PA_CHECK_ARG(nrel >= 1 && rels, "at least one relation");
  for (int i = 0; i < nrel; ++i) check_relation(ctx, rels[i], nvars);
  PA_CHECK_ARG(nexposed >= 0 && nexposed <= PA_MAX_DIM && (nexposed == 0 || exposed),
               "exposed: 0..8 variables");
  check_array(ctx, out, "out");
  PA_CHECK_ARG(out->ndim == nexposed, "out: ndim must equal nexposed");
  n.exposed.clear();
  for (int i = 0; i < nexposed; ++i) {
    PA_CHECK_ARG(exposed[i] >= 0 && exposed[i] < nvars, "exposed: variable out of range");
    for (int j = 0; j < i; ++j) PA_CHECK_ARG(exposed[j] != exposed[i], "exposed: repeated");
    PA_CHECK_ARG(out->vars[i] == exposed[i] && out->res[i] == axes[exposed[i]].res,
                 "out: vars/res must match the exposed variables");
    n.exposed.push_back(exposed[i]);
  }
  n.order = opts ? opts->order : PA_ORDER_GREEDY;
  PA_CHECK_ARG(n.order == PA_ORDER_GREEDY || n.order == PA_ORDER_GIVEN || n.order == PA_ORDER_LEFT ||
                   n.order == PA_ORDER_LEARNED || n.order == PA_ORDER_OPTIMAL,
               "opts: unknown order");
  PA_CHECK_ARG(n.order != PA_ORDER_LEARNED || opts->model, "opts: PA_ORDER_LEARNED needs a model");
  n.pairs = nullptr;
  if (n.order == PA_ORDER_GIVEN) {
    PA_CHECK_ARG(plan_valid_given(nrel, opts->npairs, opts->pairs),
                 "opts: pairs must be nrel-1 joins of distinct live slots");
    n.pairs = opts->pairs;
  }
  n.strict = (opts && opts->strict) ? 1 : 0;
  n.nvars = nvars;
  n.axes = axes;
  n.nrel = nrel;
  n.rels = rels;
  n.target = from_pa(*out);
}


// ------------------------------------------------------------ learned order
// Everything the cost model sees is computed here, on the host, from shapes and
// estimated densities, so that planning never waits for the solve.
constexpr int kFeat = PA_FEATURES;

uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double nest_host(int k, int rem, const double*& cp, const double* x) {
  if (k < 0) return *cp++;
  double s = 0.0, pw = 1.0;
  for (int e = 0; e <= rem; ++e) {
    s += nest_host(k - 1, rem - e, cp, x) * pw;
    pw *= x[k];
  }
  return s;
}

// Fraction of pixels a plot turns on, estimated from 512 sampled pixel centres:
// for f = 0 by a Gaussian kernel estimate of the density of f(c) at 0 (times
// the width 2 eps of the accepted band), for f <= 0 / f < 0 by counting.
// An expression relation at one point (host; only density estimates use it,
// so the math library's last bits do not matter here).
double expr_host(const pa_expr& e, const double* x) {
  double st[PA_EXPR_MAX_STACK];
  int sp = 0;
  for (int k = 0; k < e.nops; ++k) {
    const int op = e.ops[k] & 0xff, arg = e.ops[k] >> 8;
    if (op == PA_X_CONST) { st[sp++] = e.consts[arg]; continue; }
    if (op == PA_X_VAR) { st[sp++] = x[arg]; continue; }
    if ((op >= PA_X_ADD && op <= PA_X_DIV) || op == PA_X_POW) {
      const double b = st[--sp], a = st[sp - 1];
      st[sp - 1] = op == PA_X_ADD ? a + b : op == PA_X_SUB ? a - b : op == PA_X_MUL ? a * b
                   : op == PA_X_DIV ? a / b : pow(a, b);
      continue;
    }
    const double a = st[sp - 1];
    double r = NAN;
    switch (op) {
      case PA_X_NEG: r = -a; break;
      case PA_X_ABS: r = fabs(a); break;
      case PA_X_SQRT: r = sqrt(a); break;
      case PA_X_EXP: r = exp(a); break;
      case PA_X_LOG: r = log(a); break;
      case PA_X_SIN: r = sin(a); break;
      case PA_X_COS: r = cos(a); break;
      case PA_X_TAN: r = tan(a); break;
      case PA_X_SINH: r = sinh(a); break;
      case PA_X_COSH: r = cosh(a); break;
      case PA_X_TANH: r = tanh(a); break;
      case PA_X_ATAN: r = atan(a); break;
      case PA_X_POWI: r = pow(a, (double)arg); break;
    }
    st[sp - 1] = r;
  }
  return st[0];
}

double estimate_density(const pa_relation& r, const pa_axis* axes, double eps) {
  const int S = 512;
  std::vector<int64_t> ord;
  if (!r.expr) ord = nest_order(r.arity, r.degree);
  std::vector<double> nc(ord.size());
  for (size_t k = 0; k < ord.size(); ++k) nc[k] = r.coeffs[ord[k]];
  std::vector<double> f(S);
  uint64_t seed = 0x160900061ull;
  for (int p = 0; p < r.arity; ++p) seed = mix64(seed ^ (uint64_t)axes[r.vars[p]].res);
  for (int i = 0; i < S; ++i) {
    double x[kMaxDim];
    for (int p = 0; p < r.arity; ++p) {
      const pa_axis& ax = axes[r.vars[p]];
      const int64_t idx = (int64_t)(mix64(seed + (uint64_t)i * 16 + p) % (uint64_t)ax.res);
      x[p] = ax.lo + ((double)idx + 0.5) * ((ax.hi - ax.lo) / (double)ax.res);
    }
    if (r.expr) {
      f[i] = expr_host(*r.expr, x);
    } else {
      const double* cp = nc.data();
      f[i] = nest_host(r.arity - 1, r.degree, cp, x);
    }
  }
  // non-finite values (undefined points) are off and stay out of the estimate
  f.erase(std::remove_if(f.begin(), f.end(), [](double v) { return !std::isfinite(v); }), f.end());
  if (f.empty()) return 1e-6;
  int direct = 0;
  for (double v : f)
    direct += (r.kind == PA_EQ) ? (fabs(v) <= eps) : (v <= eps);
  double est = (double)direct / S;
  if (r.kind == PA_EQ) {
    // the kernel estimate over the finite samples, scaled by their share
    const double n = (double)f.size();
    double mean = 0, var = 0;
    for (double v : f) mean += v;
    mean /= n;
    for (double v : f) var += (v - mean) * (v - mean);
    const double sd = sqrt(var / n);
    const double h = std::max(1e-300, 1.06 * sd * pow(n, -0.2));
    double acc = 0;
    for (double v : f) acc += exp(-0.5 * (v / h) * (v / h));
    const double pdf0 = acc / (S * h * sqrt(2.0 * M_PI));
    est = std::max(est, std::min(1.0, 2.0 * eps * pdf0));
  }
  return std::min(1.0, std::max(est, 1e-6));
}

// fraction of set bits after OR-ing `n` independent entries of density rho
double or_density(double rho, double n) {
  if (rho >= 1.0) return 1.0;
  return 1.0 - exp(n * log1p(-rho));
}

double lg2(double v) { return log2(std::max(v, 1e-30)); }

// The cost model's inputs for one join, and the estimated density of its result.
void join_features(const JoinShape& js, double rx, double ry, float* f, double* rho_out) {
  double ra = js.swap ? ry : rx, rb = js.swap ? rx : ry;
  ra = or_density(ra, js.private_a);
  rb = or_density(rb, js.private_b);
  double rc, work, m, n, k, batch;
  if (js.hadamard) {
    rc = ra * rb;
    m = 1, n = js.result_bits, k = 1, batch = 1;
    work = js.result_bits / 64.0;
  } else {
    rc = or_density(ra * rb, (double)js.K);
    m = (double)js.M, n = js.nbits, k = (double)js.K, batch = (double)js.nbatch;
    work = ra * m * k * batch * ceil(n / 64.0);
  }
  f[0] = (float)(lg2(m) / 16);
  f[1] = (float)(lg2(n) / 16);
  f[2] = (float)(lg2(k) / 16);
  f[3] = (float)(lg2(batch) / 16);
  f[4] = (float)(lg2(1 + js.reshape_bits) / 32);
  f[5] = (float)(lg2(js.cost) / 48);
  f[6] = (float)(lg2(js.result_bits) / 32);
  f[7] = (float)ra;
  f[8] = (float)rb;
  f[9] = (float)(lg2(ra + 1e-9) / 30);
  f[10] = (float)(lg2(rb + 1e-9) / 30);
  f[11] = (float)(lg2(1 + work) / 40);
  f[12] = (float)(lg2(1 + rc * js.result_bits) / 32);
  f[13] = js.hadamard ? 1.0f : 0.0f;
  f[14] = (float)(lg2(js.private_a * js.private_b) / 32);
  f[15] = 1.0f;
  if (rho_out) *rho_out = rc;
}

struct SimResult {
  std::vector<float> feats;  // one row of kFeat per join
  double peak_bits = 0;
};

// Walk a plan on the host: layouts as join() would build them, densities
// propagated from the plot estimates.
SimResult simulate_plan(const Network& n, const Plan& plan, const std::vector<double>& plot_dens) {
  SimResult r;
  std::vector<int64_t> vres(n.nvars);
  for (int v = 0; v < n.nvars; ++v) vres[v] = n.axes[v].res;
  std::vector<BitArr> slots;
  std::vector<double> dens;
  for (int i = 0; i < n.nrel; ++i) {
    std::vector<int> dv = distinct_vars(n.rels[i]);
    slots.push_back(make_arr(dv, vres, 1));
    dens.push_back(plot_dens[i]);
  }
  for (const Join& jn : plan.joins) {
    const JoinShape js = analyze_join(slots[jn.a], slots[jn.b], jn.keep, vres);
    float f[kFeat];
    double rc = 0;
    join_features(js, dens[jn.a], dens[jn.b], f, &rc);
    r.feats.insert(r.feats.end(), f, f + kFeat);
    r.peak_bits = std::max(r.peak_bits, js.result_bits);
    slots.push_back(join_result_layout(js, jn.keep, vres));
    dens.push_back(rc);
  }
  return r;
}

// Subtree key of every join of a plan (the keys build_networks gives slots).
std::vector<uint64_t> plan_keys(const Network& n, const Plan& plan) {
  std::vector<uint64_t> k(n.nrel + plan.joins.size());
  for (int i = 0; i < n.nrel; ++i) k[i] = relation_key(n.rels[i], n.axes);
  for (size_t t = 0; t < plan.joins.size(); ++t) {
    const Join& jn = plan.joins[t];
    k[n.nrel + t] = subtree_key(k[jn.a], k[jn.b], jn.keep);
  }
  return std::vector<uint64_t>(k.begin() + n.nrel, k.end());
}

Plan plan_of(const Network& n, int order, const int32_t* pairs, uint64_t policy) {
  std::vector<double> vresd(n.nvars);
  for (int v = 0; v < n.nvars; ++v) vresd[v] = n.axes[v].res;
  std::vector<std::vector<int>> rv;
  for (int i = 0; i < n.nrel; ++i) rv.push_back(distinct_vars(n.rels[i]));
  return plan_joins_policy(n.nvars, vresd, rv, n.exposed, order, pairs, policy);
}

// Key of a relation's density estimate: its arity, degree, kind, eps,
// coefficients and the boxes and resolutions of its variables (SplitMix64
// finaliser over the bytes, 8 at a time).
uint64_t relation_key(const pa_relation& r, const pa_axis* axes) {
  uint64_t h = 0x160900061ull;
  auto add = [&](uint64_t v) { h = mix64(h ^ v); };
  auto addd = [&](double x) {
    uint64_t v;
    memcpy(&v, &x, 8);
    add(v);
  };
  add((uint64_t)r.arity << 32 | (uint32_t)r.degree);
  add((uint64_t)r.kind | (uint64_t)(uint32_t)r.rule << 8);
  addd(r.eps);
  for (int p = 0; p < r.arity; ++p) {
    const pa_axis& a = axes[r.vars[p]];
    addd(a.lo);
    addd(a.hi);
    add((uint64_t)a.res << 8 | (uint64_t)p);
  }
  if (r.expr) {
    add(0xE1u);
    for (int k = 0; k < r.expr->nops; ++k) add((uint64_t)(uint32_t)r.expr->ops[k]);
    for (int k = 0; k < r.expr->nconsts; ++k) addd(r.expr->consts[k]);
    return h;
  }
  const int64_t nc = coeff_count(r.arity, r.degree);
  for (int64_t i = 0; i < nc; ++i) addd(r.coeffs[i]);
  return h;
}

// Estimated plot densities of a network's relations; with a context, kept in
// its cache so that solving the same relations again skips the sampling.
std::vector<double> plot_densities(const Network& n, pa_ctx* ctx) {
  std::vector<double> d;
  for (int i = 0; i < n.nrel; ++i) {
    const pa_relation& r = n.rels[i];
    uint64_t key = 0;
    if (ctx) {
      key = relation_key(r, n.axes);
      auto it = ctx->dens_cache.find(key);
      if (it != ctx->dens_cache.end()) {
        d.push_back(it->second);
        continue;
      }
    }
    const double v = estimate_density(r, n.axes, relation_eps(r, n.axes));
    if (ctx) {
      if (ctx->dens_cache.size() >= (1u << 16)) ctx->dens_cache.clear();
      ctx->dens_cache[key] = v;
    }
    d.push_back(v);
  }
  return d;
}

struct LearnedChoice {
  std::vector<int32_t> pairs;
  bool learned = false;
  float pred_chosen = 0, pred_greedy = 0;
};

std::vector<LearnedChoice> plan_learned(pa_ctx* ctx, Mlp* mlp, const std::vector<Network>& nets,
                                        int ncand) {
  if (ncand <= 0) ncand = 16;
  struct Cand {
    size_t net;
    Plan plan;
    size_t row0, rows;
    double peak;
    std::vector<uint64_t> keys;  // subtree key of every join
  };
  std::vector<Cand> cands;
  std::vector<float> X;
  std::vector<size_t> first(nets.size());
  // the candidate orders of every network, planned in parallel (pure
  // functions of the shapes)
  std::vector<std::vector<Plan>> cplans(nets.size());
  parallel_for(nets.size(), 1, [&](size_t k) {
    const Network& n = nets[k];
    for (int c = 0; c < ncand; ++c)
      cplans[k].push_back((c == 0)   ? plan_of(n, PA_ORDER_GREEDY, nullptr, 0)
                          : (c == 1) ? plan_of(n, PA_ORDER_OPTIMAL, nullptr, 0)
                          : (c == 2) ? plan_of(n, PA_ORDER_GREEDY, nullptr, 1)
                          : (c == 3) ? plan_of(n, PA_ORDER_LEFT, nullptr, 0)
                                     : plan_of(n, PA_ORDER_GREEDY, nullptr, 2 + (uint64_t)c * 7919 + k));
  });
  for (size_t k = 0; k < nets.size(); ++k) {
    const Network& n = nets[k];
    first[k] = cands.size();
    const std::vector<double> dens = plot_densities(n, ctx);
    std::vector<std::vector<int32_t>> seen;
    for (int c = 0; c < ncand; ++c) {
      const Plan& p = cplans[k][c];
      std::vector<int32_t> key;
      for (const Join& j : p.joins) {
        key.push_back(j.a);
        key.push_back(j.b);
      }
      if (c > 0 && std::find(seen.begin(), seen.end(), key) != seen.end()) continue;
      seen.push_back(key);
      SimResult sim = simulate_plan(n, p, dens);
      Cand cd{k, p, X.size() / kFeat, sim.feats.size() / kFeat, sim.peak_bits, plan_keys(n, p)};
      X.insert(X.end(), sim.feats.begin(), sim.feats.end());
      cands.push_back(cd);
    }
  }
  const int nrows = (int)(X.size() / kFeat);
  std::vector<float> Y(nrows, 0.0f);
  if (nrows > 0) {
    float *dX = nullptr, *dY = nullptr;
    check_cuda(ctx, cudaMalloc(&dX, X.size() * 4), "cudaMalloc");
    cudaError_t e = cudaMalloc(&dY, (size_t)nrows * 4);
    if (e == cudaSuccess) e = cudaMemcpy(dX, X.data(), X.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mlp->forward(dX, nrows, dY, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(Y.data(), dY, (size_t)nrows * 4, cudaMemcpyDeviceToHost);
    cudaFree(dX);
    if (dY) cudaFree(dY);
    check_cuda(ctx, e, "cost model forward");
  }
  std::vector<LearnedChoice> out(nets.size());
  for (size_t k = 0; k < nets.size(); ++k) {
    const size_t c0 = first[k], c1 = (k + 1 < nets.size()) ? first[k + 1] : cands.size();
    // a join the solver has timed (pa_join_log) counts with its measured
    // microseconds, any other with the model's prediction
    auto total = [&](const Cand& cd) {
      double t = 0;
      for (size_t r = cd.row0; r < cd.row0 + cd.rows; ++r) {
        auto it = ctx->obs_time.find(cd.keys[r - cd.row0]);
        t += (it != ctx->obs_time.end()) ? it->second : exp2(8.0 * (double)Y[r]);
      }
      return t;
    };
    const double tg = total(cands[c0]);
    size_t best = c0;
    double tb = tg;
    for (size_t c = c0 + 1; c < c1; ++c) {
      const double t = total(cands[c]);
      if (t < tb) {
        tb = t;
        best = c;
      }
    }
    // the greedy order judges: keep the learned one only when it is predicted
    // faster and its largest intermediate stays within 4x the greedy one
    const bool take = best != c0 && tb < tg && cands[best].peak <= 4.0 * cands[c0].peak;
    const Cand& ch = take ? cands[best] : cands[c0];
    for (const Join& j : ch.plan.joins) {
      out[k].pairs.push_back(j.a);
      out[k].pairs.push_back(j.b);
    }
    out[k].learned = take;
    out[k].pred_chosen = (float)(take ? tb : tg);
    out[k].pred_greedy = (float)tg;
  }
  return out;
}

}  // namespace
}  // namespace pa

using namespace pa;

// ---------------------------------------------------------------- batches
struct pa_batch {
  pa_ctx* ctx = nullptr;
  char* mem = nullptr;      // the batch's own workspace; its blob sits at offset 0
  size_t mem_size = 0;
  char* h_blob = nullptr;   // pinned host image of the blob, copied in by every replay
  size_t blob_size = 0;
  std::vector<Op> ops;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  pa_stats st{};
};

struct pa_mlp {
  pa_ctx* ctx = nullptr;
  Mlp* net = nullptr;
};

// Replace PA_ORDER_LEARNED by the orders the cost model picks (given pairs).
static pa_status resolve_learned(pa_ctx* ctx, const pa_options* opts, std::vector<Network>& nets) {
  if (!opts || opts->order != PA_ORDER_LEARNED) return PA_OK;
  try {
    check_cuda(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    std::vector<LearnedChoice> ch = plan_learned(ctx, opts->model->net, nets, opts->ncand);
    for (size_t k = 0; k < nets.size(); ++k) {
      nets[k].own_pairs = ch[k].pairs;
      nets[k].order = PA_ORDER_GIVEN;
      nets[k].pairs = nets[k].own_pairs.data();
    }
    return PA_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

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
  bool ev_ok = true;
  for (int i = 0; i < pa_ctx::kNStage; ++i)
    ev_ok = ev_ok && cudaEventCreateWithFlags(&ctx->stage_done[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ev_ok ||
      cudaMalloc(reinterpret_cast<void**>(&ctx->d_err), sizeof(int)) != cudaSuccess ||
      cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&ctx->d_stat), sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(ctx->d_stat, 0, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    for (int i = 0; i < pa_ctx::kNStage; ++i)
      if (ctx->stage_done[i]) cudaEventDestroy(ctx->stage_done[i]);
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
  for (int i = 0; i < pa_ctx::kNStage; ++i)
    if (ctx->stage_pending[i]) cudaEventSynchronize(ctx->stage_done[i]);
  delete ctx->memo;  // its graph before the arena it points into
  ctx->memo = nullptr;
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->d_stat) cudaFree(ctx->d_stat);
  for (int i = 0; i < pa_ctx::kNStage; ++i) {
    if (ctx->h_stage[i]) cudaFreeHost(ctx->h_stage[i]);
    if (ctx->stage_done[i]) cudaEventDestroy(ctx->stage_done[i]);
  }
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
}

const char* pa_last_error(const pa_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

pa_status pa_set_contract_path(pa_ctx* ctx, int32_t path) {
  if (!ctx) return PA_ERR_INVALID_ARG;
  if (path != PA_PATH_AUTO && path != PA_PATH_ROWOR && path != PA_PATH_MMA)
    return set_err(ctx, PA_ERR_INVALID_ARG, "contract path must be PA_PATH_AUTO, _ROWOR or _MMA");
  ctx->path = path;
  ctx->plan_epoch++;
  return PA_OK;
}

pa_status pa_get_rates(const pa_ctx* ctx, pa_rates* out) {
  if (!ctx || !out) return PA_ERR_INVALID_ARG;
  out->rowor_words_per_us = ctx->rate_or;
  out->rowor_words_per_us_dense = ctx->rate_or_dense;
  out->mma_macs_per_us = ctx->rate_mma;
  return PA_OK;
}

pa_status pa_set_rates(pa_ctx* ctx, const pa_rates* r) {
  if (!ctx || !r) return PA_ERR_INVALID_ARG;
  for (double v : {r->rowor_words_per_us, r->rowor_words_per_us_dense, r->mma_macs_per_us})
    if (!(v > 0) || !isfinite(v))
      return set_err(ctx, PA_ERR_INVALID_ARG, "rates must be finite and positive");
  ctx->rate_or = r->rowor_words_per_us;
  ctx->rate_or_dense = r->rowor_words_per_us_dense;
  ctx->rate_mma = r->mma_macs_per_us;
  ctx->plan_epoch++;
  return PA_OK;
}

pa_status pa_autotune(pa_ctx* ctx, pa_rates* out, void* stream) {
  if (!ctx) return PA_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, PA_ERR_CUDA, "cudaSetDevice failed");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  constexpr int64_t R = 2048, W = R / 64;
  uint64_t *A = nullptr, *B = nullptr, *C = nullptr;
  uint8_t *Ab = nullptr, *Bb = nullptr;
  char* tab = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  pa_status st = PA_OK;
  auto fail = [&](const char* what) {
    cudaGetLastError();
    st = set_err(ctx, PA_ERR_CUDA, std::string("autotune: ") + what);
  };
  // time `reps` runs of f after one warm-up
  auto time_us = [&](auto&& f, int reps) -> double {
    f();
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) f();
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms * 1000.0 / reps;
  };
  do {
    if (cudaMalloc(&A, R * W * 8) != cudaSuccess || cudaMalloc(&B, R * W * 8) != cudaSuccess ||
        cudaMalloc(&C, R * W * 8) != cudaSuccess || cudaMalloc(&tab, 4096) != cudaSuccess ||
        cudaMalloc(&Ab, R * R) != cudaSuccess || cudaMalloc(&Bb, R * R) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      fail("device allocation failed");
      break;
    }
    launch_random_bits(B, R * W, W, R, 0.02, 0x260900061ull, s);
    // row-OR: words OR-ed counted by the kernel
    RowOrDesc rd;
    memset(&rd, 0, sizeof rd);
    rd.A = A;
    rd.B = B;
    rd.C = C;
    rd.nbatch = 1;
    rd.M = R;
    rd.K = R;
    rd.Nw = W;
    rd.a_row_words = W;
    rd.err = ctx->d_err;
    rd.stat = ctx->d_stat;
    rowor_plan(rd, 152);
    CUtensorMap rmap;
    if (rowor_encode_map(rd, &rmap) != cudaSuccess) {
      fail("tensor map (row-OR)");
      break;
    }
    const int64_t rcta[2] = {0, rowor_ctas(rd)};
    MmaDesc md;
    memset(&md, 0, sizeof md);
    md.A = A;
    md.B = B;
    md.C = C;
    md.M = R;
    md.N = R;
    md.K = R;
    md.a_row_words = W;
    md.nbatch = 1;
    md.err = ctx->d_err;
    mma_plan(md);
    md.Ab = Ab;
    md.Bb = Bb;
    CUtensorMap mmaps[2];
    if (mma_encode_maps(md, mmaps) != cudaSuccess) {
      fail("tensor maps (tensor-core path)");
      break;
    }
    const int64_t mcta[2] = {0, mma_ctas(md)};
    // pageable sources: each copy returns once the driver has taken the bytes
    cudaMemcpyAsync(tab, &rd, sizeof rd, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(tab + 1024, &rmap, sizeof rmap, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(tab + 2048, rcta, sizeof rcta, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(tab + 3072, &md, sizeof md, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(tab + 2048 + 64, mcta, sizeof mcta, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(tab + 1024 + 128, mmaps, sizeof mmaps, cudaMemcpyHostToDevice, s);
    const size_t rsmem = rowor_smem_bytes(rd);
    const int reps = 5;
    // row-OR at two densities of A (words OR-ed counted by the kernel)
    double rate_or[2] = {0, 0};
    const double dens[2] = {0.02, 0.16};
    for (int i = 0; i < 2; ++i) {
      launch_random_bits(A, R * W, W, R, dens[i], 0x160900061ull + i, s);
      unsigned long long zero = 0, words = 0;
      cudaMemcpyAsync(ctx->d_stat, &zero, sizeof zero, cudaMemcpyHostToDevice, s);
      const double t_or = time_us(
          [&] {
            launch_rowor(reinterpret_cast<const RowOrDesc*>(tab),
                         reinterpret_cast<const CUtensorMap*>(tab + 1024),
                         reinterpret_cast<const int64_t*>(tab + 2048), 1, rcta[1], rsmem, rd.Nt, s);
          },
          reps);
      cudaMemcpy(&words, ctx->d_stat, sizeof words, cudaMemcpyDeviceToHost);
      cudaMemset(ctx->d_stat, 0, sizeof words);
      if (t_or > 0 && words > 0) rate_or[i] = (double)words / (reps + 1) / t_or;
    }
    // the tensor path's rate includes expanding both operands
    const double t_mma = time_us(
        [&] {
          launch_unpack(reinterpret_cast<const MmaDesc*>(tab + 3072), 1, unpack_blocks_a(md),
                        unpack_blocks_b(md), s);
          launch_mma(reinterpret_cast<const MmaDesc*>(tab + 3072),
                     reinterpret_cast<const CUtensorMap*>(tab + 1024 + 128),
                     reinterpret_cast<const int64_t*>(tab + 2048 + 64), 1, mcta[1], s);
        },
        reps);
    if (cudaGetLastError() != cudaSuccess || rate_or[0] <= 0 || rate_or[1] <= 0 || t_mma <= 0) {
      fail("timing runs failed");
      break;
    }
    int herr = 0;
    cudaMemcpy(&herr, ctx->d_err, sizeof herr, cudaMemcpyDeviceToHost);
    if (herr) {
      st = set_err(ctx, PA_ERR_TIMEOUT, "autotune: a bounded device wait ran out");
      cudaMemset(ctx->d_err, 0, sizeof herr);
      break;
    }
    ctx->rate_or = rate_or[0];
    ctx->rate_or_dense = rate_or[1];
    ctx->rate_mma = (double)R * R * R / t_mma;
    ctx->plan_epoch++;
  } while (false);
  if (st == PA_OK && out) pa_get_rates(ctx, out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (void* p : {(void*)A, (void*)B, (void*)C, (void*)Ab, (void*)Bb, (void*)tab})
    if (p) cudaFree(p);
  return st;
}

pa_status pa_wait_selftest(pa_ctx* ctx, int64_t limit_ns, void* stream) {
  if (!ctx || limit_ns < 1000 || limit_ns > 2000000000ll) return PA_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, PA_ERR_CUDA, "cudaSetDevice failed");
  }
  cudaError_t e = launch_wait_selftest(ctx->d_err, (long long)limit_ns, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return set_err(ctx, PA_ERR_CUDA, cudaGetErrorString(e));
  return PA_OK;
}

pa_status pa_measure_peaks(pa_ctx* ctx, pa_peaks* out, void* stream) {
  if (!ctx || !out) return PA_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, PA_ERR_CUDA, "cudaSetDevice failed");
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (sms <= 0) return set_err(ctx, PA_ERR_CUDA, "multiprocessor count");
  memset(out, 0, sizeof *out);
  out->sms = sms;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double clk = 0, clk2 = 0;
  cudaError_t e = run_probe(0, sms, s, &out->lop3_ops_per_s, &out->lop3_per_clk_sm, &clk);
  if (e == cudaSuccess)
    e = run_probe(1, sms, s, &out->smem_bytes_per_s, &out->smem_bytes_per_clk_sm, &clk2);
  if (e == cudaSuccess)
    e = run_probe(2, sms, s, &out->fp32_flops_per_s, &out->fp32_flops_per_clk_sm, &clk2);
  if (e == cudaSuccess)
    e = run_probe(3, sms, s, &out->fp64_flops_per_s, &out->fp64_flops_per_clk_sm, &clk2);
  out->sm_clock_hz = clk;
  if (e != cudaSuccess) return set_err(ctx, PA_ERR_CUDA, std::string("probe: ") + cudaGetErrorString(e));
  return PA_OK;
}

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
    if (rel->expr) return PA_ERR_UNSUPPORTED;
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
  PlotReq req{rel, axes, strict ? 1 : 0, out->words};
  return run_call(ctx, static_cast<cudaStream_t>(stream), nullptr,
                  [&](Builder& bd) { plot_all(bd, {req}); });
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
  return run_call(ctx, static_cast<cudaStream_t>(stream), nullptr, [&](Builder& bd) {
    BitArr r = join(bd, a, b, kv, vres, &target, 152);
    flush_rowor(bd);
    if (r.w != target.w) reshape(bd, r, target);
  });
}

pa_status pa_contract_count(pa_ctx* ctx, const pa_array* A, const pa_array* B, int32_t nkeep,
                            const int32_t* keep, uint32_t* counts, void* stream) {
  if (!ctx) return PA_ERR_INVALID_ARG;
  std::vector<int> kv;
  std::vector<int64_t> vres;
  try {
    check_array(ctx, A, "A");
    check_array(ctx, B, "B");
    PA_CHECK_ARG(counts != nullptr, "counts: null pointer");
    PA_CHECK_ARG(nkeep >= 1 && nkeep <= PA_MAX_DIM && keep, "keep: 1..8 variables");
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
      for (int j = 0; j < i; ++j) PA_CHECK_ARG(keep[j] != v, "keep: repeated variable");
      kv.push_back(v);
    }
  } catch (const Fail& f) {
    return f.st;
  }
  BitArr a = from_pa(*A), b = from_pa(*B);
  return run_call(ctx, static_cast<cudaStream_t>(stream), nullptr,
                  [&](Builder& bd) { join_count(bd, a, b, kv, vres, counts); });
}

pa_status pa_solve_network(pa_ctx* ctx, int32_t nvars, const pa_axis* axes, int32_t nrel,
                           const pa_relation* rels, int32_t nexposed, const int32_t* exposed,
                           const pa_options* opts, pa_array* out, pa_stats* stats,
                           void* stream) {
  if (!ctx) return PA_ERR_INVALID_ARG;
  std::vector<Network> nets(1);
  try {
    check_network(ctx, nvars, axes, nrel, rels, nexposed, exposed, opts, out, nets[0]);
  } catch (const Fail& f) {
    return f.st;
  }
  // a learned order depends on a model that may change between calls: never kept
  const bool keep = !(opts && opts->order == PA_ORDER_LEARNED);
  std::vector<char> key;
  if (keep) {
    key = solve_key(ctx, nvars, axes, nrel, rels, nexposed, exposed, opts, out, stream);
    if (ctx->memo && ctx->memo->key == key)
      return run_memo(ctx, static_cast<cudaStream_t>(stream), stats);
  }
  pa_status st = resolve_learned(ctx, opts, nets);
  if (st != PA_OK) return st;
  return run_call(ctx, static_cast<cudaStream_t>(stream), stats,
                  [&](Builder& bd) { build_networks(bd, nets); }, keep ? &key : nullptr);
}

static pa_status check_batch(pa_ctx* ctx, int32_t nsys, const pa_system* systems, pa_array* outs,
                             const pa_options* opts, std::vector<Network>& nets) {
  try {
    PA_CHECK_ARG(nsys >= 1 && systems && outs, "batch: null pointer or no systems");
    PA_CHECK_ARG(!opts || opts->order != PA_ORDER_GIVEN, "batch: given orders are per system");
    nets.resize(nsys);
    for (int k = 0; k < nsys; ++k) {
      const pa_system& s = systems[k];
      check_network(ctx, s.nvars, s.axes, s.nrel, s.rels, s.nexposed, s.exposed, opts, &outs[k],
                    nets[k]);
    }
  } catch (const Fail& f) {
    return f.st;
  }
  return resolve_learned(ctx, opts, nets);
}

pa_status pa_solve_batch(pa_ctx* ctx, int32_t nsys, const pa_system* systems, pa_array* outs,
                         const pa_options* opts, pa_stats* stats, void* stream) {
  if (!ctx) return PA_ERR_INVALID_ARG;
  std::vector<Network> nets;
  pa_status st = check_batch(ctx, nsys, systems, outs, opts, nets);
  if (st != PA_OK) return st;
  return run_call(ctx, static_cast<cudaStream_t>(stream), stats,
                  [&](Builder& bd) { build_networks(bd, nets); });
}

void pa_batch_destroy(pa_batch* bt);

pa_status pa_batch_create(pa_ctx* ctx, int32_t nsys, const pa_system* systems, pa_array* outs,
                          const pa_options* opts, pa_batch** out) {
  if (!ctx || !out) return PA_ERR_INVALID_ARG;
  *out = nullptr;
  std::vector<Network> nets;
  pa_status st = check_batch(ctx, nsys, systems, outs, opts, nets);
  if (st != PA_OK) return st;
  pa_batch* bt = new pa_batch();
  bt->ctx = ctx;
  cudaStream_t cs = nullptr;
  try {
    check_cuda(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    Builder dry(ctx, true, nullptr, 0);
    build_networks(dry, nets);
    const size_t blob_cap = round_up(dry.blob.size() + 64, kAlign);
    bt->mem_size = dry.used + blob_cap + kAlign;
    if (ctx->cap && bt->mem_size > ctx->cap)
      throw Fail{set_err(ctx, PA_ERR_OOM, "batch workspace exceeds the context's cap")};
    if (cudaMalloc(reinterpret_cast<void**>(&bt->mem), bt->mem_size) != cudaSuccess) {
      cudaGetLastError();
      bt->mem = nullptr;
      throw Fail{set_err(ctx, PA_ERR_OOM, "cudaMalloc of the batch workspace failed")};
    }
    Builder bd(ctx, false, bt->mem, blob_cap);
    bd.d_err = ctx->d_err;
    build_networks(bd, nets);
    bt->ops = bd.ops;
    bt->st = bd.st;
    bt->st.workspace_bytes = (int64_t)bd.used;
    bt->st.n_launches = (int32_t)bd.ops.size();
    bt->blob_size = bd.blob.size();
    check_cuda(ctx, cudaMallocHost(reinterpret_cast<void**>(&bt->h_blob),
                                   std::max<size_t>(1, bt->blob_size)),
               "cudaMallocHost");
    memcpy(bt->h_blob, bd.blob.data(), bt->blob_size);
    // capture the blob copy and every launch as one graph
    check_cuda(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
    check_cuda(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal),
               "cudaStreamBeginCapture");
    cudaError_t ce = cudaMemcpyAsync(bt->mem, bt->h_blob, bt->blob_size, cudaMemcpyHostToDevice, cs);
    bool ran = false;
    if (ce == cudaSuccess) {
      try {
        run_ops(ctx, bt->ops, bt->mem, cs, false);
        ran = true;
      } catch (const Fail&) {
        ran = false;
      }
    }
    cudaError_t ee = cudaStreamEndCapture(cs, &bt->graph);
    check_cuda(ctx, ce, "cudaMemcpyAsync (capture)");
    if (!ran) throw Fail{PA_ERR_CUDA};
    check_cuda(ctx, ee, "cudaStreamEndCapture");
    check_cuda(ctx, cudaGraphInstantiate(&bt->exec, bt->graph, 0), "cudaGraphInstantiate");
    cudaStreamDestroy(cs);
    cs = nullptr;
    *out = bt;
    return PA_OK;
  } catch (const Fail& f) {
    if (cs) cudaStreamDestroy(cs);
    pa_batch_destroy(bt);
    return f.st;
  }
}

pa_status pa_batch_run(pa_batch* bt, void* stream) {
  if (!bt || !bt->exec) return PA_ERR_INVALID_ARG;
  pa_ctx* ctx = bt->ctx;
  cudaSetDevice(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  pa_ctx::Rec rec;
  try {
    if (ctx->prof) {
      rec.name = "batch_graph";
      rec.a = next_event(ctx);
      rec.b = next_event(ctx);
      check_cuda(ctx, cudaEventRecord(rec.a, s), "cudaEventRecord");
    }
    check_cuda(ctx, cudaGraphLaunch(bt->exec, s), "cudaGraphLaunch");
    if (ctx->prof) {
      check_cuda(ctx, cudaEventRecord(rec.b, s), "cudaEventRecord");
      ctx->recs.push_back(rec);
    }
  } catch (const Fail& f) {
    return f.st;
  }
  return PA_OK;
}

pa_status pa_batch_stats(const pa_batch* bt, pa_stats* stats) {
  if (!bt || !stats) return PA_ERR_INVALID_ARG;
  *stats = bt->st;
  return PA_OK;
}

void pa_batch_destroy(pa_batch* bt) {
  if (!bt) return;
  if (bt->ctx) cudaSetDevice(bt->ctx->device);
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  if (bt->mem) {
    cudaDeviceSynchronize();  // replays in flight may still use the workspace
    cudaFree(bt->mem);
  }
  if (bt->h_blob) cudaFreeHost(bt->h_blob);
  delete bt;
}

pa_status pa_mlp_create(pa_ctx* ctx, int32_t hidden, int32_t nlayers, uint64_t seed,
                        pa_mlp** model) {
  if (!ctx || !model || hidden < 1 || hidden > 1024 || nlayers < 0 || nlayers > 8)
    return PA_ERR_INVALID_ARG;
  *model = nullptr;
  cudaSetDevice(ctx->device);
  pa_mlp* m = new pa_mlp();
  m->ctx = ctx;
  m->net = new Mlp(PA_FEATURES, hidden, nlayers);
  if (m->net->alloc_params() != cudaSuccess) {
    cudaGetLastError();
    pa_mlp_destroy(m);
    return set_err(ctx, PA_ERR_OOM, "cost model: cudaMalloc failed");
  }
  // He-uniform weights from a SplitMix64 stream, zero biases
  std::vector<float> p(m->net->np, 0.0f);
  uint64_t st = seed;
  for (size_t l = 0; l + 1 < m->net->sizes.size(); ++l) {
    const int ni = m->net->sizes[l], no = m->net->sizes[l + 1];
    const double lim = sqrt(6.0 / ni);
    for (int64_t k = 0; k < (int64_t)no * ni; ++k) {
      const uint64_t z = mix64(st++);
      const double u = (double)(z >> 11) * 0x1p-53;
      p[m->net->woff[l] + k] = (float)((2.0 * u - 1.0) * lim);
    }
  }
  if (cudaMemcpy(m->net->p, p.data(), p.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    pa_mlp_destroy(m);
    return set_err(ctx, PA_ERR_CUDA, "cost model: parameter upload failed");
  }
  *model = m;
  return PA_OK;
}

void pa_mlp_destroy(pa_mlp* model) {
  if (!model) return;
  if (model->ctx) cudaSetDevice(model->ctx->device);
  delete model->net;
  delete model;
}

int64_t pa_mlp_num_params(const pa_mlp* model) { return model ? model->net->np : -1; }

static pa_status mlp_copy(const pa_mlp* model, void* dst, const void* src, size_t bytes,
                          cudaMemcpyKind kind) {
  if (!model || !dst || !src) return PA_ERR_INVALID_ARG;
  cudaSetDevice(model->ctx->device);
  if (cudaMemcpy(dst, src, bytes, kind) != cudaSuccess) {
    cudaGetLastError();
    return set_err(model->ctx, PA_ERR_CUDA, "cost model: copy failed");
  }
  return PA_OK;
}

pa_status pa_mlp_get_params(const pa_mlp* model, float* params) {
  if (!model) return PA_ERR_INVALID_ARG;
  return mlp_copy(model, params, model->net->p, model->net->np * 4, cudaMemcpyDeviceToHost);
}

pa_status pa_mlp_set_params(pa_mlp* model, const float* params) {
  if (!model) return PA_ERR_INVALID_ARG;
  return mlp_copy(model, model->net->p, params, model->net->np * 4, cudaMemcpyHostToDevice);
}

pa_status pa_mlp_get_grads(const pa_mlp* model, float* grads) {
  if (!model) return PA_ERR_INVALID_ARG;
  return mlp_copy(model, grads, model->net->g, model->net->np * 4, cudaMemcpyDeviceToHost);
}

pa_status pa_mlp_forward(pa_mlp* model, const float* x, int32_t n, float* y, void* stream) {
  if (!model || !x || !y || n < 0) return PA_ERR_INVALID_ARG;
  if (n == 0) return PA_OK;
  cudaSetDevice(model->ctx->device);
  if (model->net->forward(x, n, y, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    cudaGetLastError();
    return set_err(model->ctx, PA_ERR_CUDA, "cost model: forward failed");
  }
  return PA_OK;
}

pa_status pa_mlp_backward(pa_mlp* model, const float* x, const float* t, int32_t n, float* loss,
                          void* stream) {
  if (!model || !x || !t || n <= 0) return PA_ERR_INVALID_ARG;
  cudaSetDevice(model->ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (model->net->backward(x, t, n, s) != cudaSuccess) {
    cudaGetLastError();
    return set_err(model->ctx, PA_ERR_CUDA, "cost model: backward failed");
  }
  if (loss) {
    if (cudaMemcpyAsync(loss, model->net->loss, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return set_err(model->ctx, PA_ERR_CUDA, "cost model: loss read failed");
    }
  }
  return PA_OK;
}

pa_status pa_mlp_adam(pa_mlp* model, float lr, float beta1, float beta2, float eps, void* stream) {
  if (!model || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return PA_ERR_INVALID_ARG;
  cudaSetDevice(model->ctx->device);
  if (model->net->adam(lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    cudaGetLastError();
    return set_err(model->ctx, PA_ERR_CUDA, "cost model: adam failed");
  }
  return PA_OK;
}

pa_status pa_join_log(pa_ctx* ctx, const pa_system* sys, const pa_options* opts, pa_array* out,
                      int32_t max_joins, float* features, float* micros, float* densities,
                      int32_t* njoins, void* stream) {
  if (!ctx || !sys || !njoins || max_joins < 0 ||
      (max_joins > 0 && (!features || !micros || !densities)))
    return PA_ERR_INVALID_ARG;
  std::vector<Network> nets(1);
  try {
    check_network(ctx, sys->nvars, sys->axes, sys->nrel, sys->rels, sys->nexposed, sys->exposed,
                  opts, out, nets[0]);
  } catch (const Fail& f) {
    return f.st;
  }
  pa_status st = resolve_learned(ctx, opts, nets);
  if (st != PA_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long* dcnt = nullptr;
  std::vector<cudaEvent_t> evs;
  try {
    check_cuda(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
    Builder dry(ctx, true, nullptr, 0);
    build_networks(dry, nets, true);
    const size_t blob_cap = round_up(dry.blob.size() + 64, kAlign);
    st = ensure_arena(ctx, dry.used + blob_cap + kAlign);
    if (st != PA_OK) return st;
    Builder bd(ctx, false, ctx->arena, blob_cap);
    bd.d_err = ctx->d_err;
    std::vector<BitArr> results;
    build_networks(bd, nets, true, &results);
    upload_blob(ctx, bd.blob, s);
    // one event pair per op
    const size_t nops = bd.ops.size();
    evs.resize(2 * nops, nullptr);
    for (auto& e : evs) check_cuda(ctx, cudaEventCreate(&e), "cudaEventCreate");
    for (size_t q = 0; q < nops; ++q) {
      std::vector<Op> one(1, bd.ops[q]);
      check_cuda(ctx, cudaEventRecord(evs[2 * q], s), "cudaEventRecord");
      run_ops(ctx, one, ctx->arena, s, false);
      check_cuda(ctx, cudaEventRecord(evs[2 * q + 1], s), "cudaEventRecord");
    }
    const int nj = (int)results.size();
    check_cuda(ctx, cudaMalloc(&dcnt, std::max(1, nj) * sizeof(unsigned long long)), "cudaMalloc");
    check_cuda(ctx, cudaMemsetAsync(dcnt, 0, std::max(1, nj) * sizeof(unsigned long long), s),
               "cudaMemsetAsync");
    for (int t = 0; t < nj; ++t) launch_popcount(results[t].w, results[t].words(), dcnt + t, s);
    check_cuda(ctx, cudaGetLastError(), "popcount_kernel");
    std::vector<unsigned long long> cnt(std::max(1, nj));
    check_cuda(ctx, cudaMemcpyAsync(cnt.data(), dcnt, cnt.size() * 8, cudaMemcpyDeviceToHost, s),
               "cudaMemcpyAsync");
    check_cuda(ctx, cudaStreamSynchronize(s), "cudaStreamSynchronize");
    std::vector<double> us(nj, 0.0);
    for (size_t q = 0; q < nops; ++q) {
      float ms = 0;
      check_cuda(ctx, cudaEventElapsedTime(&ms, evs[2 * q], evs[2 * q + 1]), "cudaEventElapsedTime");
      if (bd.ops[q].join >= 0 && bd.ops[q].join < nj) us[bd.ops[q].join] += 1000.0 * ms;
    }
    const Plan plan = plan_of(nets[0], nets[0].order, nets[0].pairs, 0);
    const SimResult sim = simulate_plan(nets[0], plan, plot_densities(nets[0], ctx));
    *njoins = nj;
    for (int t = 0; t < nj && t < max_joins; ++t) {
      for (int k = 0; k < kFeat; ++k) features[t * kFeat + k] = sim.feats[t * kFeat + k];
      micros[t] = (float)us[t];
      densities[t] = (float)((double)cnt[t] / (double)std::max<int64_t>(1, results[t].bits()));
    }
    // remember the measured densities for later path choices on these
    // relations, and the measured join times for the learned order's judge
    // (a subtree key names the whole join tree below a result, so a time is
    // only reused for the very same join)
    const Network& n0 = nets[0];
    if ((int)n0.slot_keys.size() == n0.nrel + nj) {
      ctx->plan_epoch++;
      if (ctx->obs_dens.size() >= (1u << 16)) ctx->obs_dens.clear();
      if (ctx->obs_time.size() >= (1u << 16)) ctx->obs_time.clear();
      for (int t = 0; t < nj; ++t) {
        ctx->obs_dens[n0.slot_keys[n0.nrel + t]] =
            (double)cnt[t] / (double)std::max<int64_t>(1, results[t].bits());
        ctx->obs_time[n0.slot_keys[n0.nrel + t]] = us[t];
      }
    }
  } catch (const Fail& f) {
    st = f.st;
  }
  if (dcnt) cudaFree(dcnt);
  for (auto e : evs)
    if (e) cudaEventDestroy(e);
  return st;
}

pa_status pa_plan_learned(pa_ctx* ctx, const pa_mlp* model, int32_t nsys, const pa_system* systems,
                          int32_t ncand, int32_t* pairs_out, int32_t* learned, float* pred_us) {
  if (!ctx || !model || nsys < 1 || !systems || !pairs_out || !learned || !pred_us)
    return PA_ERR_INVALID_ARG;
  std::vector<Network> nets(nsys);
  try {
    for (int k = 0; k < nsys; ++k) {
      const pa_system& sy = systems[k];
      check_axes(ctx, sy.nvars, sy.axes);
      PA_CHECK_ARG(sy.nrel >= 1 && sy.rels, "at least one relation");
      for (int i = 0; i < sy.nrel; ++i) check_relation(ctx, sy.rels[i], sy.nvars);
      Network& n = nets[k];
      n.nvars = sy.nvars;
      n.axes = sy.axes;
      n.nrel = sy.nrel;
      n.rels = sy.rels;
      n.exposed.assign(sy.exposed, sy.exposed + sy.nexposed);
      for (int v : n.exposed) PA_CHECK_ARG(v >= 0 && v < sy.nvars, "exposed: variable out of range");
      n.order = PA_ORDER_GREEDY;
      n.pairs = nullptr;
      n.strict = 0;
    }
    std::vector<LearnedChoice> ch = plan_learned(ctx, model->net, nets, ncand);
    size_t off = 0;
    for (int k = 0; k < nsys; ++k) {
      for (int32_t v : ch[k].pairs) pairs_out[off++] = v;
      learned[k] = ch[k].learned ? 1 : 0;
      pred_us[2 * k] = ch[k].pred_chosen;
      pred_us[2 * k + 1] = ch[k].pred_greedy;
    }
    return PA_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

pa_status pa_plan_order(int32_t nvars, const pa_axis* axes, int32_t nrel, const pa_relation* rels,
                        int32_t nexposed, const int32_t* exposed, int32_t order,
                        int32_t* pairs_out, double* pixel_ops_out, int64_t* peak_bits_out) {
  pa_ctx* ctx = nullptr;
  try {
    check_axes(ctx, nvars, axes);
    PA_CHECK_ARG(nrel >= 1 && rels && (nexposed == 0 || exposed), "null pointer");
    PA_CHECK_ARG(order == PA_ORDER_GREEDY || order == PA_ORDER_LEFT || order == PA_ORDER_OPTIMAL,
                 "order");
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

// ================================================= solve without allocation
// pa_solve_network_static: the whole-method solve with its workspace in a
// fixed device array instead of memory the library allocates.  The array's
// host-side name is only a stand-in; its device address is looked up once per
// device (cudaGetSymbolAddress, with that device current) and cached.
static __device__ __align__(256) unsigned char g_pa_static_scratch[PA_STATIC_SCRATCH_BYTES];

namespace {
std::mutex g_static_mu;
constexpr int kMaxDevices = 256;
char* g_static_addr[kMaxDevices] = {};
constexpr size_t kStaticHeader = 256;  // device error word lives here
}  // namespace

extern "C" pa_status pa_solve_network_static(int32_t nvars, const pa_axis* axes, int32_t nrel,
                                             const pa_relation* rels, int32_t nexposed,
                                             const int32_t* exposed, const pa_options* opts,
                                             pa_array* out, pa_stats* stats, void* stream) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return PA_ERR_CUDA;
  }
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_pa_static_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return PA_ERR_CUDA;
      }
      g_static_addr[dev] = static_cast<char*>(p);
    }
    base = g_static_addr[dev];
  }
  pa_ctx* ctx = nullptr;  // no context: errors are reported by the return code only
  // the learned order ranks candidates with a context's model: not available here
  if (opts && opts->order == PA_ORDER_LEARNED) return PA_ERR_INVALID_ARG;
  std::vector<Network> nets(1);
  try {
    check_network(ctx, nvars, axes, nrel, rels, nexposed, exposed, opts, out, nets[0]);
  } catch (const Fail& f) {
    return f.st;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  try {
    Builder dry(ctx, true, nullptr, 0);
    build_networks(dry, nets);
    const size_t blob_cap = round_up(dry.blob.size() + 64, kAlign);
    const size_t need = kStaticHeader + dry.used + blob_cap + kAlign;
    if (need > PA_STATIC_SCRATCH_BYTES) {
      if (stats) {
        *stats = dry.st;
        stats->workspace_bytes = (int64_t)need;
      }
      return PA_ERR_TOO_LARGE;
    }
    char* work = base + kStaticHeader;
    Builder bd(ctx, false, work, blob_cap);
    bd.d_err = reinterpret_cast<int*>(base);
    build_networks(bd, nets);
    if (bd.blob.size() > blob_cap) return PA_ERR_CUDA;
    // the array keeps the previous call's contents: the error word starts at zero
    check_cuda(ctx, cudaMemsetAsync(base, 0, kStaticHeader, s), "cudaMemsetAsync");
    // pageable source: the copy returns once the driver has taken the bytes
    check_cuda(ctx, cudaMemcpyAsync(work, bd.blob.data(), bd.blob.size(), cudaMemcpyHostToDevice, s),
               "cudaMemcpyAsync");
    run_ops(ctx, bd.ops, work, s, false);
    bd.st.workspace_bytes = (int64_t)(kStaticHeader + bd.used);
    bd.st.n_launches = (int32_t)bd.ops.size() + 2;
    if (stats) *stats = bd.st;
    return PA_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}
