/*
 * pa.h -- C interface of the GB300 pixel array engine.
 *
 * The pixel array method (Spivak, Dobson, Kumari, Wu, arXiv 1609.00061) solves a
 * system of relations over a box by (1) plotting each relation as a Boolean
 * pixel array (Sec. 3.2, sample-in-center plot) and (2) combining the plots by
 * generalized array multiplication over the Boolean semiring (Sec. 3.3,
 * Algorithm 1 and Eq. GAM), one cluster at a time (Sec. 3.5), until only the
 * exposed variables remain (Sec. 3.6).
 *
 * Every entry point takes plain pointers and sizes.  Device work is enqueued on
 * the CUDA stream passed as `stream` (a cudaStream_t cast to void*; NULL is the
 * legacy default stream) and is asynchronous to the host unless stated.
 *
 * ---------------------------------------------------------------- conventions
 * Variables are numbered 0..nvars-1.  Variable v ranges over [lo, hi) at
 * resolution res >= 2 (Sec. 3.1, Definition of a pack): pixel i (0-based) of v
 * covers [lo + i*delta, lo + (i+1)*delta) with delta = (hi - lo) / res, and its
 * centre is computed as lo + ((double)i + 0.5) * delta (two IEEE roundings).
 *
 * Relations are polynomials f(x_1..x_n) compared with 0 (pa_kind).  The
 * coefficients of all monomials of total degree <= degree are given in graded
 * lexicographic order: total degree 0, 1, ..., degree; within one degree the
 * exponent tuples (e_1, ..., e_n) in descending lexicographic order.  Two
 * variables, degree 3: 1, x, y, x^2, xy, y^2, x^3, x^2y, xy^2, y^3.  f is evaluated
 * in IEEE double precision without fused multiply-add, in the nested form
 *   f = sum_{e_n} ( ... ( sum_{e_1} c_e * x_1^{e_1} ) * x_2^{e_2} ... ) * x_n^{e_n},
 * every sum taken left to right from its e = 0 term, powers by repeated
 * multiplication from 1.0.  This fixes every rounding, so results are
 * reproducible bit for bit on any IEEE machine.
 *
 * A pixel is on when f at its centre is finite and (Sec. 3.2, "the error at the
 * centre achieves eps"):  PA_EQ: |f| <= eps;  PA_LE: f <= eps;  PA_LT: f < eps.
 * With strict = 1 every "<=" becomes "<" (the test used by the paper's
 * Appendix A code).  NaN and +-Inf turn the pixel off (Sec. 2.4).
 *
 * Bit-packed arrays (pa_array): axes in the order of `vars`, last axis fastest.
 * Every last-axis row is packed LSB-first into ceil(res_last / 64) uint64 words
 * (bit b of word w is pixel 64*w + b); unused high bits of the last word are 0.
 * Rows follow each other in row-major order of the other axes.  A 0-dimensional
 * array (no exposed variables: "does a solution exist") is one word, bit 0.
 *
 * Ownership: the caller allocates every pa_array's words on the context's
 * device and keeps them alive until the stream work finishes; the library
 * never frees them.  The context owns only its own scratch workspace.
 *
 * Errors: every call returns a pa_status; nothing is thrown across the ABI.
 * pa_last_error(ctx) gives a message for the last failure on that context.
 * Shapes and arguments are checked before any launch; a launch failure is
 * reported by the call that made it; a fault inside a kernel surfaces at the
 * next synchronisation of the stream.
 *
 * Concurrency: one context serves one stream at a time.  Two calls on the same
 * context must be ordered on the device (same stream, or events) because they
 * share the context's workspace.  Use one context per concurrent stream.
 */
#ifndef PA_H_
#define PA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PA_MAX_DIM 8     /* ports per relation / axes per array */
#define PA_MAX_DEGREE 16 /* total degree of a relation's polynomial */

typedef enum {
  PA_OK = 0,
  PA_ERR_INVALID_ARG = 1, /* a null pointer, a bad size, inconsistent shapes */
  PA_ERR_UNSUPPORTED = 2, /* valid input outside the library's limits */
  PA_ERR_TOO_LARGE = 3,   /* an array or index would overflow 2^62 bits */
  PA_ERR_OOM = 4,         /* the workspace could not be allocated */
  PA_ERR_CUDA = 5,        /* a CUDA call failed; see pa_last_error */
  PA_ERR_TIMEOUT = 6      /* a bounded device wait ran out */
} pa_status;

/* Target set S of a relation f(x) in S (Sec. 3.2, functionally-defined
 * relations): {0}, (-inf, 0] or (-inf, 0). */
typedef enum { PA_EQ = 0, PA_LE = 1, PA_LT = 2 } pa_kind;

/* One variable's range [lo, hi) and resolution (Sec. 3.1, pack). lo < hi,
 * both finite, res >= 2. */
typedef struct {
  double lo;
  double hi;
  int32_t res;
} pa_axis;

/* ------------------------------------------------------ expression relations
 * A relation may also be any expression built from the ports with the
 * operations below (the paper's own examples mix polynomials with |.|, cos,
 * ln, tan, cosh, exp and reciprocals: Sec. 2.1 and Sec. 2.4).  The expression
 * is a postfix program over a stack of doubles: each instruction is one
 * int32, op | (arg << 8) with a signed 24-bit arg.
 *   PA_X_CONST  push consts[arg]        PA_X_VAR   push port arg's coordinate
 *   PA_X_ADD, PA_X_SUB, PA_X_MUL, PA_X_DIV, PA_X_POW: pop b, pop a, push a op b
 *   PA_X_NEG, PA_X_ABS, PA_X_SQRT, PA_X_EXP, PA_X_LOG (natural), PA_X_SIN,
 *   PA_X_COS, PA_X_TAN, PA_X_SINH, PA_X_COSH, PA_X_TANH, PA_X_ATAN: pop a,
 *   push op(a)
 *   PA_X_POWI   pop a, push a^arg for an integer arg: |arg| - 1 products from
 *               a, left to right, then 1 / that for arg < 0 (arg = 0: 1.0)
 * A program must leave exactly one value; it may not pop an empty stack or
 * hold more than PA_EXPR_MAX_STACK values.  Every operation is evaluated in
 * IEEE double precision: +, -, *, / and sqrt correctly rounded, the others by
 * the CUDA math library (results may differ from another library's in the
 * last bits; a pixel whose |f| lies within that difference of eps may then
 * be decided differently).  Non-finite results turn the pixel off as for
 * polynomials.  An expression relation needs its own eps >= 0: the library
 * computes valid tolerances for polynomials only. */
#define PA_EXPR_MAX_OPS 256
#define PA_EXPR_MAX_STACK 16
typedef enum {
  PA_X_CONST = 0, PA_X_VAR = 1, PA_X_ADD = 2, PA_X_SUB = 3, PA_X_MUL = 4, PA_X_DIV = 5,
  PA_X_NEG = 6, PA_X_ABS = 7, PA_X_SQRT = 8, PA_X_EXP = 9, PA_X_LOG = 10, PA_X_SIN = 11,
  PA_X_COS = 12, PA_X_TAN = 13, PA_X_SINH = 14, PA_X_COSH = 15, PA_X_TANH = 16,
  PA_X_ATAN = 17, PA_X_POWI = 18, PA_X_POW = 19
} pa_expr_op;

typedef struct {
  int32_t nops;
  const int32_t* ops;   /* HOST pointer: nops instructions */
  int32_t nconsts;
  const double* consts; /* HOST pointer: nconsts doubles */
} pa_expr;

/* ------------------------------------------------------------ sample rules
 * PA_RULE_CENTER (default) is the paper's sample-in-center plot (above).
 * PA_RULE_CORNER is an optional alternative that samples f on the lattice of
 * grid corners instead: variable v has the res + 1 lattice coordinates
 * lo + (double)i * delta, i = 0..res (one product and one sum, each rounded),
 * and pixel e has the 2^d corners that take index e_v or e_v + 1 on each of
 * the relation's d distinct variables (a variable on two ports reads the same
 * coordinate on both).  The pixel is on when some corner c with finite f(c)
 * passes the same comparison as the centre rule (|f(c)| <= eps for PA_EQ,
 * f(c) <= eps for PA_LE, f(c) < eps for PA_LT, strict as above), or, for
 * PA_EQ, when the finite corner values include one above 0 and one below 0 (a
 * sign change inside the pixel).  Non-finite corner values take part in
 * neither test; a value of exactly 0 has no sign.  The valid tolerance of this
 * rule uses the full pixel width delta_p where the centre rule uses
 * delta_p / 2 (pa_valid_tolerance), since every point of a pixel lies within
 * delta_p of each of its corners along each axis.  Polynomial and expression
 * relations both support it; the corner values are evaluated in the same
 * IEEE double order as the centre values. */
typedef enum { PA_RULE_CENTER = 0, PA_RULE_CORNER = 1 } pa_rule;

/* A relation over `arity` ports; port p reads variable vars[p].  A variable
 * may fill several ports (a loop in the wiring diagram, Sec. 3.1): the
 * relation is then plotted on the diagonal.  With expr == NULL the relation is
 * a polynomial: `coeffs` is a HOST pointer to C(arity + degree, degree)
 * doubles in graded lex order.  With expr != NULL the relation is that
 * expression of the ports (degree and coeffs are ignored).  eps >= 0 is the
 * tolerance; eps < 0 asks the library for a valid one (pa_valid_tolerance;
 * polynomials only).  rule is a pa_rule (0, the paper's centre rule, when the
 * structure is zero-initialised). */
typedef struct {
  int32_t arity;
  int32_t vars[PA_MAX_DIM];
  int32_t degree;
  const double* coeffs;
  int32_t kind;
  double eps;
  const pa_expr* expr;
  int32_t rule;
} pa_relation;

/* A bit-packed Boolean array on the device (layout above).  `words` holds
 * pa_array_words(this) uint64 words.  vars are distinct. */
typedef struct {
  uint64_t* words;
  int32_t ndim;
  int32_t vars[PA_MAX_DIM];
  int32_t res[PA_MAX_DIM];
} pa_array;

/* Contraction order of pa_solve_network.  Any order gives the same bits
 * (Sec. 3.3, Thm. associative); only the time differs. */
typedef enum {
  PA_ORDER_GREEDY = 0, /* repeatedly join the pair with the smallest result */
  PA_ORDER_GIVEN = 1,  /* join the pairs listed in pa_options.pairs */
  PA_ORDER_LEFT = 2,   /* fold the relations left to right */
  PA_ORDER_LEARNED = 3, /* rank candidate orders with a learned cost model
                           (pa_options.model); the greedy order is the fallback */
  PA_ORDER_OPTIMAL = 4  /* the pairwise cluster tree of least naive cost
                           sum r^Lambda (Sec. 3.5, cost polynomial), ties to the
                           smaller parallel cost: exact over every pairwise
                           tree up to 16 relations; beyond, the greedy tree
                           with every subtree of at most 16 relations
                           replaced by its exact optimum */
} pa_order;

typedef struct pa_mlp pa_mlp;

typedef struct {
  int32_t strict;       /* 1: strict comparison (see above); 0: default */
  int32_t order;        /* pa_order */
  int32_t npairs;       /* PA_ORDER_GIVEN: nrel - 1 joins */
  const int32_t* pairs; /* PA_ORDER_GIVEN: 2*npairs slot indices, host; slots
                           0..nrel-1 are the plots, join t creates slot nrel+t */
  const pa_mlp* model;  /* PA_ORDER_LEARNED: the cost model */
  int32_t ncand;        /* PA_ORDER_LEARNED: candidate orders per system (0: 16) */
} pa_options;

typedef struct {
  double pixels_plotted;     /* sum over relations of the pixels evaluated */
  double pixel_ops_dense;    /* sum over joins of r^Lambda (Sec. 3.5, naive cost) */
  double words_or_executed;  /* reserved, 0: the table words the row-OR kernels
                                OR are counted only in profiling mode and
                                reported by pa_profile_read ("words_or") */
  int32_t n_plots;
  int32_t n_joins;
  int32_t n_reshapes;
  int32_t n_launches;        /* kernels and memsets enqueued by the call */
  int64_t peak_words;        /* largest intermediate array, words */
  int64_t workspace_bytes;   /* workspace in use by the call */
  double mma_macs;           /* multiply-adds of the clusters contracted on the
                                tensor cores: sum of nbatch * M * N * K */
  int32_t n_mma;             /* clusters contracted on the tensor cores */
} pa_stats;

/* One independent system for the batched entry points: its own variables,
 * boxes, relations and exposed set (same meaning as pa_solve_network's
 * arguments; all pointers are host pointers). */
typedef struct {
  int32_t nvars;
  const pa_axis* axes;
  int32_t nrel;
  const pa_relation* rels;
  int32_t nexposed;
  const int32_t* exposed;
} pa_system;

typedef struct pa_ctx pa_ctx;
typedef struct pa_batch pa_batch;

/* Create a context on `device`.  workspace_cap bounds the scratch memory the
 * context may hold (0: no bound).  Returns PA_ERR_CUDA when the device cannot
 * be used (no GPU, wrong architecture).  A context is used by one host thread
 * at a time, and its calls share one workspace: calls on different streams
 * must be ordered by the caller (one context per stream otherwise). */
pa_status pa_create(pa_ctx** ctx, int device, size_t workspace_cap);
void pa_destroy(pa_ctx* ctx);
const char* pa_last_error(const pa_ctx* ctx);
/* Block the host until the work this context enqueued on `stream` is done and
 * report any device-side error. */
pa_status pa_sync(pa_ctx* ctx, void* stream);

/* Kernel timing.  While enabled, every kernel (and memset) the context enqueues
 * is bracketed by a pair of CUDA events on the same stream.  pa_profile_read
 * waits for those events, adds the elapsed times up per kernel name and clears
 * the record.  names receives up to max_kernels NUL-terminated names of at most
 * 31 characters, 32 bytes apart; launches[k] and total_ms[k] the count and the
 * summed milliseconds of kernel k; *nkernels the number of distinct kernels.
 * The last entry is not a kernel: "words_or", whose launches field counts the
 * 64-bit words the contraction kernels OR-ed while timing was on. */
pa_status pa_profile_enable(pa_ctx* ctx, int32_t on);
pa_status pa_profile_read(pa_ctx* ctx, int32_t max_kernels, char* names, int64_t* launches,
                          double* total_ms, int32_t* nkernels);

/* How a matrix-form cluster (Sec. 3.5) is contracted.  Both give the same
 * bits.  PA_PATH_ROWOR: bit-packed row-OR on the CUDA cores (work follows the
 * set bits of A).  PA_PATH_MMA: 0/1 E4M3 matrix product on the tensor cores
 * (tcgen05, FP32 accumulation, thresholded at > 0; work follows M x N x K;
 * both operands are first expanded once into E4M3 byte arrays in the
 * workspace, (M + N) x K bytes per batch entry).
 * PA_PATH_AUTO (default): per cluster, the faster by the context's rates and
 * the operands' estimated densities. */
typedef enum { PA_PATH_AUTO = 0, PA_PATH_ROWOR = 1, PA_PATH_MMA = 2 } pa_path;
pa_status pa_set_contract_path(pa_ctx* ctx, int32_t path);

/* The rates PA_PATH_AUTO compares.  Defaults were measured on a GB300;
 * pa_autotune re-measures them on this context's GPU (a 2048 x 2048 x 2048
 * contraction of random operands through each path, five runs timed with CUDA
 * events on `stream` after one warm-up run) and keeps them for later calls.
 * The row-OR rate depends on the density of A and is measured at 2 % and 16 %
 * (log-linear in between); the tensor-core rate includes the expansion of both
 * operands.  Blocks the host; allocates and frees about 10 MB of device memory. */
typedef struct {
  double rowor_words_per_us;        /* 64-bit words OR-ed by the row-OR kernel, A 2 % dense */
  double rowor_words_per_us_dense;  /* the same, A 16 % dense */
  double mma_macs_per_us;           /* multiply-adds of the tensor-core path */
} pa_rates;
pa_status pa_autotune(pa_ctx* ctx, pa_rates* out, void* stream);
pa_status pa_get_rates(const pa_ctx* ctx, pa_rates* out);
pa_status pa_set_rates(pa_ctx* ctx, const pa_rates* rates);

/* Check of the failure path of the bounded device waits: enqueues one kernel
 * whose mbarrier wait can never complete and gives up after limit_ns
 * (1e3 .. 2e9), exactly as the contraction kernels' waits do, leaving the
 * context's error word set.  The next pa_sync on that stream returns
 * PA_ERR_TIMEOUT, clears the word, and the context stays usable. */
pa_status pa_wait_selftest(pa_ctx* ctx, int64_t limit_ns, void* stream);

/* Measured throughput of the pipes this library's kernels run on (the
 * denominators of their rooflines), on the context's GPU: long chains of
 * independent operations in 1024 threads on every SM, timed with CUDA events
 * after a warm-up launch on `stream`, with each block's SM cycle counter.
 * Blocks the host; allocates and frees a few KB of device memory. */
typedef struct {
  int32_t sms;                  /* streaming multiprocessors used */
  double sm_clock_hz;           /* SM clock during the LOP3 probe */
  double lop3_ops_per_s;        /* 32-bit three-input logic operations (lop3.b32) */
  double lop3_per_clk_sm;
  double smem_bytes_per_s;      /* shared-memory load bandwidth, 8-byte loads */
  double smem_bytes_per_clk_sm;
  double fp32_flops_per_s;      /* FP32 fused multiply-add, 2 flops each */
  double fp32_flops_per_clk_sm;
  double fp64_flops_per_s;      /* FP64 multiply and add, not fused */
  double fp64_flops_per_clk_sm;
} pa_peaks;
pa_status pa_measure_peaks(pa_ctx* ctx, pa_peaks* out, void* stream);

/* Number of uint64 words of a pa_array of this shape (host only, no GPU). */
int64_t pa_array_words(int32_t ndim, const int32_t* res);

/* A valid tolerance for the polynomial relation `rel` on the box `axes`
 * (indexed by variable id), Sec. 3.2 Eq. (continuity): eps with
 * |f(x) - f(c)| <= eps whenever x lies in the pixel centred at c (an
 * expression relation returns PA_ERR_UNSUPPORTED).  Computed on the host as
 *   (1 + 2^-30) * sum_p S_p * delta_p / 2   (PA_RULE_CORNER: delta_p, c a corner),
 *   S_p = sum_e |c_e| e_p M_p^(e_p - 1) prod_{q != p} M_q^(e_q),  M_q = max(|lo_q|, |hi_q|),
 * in a fixed order (ports ascending, monomials in graded lex order, factors left
 * to right).  Host only, no GPU. */
pa_status pa_valid_tolerance(const pa_relation* rel, const pa_axis* axes, int32_t nvars,
                             double* eps_out);

/* Plot one relation (Sec. 3.2, sample-in-center plot, or the corner rule when
 * rel->rule is PA_RULE_CORNER) into `out`, whose vars
 * must be the relation's distinct variables in order of first appearance and
 * whose res must match `axes`. */
pa_status pa_plot(pa_ctx* ctx, const pa_relation* rel, const pa_axis* axes, int32_t nvars,
                  int32_t strict, pa_array* out, void* stream);

/* One two-array cluster (Sec. 3.5): out = Eq. (GAM) applied to A and B with the
 * outer pack `keep`: out(e') = OR over the values of every variable of A or B
 * not in keep of A(e_A) AND B(e_B).  out->vars must equal keep (distinct, each
 * a variable of A or B); shared variables must have equal res.  A, B and out
 * must not overlap. */
pa_status pa_contract(pa_ctx* ctx, const pa_array* A, const pa_array* B, int32_t nkeep,
                      const int32_t* keep, pa_array* out, void* stream);

/* One cluster over the counting semiring instead of the Boolean one (the
 * paper notes that its arrays may take values in any semi-ring, such as the
 * natural numbers, to count solutions instead of marking them: Sec. 2.2,
 * footnote on plots): counts(e') = sum over the values of every variable of A
 * or B not in keep of A(e_A) * B(e_B), the number of latent pixel tuples
 * behind each output pixel.  `counts` is a device array of uint32, one per
 * output pixel, row-major over keep (last variable fastest, not bit-packed).
 * Runs on the tensor cores (0/1 E4M3 products summed in FP32): exact because
 * every sum is an integer of at most K = the product of the summed
 * variables' resolutions, which must be <= 2^24.  Supported when every
 * summed variable belongs to both A and B and B keeps a variable of its own;
 * other clusters return PA_ERR_UNSUPPORTED. */
pa_status pa_contract_count(pa_ctx* ctx, const pa_array* A, const pa_array* B, int32_t nkeep,
                            const int32_t* keep, uint32_t* counts, void* stream);

/* The whole method (Sec. 3.6): plot every relation, join the plots pairwise in
 * the order chosen by opts->order, and leave the array over `exposed` (in that
 * axis order) in `out`.  nexposed = 0 gives one bit: does the system have a
 * solution pixel.  opts and stats may be NULL.  The order is planned on the
 * host from the shapes alone; the call waits for the device only when the
 * host is more than four calls ahead of it (the descriptor uploads go through
 * four pinned staging slots).
 * The context keeps the program of its last call: a call whose arguments (the
 * coefficients included, compared by value), stream and output pointer, and
 * the context's path, rates, join logs and profiling state, are all the same
 * skips planning and launches that program again (from the second such call
 * on, as one CUDA graph).  Every call still reads the host coefficients,
 * uploads its descriptors and runs every kernel.  Orders of PA_ORDER_LEARNED
 * are never kept (the model may change between calls). */
pa_status pa_solve_network(pa_ctx* ctx, int32_t nvars, const pa_axis* axes, int32_t nrel,
                           const pa_relation* rels, int32_t nexposed, const int32_t* exposed,
                           const pa_options* opts, pa_array* out, pa_stats* stats,
                           void* stream);

/* Many independent systems at once (Sec. 3.6 applied to each): all plots in
 * one launch pair, and the joins of equal depth in all the systems' cluster
 * trees in one contraction launch per tile width.  outs[k] receives system k's
 * array over its exposed variables.  opts->order must not be PA_ORDER_GIVEN. */
pa_status pa_solve_batch(pa_ctx* ctx, int32_t nsys, const pa_system* systems, pa_array* outs,
                         const pa_options* opts, pa_stats* stats, void* stream);

/* A planned batch: the same work as pa_solve_batch, planned once into the
 * batch's own device memory and captured as one CUDA graph (the host-to-device
 * copy of every descriptor and coefficient, then every launch).  pa_batch_run
 * replays it on `stream`; the outputs and the coefficients are those given to
 * pa_batch_create, whose host arrays may be freed after it returns.  A batch
 * must not run concurrently with itself.  pa_batch_destroy waits for the
 * device before freeing its memory. */
pa_status pa_batch_create(pa_ctx* ctx, int32_t nsys, const pa_system* systems, pa_array* outs,
                          const pa_options* opts, pa_batch** batch);
pa_status pa_batch_run(pa_batch* batch, void* stream);
pa_status pa_batch_stats(const pa_batch* batch, pa_stats* stats);
void pa_batch_destroy(pa_batch* batch);

/* pa_solve_network for callers that cannot let the library allocate memory:
 * real-time loops that cannot afford the device-wide synchronisation of
 * cudaFree, hosts whose GPU memory is budgeted by someone else (a serving
 * process that hands the library no allocator), and code that must not grow
 * its footprint after start-up.  It allocates nothing: no cudaMalloc, no
 * cudaFree, no pinned host memory, no context.  Its workspace is one static
 * device array of PA_STATIC_SCRATCH_BYTES (16 MiB) that every GPU which loads
 * the library holds until the process exits; the inputs and `out` are the
 * caller's, exactly as for pa_solve_network, and the results are identical.
 * The paper has no counterpart.
 *   - Runs on the current CUDA device.  The first call on a device looks up the
 *     array's device address (cudaGetSymbolAddress) and caches it.
 *   - A system whose workspace would exceed the array returns PA_ERR_TOO_LARGE
 *     before any launch; stats->workspace_bytes (when stats is not NULL) then
 *     holds the bytes it would need.
 *   - Every call shares the array and sees the previous call's contents; each
 *     call clears what must start at zero.  Calls whose work overlaps on the
 *     GPU (other streams, other threads) race on the array: order them.
 *   - Orders: PA_ORDER_GREEDY, PA_ORDER_LEFT and PA_ORDER_GIVEN.  The learned
 *     order needs a context's model and returns PA_ERR_INVALID_ARG here.
 *   - Argument errors return PA_ERR_INVALID_ARG; there is no context, so no
 *     message; a device wait that runs out is not reported by this entry.
 *   - The descriptor upload reads pageable host memory and returns once the
 *     driver has copied it. */
#define PA_STATIC_SCRATCH_BYTES (16u << 20)
pa_status pa_solve_network_static(int32_t nvars, const pa_axis* axes, int32_t nrel,
                                  const pa_relation* rels, int32_t nexposed,
                                  const int32_t* exposed, const pa_options* opts, pa_array* out,
                                  pa_stats* stats, void* stream);

/* ------------------------------------------------------------ learned order
 * A small FP32 network (PA_FEATURES inputs, `nlayers` hidden layers of
 * `hidden` ReLU units, one linear output) predicts log2(microseconds)/8 of a
 * join from PA_FEATURES numbers the library computes for it: sizes of the
 * matrix form, the naive cost r^Lambda (Sec. 3.5), estimated operand and
 * result densities, reshape volume.  Plot densities are estimated on the host
 * from 512 sampled pixel centres, join densities propagated under an
 * independence assumption, so planning never waits for the solve.
 * PA_ORDER_LEARNED ranks `ncand` candidate orders per system (greedy, the
 * least-naive-cost tree of PA_ORDER_OPTIMAL, smallest-cost-first,
 * left-to-right and seeded randomised greedy variants) by their total time:
 * a join that pa_join_log has timed on this context (the same join of the
 * same relations) counts with its measured microseconds, any other with the
 * model's prediction.  The greedy order is the judge: the learned choice is
 * kept only when its total is lower than greedy's and its largest
 * intermediate is at most 4x the greedy one, so logging a system's greedy
 * order first makes greedy's side of the comparison measured.  Any order
 * gives the same bits. */
#define PA_FEATURES 16
pa_status pa_mlp_create(pa_ctx* ctx, int32_t hidden, int32_t nlayers, uint64_t seed,
                        pa_mlp** model);
void pa_mlp_destroy(pa_mlp* model);
int64_t pa_mlp_num_params(const pa_mlp* model);
/* Parameters and the last gradient as one flat FP32 vector (host memory):
 * per layer the weights [out][in] row-major, then the biases. */
pa_status pa_mlp_get_params(const pa_mlp* model, float* params);
pa_status pa_mlp_set_params(pa_mlp* model, const float* params);
pa_status pa_mlp_get_grads(const pa_mlp* model, float* grads);
/* y[n] = net(x[n][PA_FEATURES]); device pointers, enqueued on `stream`. */
pa_status pa_mlp_forward(pa_mlp* model, const float* x, int32_t n, float* y, void* stream);
/* Gradient of 0.5 * mean_n (net(x_n) - t_n)^2 with respect to the parameters
 * (device x, t); *loss (host, may be NULL) receives the loss after a sync. */
pa_status pa_mlp_backward(pa_mlp* model, const float* x, const float* t, int32_t n, float* loss,
                          void* stream);
/* One Adam step on the last gradient. */
pa_status pa_mlp_adam(pa_mlp* model, float lr, float beta1, float beta2, float eps, void* stream);

/* Solver log for training the cost model: solve one system with one join per
 * launch, time every join with CUDA events (its reshapes included) and count
 * the set bits of its result.  Writes, for join t < *njoins (at most
 * max_joins), features[t*PA_FEATURES ..], micros[t] and densities[t] (the
 * result's fraction of set bits).  Synchronises the stream. */
pa_status pa_join_log(pa_ctx* ctx, const pa_system* sys, const pa_options* opts, pa_array* out,
                      int32_t max_joins, float* features, float* micros, float* densities,
                      int32_t* njoins, void* stream);

/* The orders PA_ORDER_LEARNED would use, with the judge's inputs: for system k,
 * pairs_out[offsets..] receives its 2*(nrel_k-1) slot indices (systems packed
 * one after another), learned[k] whether the learned order was kept, and
 * pred_us[2k], pred_us[2k+1] the judge's totals of the chosen and the greedy
 * order (measured joins measured, the rest predicted).  Runs one forward pass
 * on the GPU and waits for it. */
pa_status pa_plan_learned(pa_ctx* ctx, const pa_mlp* model, int32_t nsys, const pa_system* systems,
                          int32_t ncand, int32_t* pairs_out, int32_t* learned, float* pred_us);

/* The join order pa_solve_network would use (host only, no GPU) for order
 * PA_ORDER_GREEDY, PA_ORDER_LEFT or PA_ORDER_OPTIMAL: writes 2*(nrel-1) slot
 * indices into pairs_out (same numbering as pa_options.pairs), the naive cost
 * sum r^Lambda of its joins and its largest intermediate in bits. */
pa_status pa_plan_order(int32_t nvars, const pa_axis* axes, int32_t nrel, const pa_relation* rels,
                        int32_t nexposed, const int32_t* exposed, int32_t order,
                        int32_t* pairs_out, double* pixel_ops_out, int64_t* peak_bits_out);

/* Cost of a cluster tree (Sec. 3.5, cost polynomial evaluated at the given
 * resolutions), host only.  Links 0..nlinks-1 have resolutions link_res.  Inner
 * pack i (0..npacks-1) has pack_nports[i] ports wired to the links listed in
 * pack_links (concatenated); the outer pack's ports are wired to outer_links.
 * The tree is a list of clusters: cluster t joins join_nchildren[t] slots
 * listed in join_children (concatenated); slots 0..npacks-1 are the packs and
 * cluster t creates slot npacks + t; the last cluster is the root.  A slot's
 * intermediate pack is the set of its links that also touch something outside
 * it (another pack or the outer pack).  A cluster costs r^(links of its
 * children's packs); the root also counts the outer pack's links.  Writes the serial cost (sum over the clusters) and the
 * parallel cost (a cluster's cost plus the largest parallel cost among its
 * children). */
pa_status pa_tree_cost(int32_t nlinks, const double* link_res, int32_t npacks,
                       const int32_t* pack_nports, const int32_t* pack_links,
                       int32_t nouter, const int32_t* outer_links, int32_t njoins,
                       const int32_t* join_nchildren, const int32_t* join_children,
                       double* serial_cost, double* parallel_cost);

#ifdef __cplusplus
}
#endif

#endif /* PA_H_ */
