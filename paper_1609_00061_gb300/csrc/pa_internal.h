// Internal declarations shared by the CUDA translation units of the pixel array
// engine.  Nothing here is part of the public C interface (include/pa.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pa.h"

namespace pa {

// Raise kernel `fn`'s dynamic shared-memory limit on the current device only
// when a launch needs more than any earlier one did (the attribute call costs
// host time on every launch otherwise).  Thread-safe.
cudaError_t smem_limit(const void* fn, size_t bytes);

constexpr int kMaxDim = PA_MAX_DIM;
constexpr int kMaxDeg = PA_MAX_DEGREE;

// ------------------------------------------------------------------ plotting
// One relation to plot.  Coefficients are in "nest order": the order in which
// the nested evaluation visits the monomials (last port outermost, every
// exponent ascending), so the device reads them front to back.
//
// Pixel centres are computed on the device as lo + ((double)i + 0.5) * delta
// with delta = (hi - lo) / res divided on the host (IEEE division is correctly
// rounded on both, so the value is the one pa.h defines).
struct PlotJob {
  const double* coeffs;             // device, nest order
  uint64_t* out;                    // device, pa_array layout
  double lo[kMaxDim];               // per port: range start of its variable
  double delta[kMaxDim];            // per port: pixel width of its variable
  const float* y32;                 // [res_last] FP32 centres of the last port (hoisted jobs)
  int64_t nrows;                    // rows = product of all but the last array axis
  int64_t row_words;                // ceil(res_last / 64)
  int64_t tile0;                    // first block of this job in the plot launch
  int32_t rows_per_tile;
  int32_t arity, degree, kind, strict;
  int32_t hoisted;                  // 1: the last port is the last array axis, used once
  int32_t ndim;                     // array axes (distinct variables)
  int32_t res[kMaxDim];             // array axis resolutions
  int32_t port_axis[kMaxDim];       // port -> array axis
  double eps;
  float eps32;                      // eps rounded to FP32
  float kfac;                       // FP32 filter: error bound factor on sum |g_j| Y^j
  float abs_margin;                 // FP32 filter: margin for eps rounding / underflow
  float ymax;                       // >= |y| for every FP32 centre of the last port
  float hword;                      // >= distance from a word's pixel 32 to any of its 64 centres
  int32_t block_off[kMaxDeg + 1];   // nest-order offset of the coefficients with e_last = j
};

// One FP32 centre table: y32[i] = fl32(lo + (i + 1/2) delta) for i < res, the
// last-port centres shared by every hoisted plot job over that axis.
struct CentreTab {
  float* y32;
  double lo, delta;
  int64_t item0;  // first item of this table in the centre-table launch
  int64_t res;
};
// One expression relation to plot (expr.cu): the postfix program and its
// constants on the device, the pixel grid as for PlotJob; word0 is the first
// word of this job in the launch's flat word space.
struct ExprJob {
  const int32_t* prog;
  const double* consts;
  uint64_t* out;
  double lo[kMaxDim];
  double delta[kMaxDim];
  double eps;
  int64_t nrows, row_words, word0;
  int32_t nops, arity, kind, strict, ndim;
  int32_t res[kMaxDim];
  int32_t port_axis[kMaxDim];
};
// Every expression plot of a call in one launch, one thread per pixel (a
// warp per 32-pixel half of an output word).
void launch_plot_expr(const ExprJob* d_jobs, int njobs, int64_t total_words, cudaStream_t s);

// One relation plotted by the corner rule (pa.h, pa_rule): a polynomial
// (prog == nullptr; coefficients in nest order) or an expression program.
// lo and delta are per port; port_axis maps a port to its axis of `out`.
struct CornerJob {
  const int32_t* prog;
  const double* consts;
  const double* coeffs;
  uint64_t* out;
  double lo[kMaxDim];
  double delta[kMaxDim];
  double eps;
  int64_t nrows, row_words, word0;
  int32_t nops, degree, arity, kind, strict, ndim;
  int32_t res[kMaxDim];
  int32_t port_axis[kMaxDim];
};
// Every corner-rule plot of a call in one launch, one thread per output byte.
void launch_plot_corner(const CornerJob* d_jobs, int njobs, int64_t total_words, cudaStream_t s);

// A range of words to clear: words [w0, w0 + words) of the launch's flat
// index space are p[0 .. words).
struct ZeroRange {
  uint64_t* p;
  int64_t words;
  int64_t w0;
};
// Every table in one launch (one thread per centre), before the plot launch;
// the plot kernel waits for it only after its row set-up (programmatic
// dependent launch), so the two overlap.
void launch_plot_centres(const CentreTab* d_tabs, int ntabs, int64_t total_items, cudaStream_t s);
// One launch plots every job: blocks of rows_per_tile rows, each computing its
// rows' polynomials and thresholds in shared memory first.  common_degree: the
// degree shared by every job (selects a specialised kernel), or -1 when they
// differ.
// The same launch also clears the `nzero` ranges (zero_words words in all)
// that later contractions OR their results into, so that no separate memset
// sits between the launches.
// Plot blocks the GPU holds at once (all SMs), for the kernel of this degree.
int plot_resident_blocks(int common_degree);
void launch_plot(const PlotJob* d_jobs, int njobs, int64_t total_tiles, int max_rows_per_tile,
                 int max_degree, int common_degree, int max_res_last, int64_t max_tile_words,
                 const ZeroRange* d_zero, int nzero, int64_t zero_words, cudaStream_t s);

// ------------------------------------------------------------- bit arrays
// A bit-packed array with `inner` trailing axes flattened into packed rows:
// rowlen = prod(res[ndim-inner..]), row_words = ceil(rowlen / 64),
// nrows = prod(res[..ndim-inner]).  The public pa_array layout is inner = 1
// (inner = 0 for ndim = 0).
struct BitArr {
  uint64_t* w = nullptr;
  int ndim = 0;
  int inner = 0;
  int vars[2 * kMaxDim] = {};
  int64_t res[2 * kMaxDim] = {};
  int64_t rowlen() const {
    int64_t r = 1;
    for (int a = ndim - inner; a < ndim; ++a) r *= res[a];
    return r;
  }
  int64_t row_words() const { return (rowlen() + 63) / 64; }
  int64_t nrows() const {
    int64_t r = 1;
    for (int a = 0; a < ndim - inner; ++a) r *= res[a];
    return r;
  }
  int64_t words() const { return nrows() * row_words(); }
  int64_t bits() const { return nrows() * rowlen(); }
};

// Reshape modes (contract.cu):
//  kReshapeBits       any mapping; every output bit gathered on its own
//  kReshapeWords      the last output axis runs along input words: every output
//                     word is one input word (OR-ed over reduced axes), found
//                     through word strides u_in over the output-word axes u_res
//  kReshapeTranspose  the last output axis L steps by input rows or whole
//                     input words and the input's last axis J is kept: 64 x 64
//                     bit blocks are transposed; u_res / u_in / u_out cover
//                     the other axes
enum { kReshapeBits = 0, kReshapeWords = 1, kReshapeTranspose = 2 };

// General gather: out bit (axes of `out`) = OR over the reduced input axes of
// the input bit with the same values of the shared axes.  An output axis that
// is missing from the input has zero strides (broadcast).
struct ReshapeDesc {
  const uint64_t* in;
  uint64_t* out;
  int64_t out_nrows, out_row_words, out_rowlen;
  int32_t out_ndim, out_inner;
  int64_t out_res[2 * kMaxDim];
  int64_t row_stride[2 * kMaxDim];  // per output axis: input row-index stride
  int64_t col_stride[2 * kMaxDim];  // per output axis: input column (bit) stride
  int32_t nred;
  int64_t red_res[2 * kMaxDim];
  int64_t red_row_stride[2 * kMaxDim];
  int64_t red_col_stride[2 * kMaxDim];
  int64_t in_row_words;
  int32_t mode;                      // kReshape*
  int32_t row_any;                   // bit mode: all packed input axes reduced (see contract.cu)
  int32_t nu;                        // axes of the word / tile decomposition
  int64_t u_res[2 * kMaxDim];
  int64_t u_in[2 * kMaxDim];         // input words per step of the axis
  int64_t u_out[2 * kMaxDim];        // output words per step (transpose mode)
  int64_t red_in_w[2 * kMaxDim];     // words mode: input words per reduced step
  int64_t tQ, tR;                    // transpose: resolutions of J and L
  int64_t t_in_L, t_out_J;           // input words per L step, output words per J step
  int64_t n_other;                   // transpose: product of u_res
};
// Kernel variant of a reshape (kRs*) and its block count; a launch runs a
// table of n descriptors of one kind, problem p on blocks [cta0[p], cta0[p+1])
// (device arrays), grid = cta0[n].
enum { kRsBits = 0, kRsWords32 = 1, kRsWords64 = 2, kRsTranspose = 3 };
int reshape_kind(const ReshapeDesc& d);
int64_t reshape_blocks(const ReshapeDesc& d);
void launch_reshape(const ReshapeDesc* d_descs, const int64_t* d_cta0, int n, int kind,
                    int64_t grid, cudaStream_t s);

// cudaSuccess when the library holds kernel code the current device can run
cudaError_t probe_kernel_image();

// Clusters that are not matrix products, batched like the contractions:
// kEwOuter  C row r (r = b * M + m) is B row b (nw words) when bit r of A is set;
// kEwDot    bit r of C = any(A row r AND B row r / M), rows of nw <= 16 words;
// kEwDotWide the same for longer rows, OR-ed into a cleared C;
// kEwAnd    C = A AND B over `rows` words.
enum { kEwOuter = 0, kEwDot = 1, kEwDotWide = 2, kEwAnd = 3 };
struct EwJob {
  const uint64_t* a;
  const uint64_t* b;
  uint64_t* c;
  int64_t rows, m, nw;
  int32_t kind;
};
int64_t ewise_blocks(const EwJob& j);
void launch_ewise(const EwJob* d_jobs, const int64_t* d_cta0, int n, int64_t grid, cudaStream_t s);

// C[b*M + m, :] |= B[b*K + k, :] for every set bit k of A[b*M + m, :].
// One CTA owns a tile of B (Kc rows x Nt words of batch b) in shared memory and
// a run of output rows; see contract.cu.
struct RowOrDesc {
  const uint64_t* A;
  const uint64_t* B;
  uint64_t* C;
  int64_t nbatch, M, K, Nw;   // Nw = words per B / C row
  int64_t a_row_words;        // = ceil(K / 64)
  int32_t Nt;                 // words per tile (power of two <= 32)
  int32_t Kc;                 // B rows per tile (multiple of 256 when use_tma)
  int64_t n_tiles, k_chunks, row_splits, rows_per_split;
  int32_t atomic;             // 1: C pre-zeroed, results OR-ed in atomically
  int32_t use_tma;            // 1: stage the tile with cp.async.bulk.tensor
  int* err;                   // device error word: set when a bounded wait runs out
  unsigned long long* stat;   // when not null: += shared-memory words OR-ed (timing mode)
};
// Choose the tile shape and grid for a contraction of this shape; the grid
// aims at about target_ctas CTAs (several contractions can share one launch).
void rowor_plan(RowOrDesc& d, int64_t target_ctas);
size_t rowor_smem_bytes(const RowOrDesc& d);
int64_t rowor_ctas(const RowOrDesc& d);
// TMA descriptor of d.B (all zero when d.use_tma is 0)
cudaError_t rowor_encode_map(const RowOrDesc& d, CUtensorMap* map);
// Independent contractions with the same tile width Nt in one launch:
// descriptors, tensor maps and CTA offsets (nprob + 1 entries) on the device.
cudaError_t launch_rowor(const RowOrDesc* d_descs, const CUtensorMap* d_maps,
                         const int64_t* d_cta0, int nprob, int64_t grid, size_t smem, int Nt,
                         cudaStream_t s);
// cuTensorMapEncodeTiled from the driver (null when unavailable)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder();

// Tensor-core contraction (mma.cu): the same problem as RowOrDesc, from the
// same bit-packed layouts, as a 0/1 E4M3 matrix product thresholded at > 0.
// The operands are first expanded into the byte arrays Ab and Bb.
struct MmaDesc {
  const uint64_t* A;          // [nbatch][M][a_row_words], K bits per row
  const uint64_t* B;          // [nbatch][K][Nw], N bits per row
  uint64_t* C;                // [nbatch][M][Nw]
  uint8_t* Ab;                // [nbatch][M][Kp] E4M3 bytes
  uint8_t* Bb;                // [nbatch][N][Kp] E4M3 bytes
  int64_t M, N, K, Kp, Nw, a_row_words, nbatch;
  int64_t m_tiles, n_tiles;
  int32_t BN;                 // columns per tile: 64, 128 or 256
  int* err;                   // device error word: set when a bounded wait runs out
  uint32_t* counts;           // when not null: the sums themselves, [nbatch][M][N]
                              // (counting semiring), and C is not written
  // Occupancy bitmaps of the 128 x 128 tiles (cleared before the expansion,
  // set by it): bit kb of occ_a[(b * m_tiles + mt) * kb_words + kb / 32] when
  // A's rows 128 mt.. and K values 128 kb.. hold a set bit, likewise occ_b per
  // BN-column tile.  The contraction multiplies only the K blocks both hold.
  uint32_t* occ_a;
  uint32_t* occ_b;
  int64_t kb_words;
  // K split: ksplit CTAs per output tile, each summing kchunk consecutive
  // 128-value K blocks and OR-ing its bits into C, which starts at zero
  // (Boolean products only; 1 when every tile is summed by one CTA)
  int32_t ksplit, kchunk;
};
// 32-bit words of the two occupancy bitmaps of a planned problem
int64_t mma_occ_words(const MmaDesc& d);
void mma_plan(MmaDesc& d);    // BN, Nw, Kp and the tile counts from M, N, K, nbatch
int64_t mma_ctas(const MmaDesc& d);
size_t mma_smem_bytes();
// TMA descriptors of Ab and Bb (needs d.Ab, d.Bb set)
cudaError_t mma_encode_maps(const MmaDesc& d, CUtensorMap* maps2);
// Expand A and B of every problem of a table into Ab and Bb (two launches;
// blocks per problem from unpack_blocks_a / _b, the largest over the table).
int64_t unpack_blocks_a(const MmaDesc& d);
int64_t unpack_blocks_b(const MmaDesc& d);
void launch_unpack(const MmaDesc* d_descs, int nprob, int64_t blocks_a, int64_t blocks_b,
                   cudaStream_t s);
// Independent problems in one launch: descriptors, two tensor maps per problem
// and CTA offsets (nprob + 1 entries) on the device.
cudaError_t launch_mma(const MmaDesc* d_descs, const CUtensorMap* d_maps, const int64_t* d_cta0,
                       int nprob, int64_t grid, cudaStream_t s);
// out[i] = in[src(i)] for a row-major array whose axes are a permutation of
// the input's: out axis a has extent d_ext[a] and steps d_stride[a] elements
// of the input (one thread per output element; d_ext and d_stride are DEVICE
// arrays of ndim entries).
void launch_permute_u32(const uint32_t* in, uint32_t* out, int ndim, const int64_t* d_ext,
                        const int64_t* d_stride, int64_t total, cudaStream_t s);
// Throughput probe `which` (0: 32-bit LOP3, 1: shared-memory load bytes,
// 2: FP32 FMA flops, 3: FP64 mul + add flops) over every SM: operations per
// second, per SM per cycle, and the SM clock it ran at.
cudaError_t run_probe(int which, int sms, cudaStream_t s, double* per_s, double* per_clk_sm,
                      double* clock_hz);
// Random bit rows of the given density (autotuning inputs); padding stays zero.
void launch_random_bits(uint64_t* w, int64_t nwords, int64_t row_words, int64_t valid,
                        double density, uint64_t seed, cudaStream_t s);

// *out += number of set bits in w[0..nwords) (padding bits are zero)
void launch_popcount(const uint64_t* w, int64_t nwords, unsigned long long* out, cudaStream_t s);
// One bounded mbarrier wait that nothing completes (sets *err after limit_ns).
cudaError_t launch_wait_selftest(int* err, long long limit_ns, cudaStream_t s);

// ----------------------------------------------------------- host helpers
int64_t coeff_count(int n, int degree);
// graded lex rank of every monomial in nest order (host)
std::vector<int64_t> nest_order(int n, int degree);
// A valid tolerance: (1 + 2^-30) sum_p S_p delta_p width, width = 1/2 for the
// centre rule (a pixel's points lie within delta_p / 2 of its centre) and 1
// for the corner rule.
double valid_tolerance(int n, int degree, const double* coeffs, const double* lo,
                       const double* hi, const int32_t* res, double width);

}  // namespace pa
