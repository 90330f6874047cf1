// Contraction kernels: Eq. (GAM) of Sec. 3.3 for one two-array cluster (Sec. 3.5)
// over the Boolean semiring, on bit-packed arrays.
//
// After the planner has brought both operands into matrix form
//   A[b][m][k]  (k packed along rows)   and   B[b][k][n]  (n packed along rows),
// the cluster is C[b][m][n] = OR_k A[b][m][k] AND B[b][k][n], computed row-wise:
// row (b, m) of C is the OR of the rows B[b][k][:] selected by the set bits of
// row (b, m) of A.  Curve plots are sparse and their set bits come in runs, so
// with ORs of aligned blocks of B rows the work is proportional to the number
// of maximal aligned all-ones blocks of A (at most its set bits) times the
// packed width of B, not to M*K*N.
#include <cuda.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>

#include "pa_internal.h"

namespace pa {

// --------------------------------------------------------------- reshape
// Every reshape launch runs a table of descriptors: problem p owns blocks
// [cta0[p], cta0[p+1]) and its descriptor is copied into shared memory; the
// kernels' grid-stride loops run over the problem's own blocks.  (One launch
// per kind serves all reshapes of one tree level of every system of a batch.)
struct RsCtx {
  int64_t bid, nblk;
};
__device__ __forceinline__ RsCtx rs_pick(const ReshapeDesc* __restrict__ descs,
                                         const int64_t* __restrict__ cta0, int n, ReshapeDesc* sd) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cta0[mid] <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const int64_t* src = reinterpret_cast<const int64_t*>(descs + lo);
  int64_t* dst = reinterpret_cast<int64_t*>(sd);
  for (int i = threadIdx.x; i < (int)(sizeof(ReshapeDesc) / 8); i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  return RsCtx{(int64_t)blockIdx.x - cta0[lo], cta0[lo + 1] - cta0[lo]};
}

// Bit mode: one warp per output word, one lane per bit (two ballots pack the
// 64 bits).  Every bit is decoded and gathered on its own, OR-ed over the
// reduced axes with an early exit.  With row_any set, every packed input axis
// is reduced and red_* hold only the reduced row axes: a bit is then the OR of
// whole input rows, scanned by words (padding bits are zero).
__global__ void reshape_kernel(const ReshapeDesc* __restrict__ descs, const int64_t* __restrict__ cta0,
                               int n) {
  __shared__ ReshapeDesc sd;
  const RsCtx rc = rs_pick(descs, cta0, n, &sd);
  const ReshapeDesc& d = sd;
  const int lane = threadIdx.x & 31;
  const int64_t total = d.out_nrows * d.out_row_words;
  const int outer = d.out_ndim - d.out_inner;
  int64_t red_total = 1;
  for (int q = 0; q < d.nred; ++q) red_total *= d.red_res[q];
  const int64_t nwarps = rc.nblk * (blockDim.x >> 5);
  for (int64_t ow = rc.bid * (blockDim.x >> 5) + (threadIdx.x >> 5); ow < total; ow += nwarps) {
    const int64_t orow = ow / d.out_row_words, w = ow % d.out_row_words;
    int64_t brow = 0, bcol = 0, rest = orow;
    for (int a = outer - 1; a >= 0; --a) {
      const int64_t v = rest % d.out_res[a];
      rest /= d.out_res[a];
      brow += v * d.row_stride[a];
      bcol += v * d.col_stride[a];
    }
    uint32_t half[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t ocol = w * 64 + h * 32 + lane;
      bool bit = false;
      if (ocol < d.out_rowlen) {
        int64_t rr = brow, cc = bcol, rest2 = ocol;
        for (int a = d.out_ndim - 1; a >= outer; --a) {
          const int64_t v = rest2 % d.out_res[a];
          rest2 /= d.out_res[a];
          rr += v * d.row_stride[a];
          cc += v * d.col_stride[a];
        }
        int64_t cnt[2 * kMaxDim] = {};
        for (int64_t s = 0; s < red_total && !bit; ++s) {
          if (d.row_any) {
            const uint64_t* row = d.in + rr * d.in_row_words;
            uint64_t acc = 0;
            for (int64_t k = 0; k < d.in_row_words && !acc; ++k) acc = row[k];
            bit = acc != 0;
          } else {
            bit = (d.in[rr * d.in_row_words + (cc >> 6)] >> (cc & 63)) & 1ull;
          }
          for (int q = d.nred - 1; q >= 0; --q) {
            rr += d.red_row_stride[q];
            cc += d.red_col_stride[q];
            if (++cnt[q] < d.red_res[q]) break;
            rr -= d.red_row_stride[q] * d.red_res[q];
            cc -= d.red_col_stride[q] * d.red_res[q];
            cnt[q] = 0;
          }
        }
      }
      half[h] = __ballot_sync(0xffffffffu, bit);
    }
    if (lane == 0) d.out[ow] = (uint64_t)half[0] | ((uint64_t)half[1] << 32);
  }
}

// Words mode: output word index -> input word index through the mixed-radix
// decomposition (u_res, u_in), then an OR over the reduced axes.  Index type I
// is 32-bit when every word index fits.
template <class I>
__global__ void reshape_words_kernel(const ReshapeDesc* __restrict__ descs,
                                     const int64_t* __restrict__ cta0, int n) {
  __shared__ ReshapeDesc sd;
  const RsCtx rc = rs_pick(descs, cta0, n, &sd);
  const ReshapeDesc& d = sd;
  const I total = (I)(d.out_nrows * d.out_row_words);
  I red_total = 1;
  for (int q = 0; q < d.nred; ++q) red_total *= (I)d.red_res[q];
  auto src_of = [&](I ow) -> I {
    I rest = ow, src = 0;
    for (int a = d.nu - 1; a >= 0; --a) {
      const I r = (I)d.u_res[a];
      const I q = rest / r;
      src += (rest - q * r) * (I)d.u_in[a];
      rest = q;
    }
    return src;
  };
  if (red_total == 1) {
    // a pure permutation of words: four loads in flight per thread
    const I stride = (I)rc.nblk * blockDim.x;
    I ow = (I)rc.bid * blockDim.x + threadIdx.x;
    for (; ow + 3 * stride < total; ow += 4 * stride) {
      uint64_t v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = d.in[src_of(ow + (I)k * stride)];
#pragma unroll
      for (int k = 0; k < 4; ++k) d.out[ow + (I)k * stride] = v[k];
    }
    for (; ow < total; ow += stride) d.out[ow] = d.in[src_of(ow)];
    return;
  }
  for (I ow = (I)rc.bid * blockDim.x + threadIdx.x; ow < total; ow += (I)rc.nblk * blockDim.x) {
    I rest = ow, src = 0;
    for (int a = d.nu - 1; a >= 0; --a) {
      const I r = (I)d.u_res[a];
      const I q = rest / r;
      src += (rest - q * r) * (I)d.u_in[a];
      rest = q;
    }
    uint64_t word = 0;
    I cnt[2 * kMaxDim] = {};
    for (I s = 0; s < red_total; ++s) {
      word |= d.in[src];
      for (int q = d.nred - 1; q >= 0; --q) {
        src += (I)d.red_in_w[q];
        if (++cnt[q] < (I)d.red_res[q]) break;
        src -= (I)d.red_in_w[q] * (I)d.red_res[q];
        cnt[q] = 0;
      }
    }
    d.out[ow] = word;
  }
}

// In-register transpose of a 64 x 64 bit block held by one warp: lane l holds
// rows l (lo) and l + 32 (hi), bit c of a row being column c.  Afterwards lane l
// holds columns l and l + 32 as rows.  Recursive block swap (halves, quarters,
// ... single bits): for block size s the rows r and r + s (r & s == 0) exchange
// the columns c + s of row r with the columns c of row r + s (c & s == 0).
__device__ __forceinline__ void transpose64(uint64_t& lo, uint64_t& hi, int lane) {
  uint64_t t = ((lo >> 32) ^ hi) & 0x00000000FFFFFFFFull;
  hi ^= t;
  lo ^= t << 32;
  const uint64_t masks[5] = {0x0000FFFF0000FFFFull, 0x00FF00FF00FF00FFull, 0x0F0F0F0F0F0F0F0Full,
                             0x3333333333333333ull, 0x5555555555555555ull};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int s = 16 >> i;
    const uint64_t m = masks[i];
    const uint64_t plo = __shfl_xor_sync(0xffffffffu, lo, s);
    const uint64_t phi = __shfl_xor_sync(0xffffffffu, hi, s);
    if (lane & s) {
      lo ^= ((plo >> s) ^ lo) & m;
      hi ^= ((phi >> s) ^ hi) & m;
    } else {
      lo ^= (((lo >> s) ^ plo) & m) << s;
      hi ^= (((hi >> s) ^ phi) & m) << s;
    }
  }
}

// Transpose mode.  A CTA tile is 256 values of L (4 output words) x 256 values
// of J (4 input words) at one value of the other axes: coalesced 32-byte loads
// of 256 input rows into shared memory, 16 warp transposes of 64 x 64 blocks,
// coalesced 32-byte stores of 256 output rows.  Rows of the shared tiles are
// padded to 5 words so the column reads of a block are free of bank conflicts.
constexpr int kTrPad = 5;
__global__ void __launch_bounds__(256)
reshape_transpose_kernel(const ReshapeDesc* __restrict__ descs, const int64_t* __restrict__ cta0, int n) {
  __shared__ ReshapeDesc sd;
  const RsCtx rc = rs_pick(descs, cta0, n, &sd);
  const ReshapeDesc& d = sd;
  __shared__ uint64_t s_in[256 * kTrPad];
  __shared__ uint64_t s_out[256 * kTrPad];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t nJT = (d.tQ + 255) / 256, nLT = (d.tR + 255) / 256;
  const int64_t tiles = d.n_other * nJT * nLT;
  // tile -> (L tile, J tile, first input and output word of its other axes)
  auto locate = [&](int64_t tile, int64_t& lt, int64_t& jt, int64_t& base_in, int64_t& base_out) {
    lt = tile % nLT;
    const int64_t r = tile / nLT;
    jt = r % nJT;
    int64_t rest = r / nJT;
    base_in = 0;
    base_out = 0;
    for (int a = d.nu - 1; a >= 0; --a) {
      const int64_t v = rest % d.u_res[a];
      rest /= d.u_res[a];
      base_in += v * d.u_in[a];
      base_out += v * d.u_out[a];
    }
  };
  // the four input words this thread loads for a tile
  auto load = [&](int64_t lt, int64_t jt, int64_t base_in, uint64_t* v) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int idx = tid + 256 * i, b = idx >> 2, c = idx & 3;
      const int64_t L = lt * 256 + b, jb = jt * 4 + c;
      v[i] = (L < d.tR && jb * 64 < d.tQ) ? d.in[base_in + L * d.t_in_L + jb] : 0ull;
    }
  };
  // the next tile's loads are issued before the current tile is transposed
  // and stored, so that their latency overlaps that work
  int64_t lt = 0, jt = 0, base_in = 0, base_out = 0;
  uint64_t nv[4] = {0, 0, 0, 0};
  if (rc.bid < tiles) {
    locate(rc.bid, lt, jt, base_in, base_out);
    load(lt, jt, base_in, nv);
  }
  for (int64_t tile = rc.bid; tile < tiles; tile += rc.nblk) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int idx = tid + 256 * i, b = idx >> 2, c = idx & 3;
      s_in[b * kTrPad + c] = nv[i];
    }
    const int64_t clt = lt, cjt = jt, cbase_out = base_out;
    if (tile + rc.nblk < tiles) {
      locate(tile + rc.nblk, lt, jt, base_in, base_out);
      load(lt, jt, base_in, nv);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int k = warp * 2 + i, cw = k >> 2, lw = k & 3;
      if ((cjt * 4 + cw) * 64 < d.tQ && clt * 256 + lw * 64 < d.tR) {
        uint64_t lo = s_in[(lw * 64 + lane) * kTrPad + cw];
        uint64_t hi = s_in[(lw * 64 + lane + 32) * kTrPad + cw];
        transpose64(lo, hi, lane);
        s_out[(cw * 64 + lane) * kTrPad + lw] = lo;
        s_out[(cw * 64 + lane + 32) * kTrPad + lw] = hi;
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int idx = tid + 256 * i, t = idx >> 2, w = idx & 3;
      const int64_t J = cjt * 256 + t, lw = clt * 4 + w;
      if (J < d.tQ && lw * 64 < d.tR) d.out[cbase_out + J * d.t_out_J + lw] = s_out[t * kTrPad + w];
    }
    __syncthreads();
  }
}

int reshape_kind(const ReshapeDesc& d) {
  if (d.mode == kReshapeTranspose) return kRsTranspose;
  if (d.mode == kReshapeWords) {
    const int64_t total = d.out_nrows * d.out_row_words;
    const int64_t blocks = reshape_blocks(d);
    int64_t in_max = 0;  // largest input word index + 1 (bounded by the sum below)
    for (int a = 0; a < d.nu; ++a) in_max += (d.u_res[a] - 1) * d.u_in[a];
    for (int q = 0; q < d.nred; ++q) in_max += (d.red_res[q] - 1) * d.red_in_w[q];
    return (total + 256 * blocks < (1ll << 31) && in_max < (1ll << 31)) ? kRsWords32 : kRsWords64;
  }
  return kRsBits;
}

int64_t reshape_blocks(const ReshapeDesc& d) {
  const int64_t total = d.out_nrows * d.out_row_words;
  if (total <= 0) return 0;
  if (d.mode == kReshapeTranspose)
    return std::min<int64_t>(d.n_other * ((d.tQ + 255) / 256) * ((d.tR + 255) / 256), 152 * 8);
  if (d.mode == kReshapeWords) return std::min<int64_t>((total + 255) / 256, 152 * 16);
  return std::min<int64_t>((total + 7) / 8, 152 * 16);  // one warp per word
}

void launch_reshape(const ReshapeDesc* d_descs, const int64_t* d_cta0, int n, int kind,
                    int64_t grid, cudaStream_t s) {
  if (n <= 0 || grid <= 0) return;
  switch (kind) {
    case kRsTranspose:
      reshape_transpose_kernel<<<(unsigned)grid, 256, 0, s>>>(d_descs, d_cta0, n);
      break;
    case kRsWords32:
      reshape_words_kernel<uint32_t><<<(unsigned)grid, 256, 0, s>>>(d_descs, d_cta0, n);
      break;
    case kRsWords64:
      reshape_words_kernel<uint64_t><<<(unsigned)grid, 256, 0, s>>>(d_descs, d_cta0, n);
      break;
    default:
      reshape_kernel<<<(unsigned)grid, 256, 0, s>>>(d_descs, d_cta0, n);
      break;
  }
}

// Long dot rows (more than 16 words) are split into runs of this many words.
constexpr int64_t kDotRun = 256;

// ------------------------------------------- outer / dot / and, batched
// Every such cluster of one tree level in one launch: job p owns blocks
// [cta0[p], cta0[p+1]) and runs the loop of its kind over them.
__global__ void __launch_bounds__(256)
ewise_kernel(const EwJob* __restrict__ jobs, const int64_t* __restrict__ cta0, int n) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cta0[mid] <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const EwJob& j = jobs[lo];
  const int64_t bid = (int64_t)blockIdx.x - cta0[lo], nblk = cta0[lo + 1] - cta0[lo];
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = bid * (blockDim.x >> 5) + (threadIdx.x >> 5), nwarps = nblk * (blockDim.x >> 5);
  const uint64_t* __restrict__ A = j.a;
  const uint64_t* __restrict__ B = j.b;
  uint64_t* __restrict__ C = j.c;
  if (j.kind == kEwAnd) {
    for (int64_t i = bid * blockDim.x + threadIdx.x; i < j.rows; i += nblk * blockDim.x) C[i] = A[i] & B[i];
  } else if (j.kind == kEwOuter) {
    // C[r][w] = bit r of A ? B[r / M][w] : 0
    const int64_t total = j.rows * j.nw;
    for (int64_t i = bid * blockDim.x + threadIdx.x; i < total; i += nblk * blockDim.x) {
      const int64_t r = i / j.nw, w = i - r * j.nw;
      const uint64_t bit = (A[r >> 6] >> (r & 63)) & 1ull;
      C[i] = bit ? B[(r / j.m) * j.nw + w] : 0ull;
    }
  } else if (j.kind == kEwDot) {
    // one warp per word of C: lanes take bits r and r + 32
    const int64_t words = (j.rows + 63) / 64;
    for (int64_t cw = gwarp; cw < words; cw += nwarps) {
      uint32_t half[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t r = cw * 64 + h * 32 + lane;
        uint64_t acc = 0;
        if (r < j.rows) {
          const uint64_t* a = A + r * j.nw;
          const uint64_t* b = B + (r / j.m) * j.nw;
          for (int64_t w = 0; w < j.nw && !acc; ++w) acc = a[w] & b[w];
        }
        half[h] = __ballot_sync(0xffffffffu, acc != 0);
      }
      if (lane == 0) C[cw] = (uint64_t)half[0] | ((uint64_t)half[1] << 32);
    }
  } else {
    // long rows: one warp per (row, run of 256 words) into the cleared C
    const int64_t nruns = (j.nw + kDotRun - 1) / kDotRun;
    const int64_t items = j.rows * nruns;
    for (int64_t it = gwarp; it < items; it += nwarps) {
      const int64_t r = it / nruns, w0 = (it - r * nruns) * kDotRun;
      const int64_t w1 = min(j.nw, w0 + kDotRun);
      const uint64_t* a = A + r * j.nw;
      const uint64_t* b = B + (r / j.m) * j.nw;
      uint64_t acc = 0;
      for (int64_t w = w0 + lane; w < w1; w += 32) acc |= a[w] & b[w];
      if (__any_sync(0xffffffffu, acc != 0) && lane == 0)
        atomicOr(reinterpret_cast<unsigned long long*>(&C[r >> 6]), 1ull << (r & 63));
    }
  }
}

int64_t ewise_blocks(const EwJob& j) {
  int64_t items;
  switch (j.kind) {
    case kEwAnd: items = (j.rows + 255) / 256; break;
    case kEwOuter: items = (j.rows * j.nw + 255) / 256; break;
    case kEwDot: items = ((j.rows + 63) / 64 + 7) / 8; break;
    default: items = (j.rows * ((j.nw + kDotRun - 1) / kDotRun) + 7) / 8; break;
  }
  return std::min<int64_t>(items, 152 * 16);
}

void launch_ewise(const EwJob* d_jobs, const int64_t* d_cta0, int n, int64_t grid, cudaStream_t s) {
  if (n <= 0 || grid <= 0) return;
  ewise_kernel<<<(unsigned)grid, 256, 0, s>>>(d_jobs, d_cta0, n);
}

// ---------------------------------------------------------------- row-OR
// One CTA owns the tile B[b][k0 .. k0+Kc)[n0 .. n0+Nt) in shared memory, staged
// by the Tensor Memory Accelerator (2-D boxes of 256 rows x Nt words) when the
// row pitch allows it, else by plain loads.  Next to it the CTA builds the ORs
// of aligned blocks of 4, 16 and 64 tile rows (tables T2, T4, T6; T0 is the
// tile itself), plus an all-zero sentinel row.  A run of set bits in a row of
// A selects a run of B rows, whose OR is the OR of the maximal aligned blocks
// covering it: the plotted relations are thick curves, so most set bits lie in
// long runs and a row needs a few block lookups instead of one per bit.
// Each warp then takes one output row at a time:
//   1. its lanes load up to 32 words of the row's A bits for this K range and
//      split each word into maximal all-ones aligned blocks of 64, 16, 4 and 1
//      bits (a few bit operations), counting them;
//   2. every lane writes the table rows of its blocks into the warp's list in
//      shared memory (256 entries: slots taken from a warp counter; a row
//      with more blocks goes through the list in ordered windows);
//   3. the warp splits into 32/Nt groups of Nt lanes; group g ORs table rows
//      list[g], list[g + 32/Nt], ... (four loads in flight per lane), lane l of
//      a group holding word n0 + l;
//   4. the groups' words are OR-ed together with shuffles and stored.
namespace {

constexpr int kRowOrThreads = 1024;
// Entries of a warp's list per window, plus sentinel padding.  A unit whose
// blocks do not fit is processed in several windows.
constexpr int kListWin = 256;
constexpr int kListCap = kListWin + 128;

// Tile rows of the tables for a K range staged in `staged` rows: T0 (rounded
// up to whole 64-row groups), the sentinel, T2, T4 and T6.
__host__ __device__ __forceinline__ int64_t rowor_r64(int64_t staged) { return (staged + 63) / 64 * 64; }
__host__ __device__ __forceinline__ int64_t rowor_table_rows(int64_t staged) {
  const int64_t r64 = rowor_r64(staged);
  return r64 + 1 + r64 / 4 + r64 / 16 + r64 / 64;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Wait for phase `parity` of an mbarrier, giving up after about `limit_ns`.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit_ns) {
  const long long t0 = clock64();
  const long long limit_cycles = limit_ns * 2;  // >= 1 cycle per ns at <= 2.1 GHz
  for (long long it = 0; it < (1ll << 26); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit_cycles) return false;
  }
  return false;
}

// Launch description: problem p owns CTAs [cta0[p], cta0[p+1]); its
// descriptor and tensor map (used when d.use_tma) live in global memory.
template <int G>
__global__ void __launch_bounds__(kRowOrThreads)
rowor_tile_kernel(const RowOrDesc* __restrict__ descs, const CUtensorMap* __restrict__ maps,
                  const int64_t* __restrict__ cta0s, int nprob) {
  extern __shared__ __align__(1024) uint64_t bs[];
  __shared__ RowOrDesc sd;
  __shared__ int s_p;
  // the next launch may be scheduled onto SMs this grid frees; it waits for
  // this grid's completion before it touches any data
  asm volatile("griddepcontrol.launch_dependents;");
  const int tid = threadIdx.x;
  const int nwarps = blockDim.x >> 5;
  if (tid == 0) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cta0s[mid] <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    s_p = lo;
    sd = descs[lo];
  }
  __syncthreads();
  const int p = s_p;
  const RowOrDesc& d = sd;
  const CUtensorMap* tmap = maps + p;
  const int64_t staged = d.use_tma ? ((int64_t)d.Kc + 255) / 256 * 256 : d.Kc;
  const int r64 = (int)rowor_r64(staged);
  const int sent = r64, t2 = r64 + 1, t4 = t2 + r64 / 4, t6 = t4 + r64 / 16;
  uint16_t* lists = reinterpret_cast<uint16_t*>(bs + rowor_table_rows(staged) * G);
  uint64_t* bar = reinterpret_cast<uint64_t*>(lists + (size_t)nwarps * kListCap);

  int64_t cta = (int64_t)blockIdx.x - cta0s[p];
  const int64_t rs = cta % d.row_splits;
  cta /= d.row_splits;
  const int64_t kc = cta % d.k_chunks;
  cta /= d.k_chunks;
  const int64_t nt = cta % d.n_tiles;
  const int64_t b = cta / d.n_tiles;
  const int64_t k0 = kc * d.Kc;
  const int kc_len = (int)min((int64_t)d.Kc, d.K - k0);
  const int64_t n0 = nt * G;

  // ---- stage the B tile
  if (d.use_tma) {
    const int nbox = (kc_len + 255) / 256;
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      // the tensor map was written to global memory by a copy before the launch
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
    }
    // everything the earlier kernels of the stream wrote (A, B) is complete
    // and visible past this point, and C may be overwritten
    asm volatile("griddepcontrol.wait;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)nbox * 256u * (uint32_t)G * 8u;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                   "r"(bytes)
                   : "memory");
      for (int j = 0; j < nbox; ++j) {
        const int x = (int)n0;
        const int y = (int)(b * d.K + k0 + 256 * j);
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(bs + (size_t)j * 256 * G)),
            "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
            : "memory");
      }
    }
    const bool ok = mbar_wait(bar, 0, 1000000000ll);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(d.err, 1);
      return;
    }
  } else {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // rows past the K range are zero (only block tables that no lookup reads
    // include them)
    for (int idx = tid; idx < r64 * G; idx += blockDim.x) {
      const int r = idx / G, c = idx % G;
      const int64_t n = n0 + c;
      bs[idx] = (r < kc_len && n < d.Nw) ? __ldg(d.B + (b * d.K + k0 + r) * d.Nw + n) : 0ull;
    }
  }
  if (tid < G) bs[(size_t)sent * G + tid] = 0ull;  // sentinel row
  __syncthreads();
  // block tables: each row the OR of four rows of the level below
  {
    const int lv_src[3] = {0, t2, t4}, lv_dst[3] = {t2, t4, t6}, lv_n[3] = {r64 / 4, r64 / 16, r64 / 64};
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      const uint64_t* src = bs + (size_t)lv_src[l] * G;
      uint64_t* dst = bs + (size_t)lv_dst[l] * G;
      for (int idx = tid; idx < lv_n[l] * G; idx += blockDim.x) {
        const int q = idx / G, c = idx - (idx / G) * G;
        const uint64_t* s0 = src + (size_t)(4 * q) * G + c;
        dst[idx] = s0[0] | s0[G] | s0[2 * G] | s0[3 * G];
      }
      __syncthreads();
    }
  }

  // ---- output rows, one warp each
  const int warp = tid >> 5, lane = tid & 31;
  const int grp = lane / G, lig = lane % G;
  constexpr int P = 32 / G;
  uint16_t* list = lists + (size_t)warp * kListCap;
  // rows are dealt out cyclically over every warp of the CTAs sharing this
  // tile, so that runs of dense rows (curves are locally thick) are spread out.
  // A warp's work is a sequence of units (row, batch of 32 A words); the A
  // words of the next four units are always in flight while one is processed.
  const int gw = (int)rs * nwarps + warp;
  const int gstride = (int)d.row_splits * nwarps;
  const int kw0 = (int)(k0 / 64);
  const int kw1 = (int)min(d.a_row_words, (k0 + kc_len + 63) / 64);
  const int nbat = (kw1 - kw0 + 31) / 32;
  const int M = (int)d.M;
  const int nrows_w = (gw < M) ? (M - gw + gstride - 1) / gstride : 0;
  const int nunits = nrows_w * nbat;
  const uint64_t* __restrict__ abase = d.A + (b * d.M) * d.a_row_words;
  const int64_t arw = d.a_row_words;
  int* wcount = reinterpret_cast<int*>(bar + 1) + warp;
  if (lane == 0) *wcount = 0;
  int wbase = 0;
  __syncwarp();
  auto load_unit = [&](int u) -> uint64_t {
    if (u >= nunits) return 0ull;
    const int i = (nbat == 1) ? u : u / nbat;
    const int q = u - i * nbat;
    const int kwl = kw0 + q * 32 + lane;
    return (kwl < kw1) ? __ldg(abase + (int64_t)(gw + i * gstride) * arw + kwl) : 0ull;
  };
  uint64_t pre0 = load_unit(0), pre1 = load_unit(1), pre2 = load_unit(2), pre3 = load_unit(3);
  uint64_t acc = 0;
  for (int u = 0; u < nunits; ++u) {
    uint64_t a = pre0;
    pre0 = pre1;
    pre1 = pre2;
    pre2 = pre3;
    pre3 = load_unit(u + 4);
    const int i = (nbat == 1) ? u : u / nbat;
    const int q = u - i * nbat;
    if (q == 0) acc = 0;
    if (__any_sync(0xffffffffu, a != 0ull)) {
      // tile row of this word's bit 0 (a multiple of 64); bits past the K
      // range are dropped
      const int base = (kw0 + q * 32 + lane) * 64 - (int)k0;
      if (base + 64 > kc_len) a &= (base >= kc_len) ? 0ull : ((1ull << (kc_len - base)) - 1ull);
      // maximal all-ones aligned blocks of the word: bit 4i of f4 when bits
      // 4i..4i+3 are set, bit 16i of f16 when bits 16i..16i+15 are set, f1 the
      // set bits in neither; a full word is one 64-block
      const bool full = (a == ~0ull);
      uint64_t f16 = 0, f4 = 0, f1 = a;
      if (!full) {
        uint64_t t = a & (a >> 1);
        t &= t >> 2;
        f4 = t & 0x1111111111111111ull;
        uint64_t u4 = f4 & (f4 >> 4);
        u4 &= u4 >> 8;
        f16 = u4 & 0x0001000100010001ull;
        const uint64_t m16 = f16 * 0xFFFFull;
        f4 &= ~m16;
        f1 = a & ~(m16 | f4 * 0xFull);
      }
      const int c = full ? 1 : __popcll(f16) + __popcll(f4) + __popcll(f1);
      const int T = (int)__reduce_add_sync(0xffffffffu, (unsigned)c);
      if (d.stat && lane == 0) atomicAdd(d.stat, (unsigned long long)T * G);
      if (T <= kListWin) {
        // one window: each lane claims its slots from the warp's counter,
        // which only grows (this unit's slots start at the units' running
        // total, known to every lane), so it never needs resetting
        int e = c ? atomicAdd(wcount, c) - wbase : 0;
        if (full) {
          list[e] = (uint16_t)(t6 + base / 64);
        } else {
          for (uint64_t m = f16; m; m &= m - 1) list[e++] = (uint16_t)(t4 + (base + __ffsll((long long)m) - 1) / 16);
          for (uint64_t m = f4; m; m &= m - 1) list[e++] = (uint16_t)(t2 + (base + __ffsll((long long)m) - 1) / 4);
          for (uint64_t m = f1; m; m &= m - 1) list[e++] = (uint16_t)(base + __ffsll((long long)m) - 1);
        }
        wbase += T;
        // pad to a whole number of rounds with the sentinel row (4P entries,
        // which is more than one per lane when the groups are narrow)
        for (int t = lane; t < 4 * P; t += 32) list[T + t] = (uint16_t)sent;
        __syncwarp();
        for (int e2 = grp; e2 < T; e2 += 4 * P) {
          const int i0 = list[e2], i1 = list[e2 + P], i2 = list[e2 + 2 * P], i3 = list[e2 + 3 * P];
          acc |= bs[i0 * G + lig] | bs[i1 * G + lig] | bs[i2 * G + lig] | bs[i3 * G + lig];
        }
        __syncwarp();
      } else {
        // several windows: this lane's entries are [o, o + c) of the unit's
        // T in a fixed order, and each window writes the ones inside it
        int o = c;
#pragma unroll
        for (int sh = 1; sh < 32; sh <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, o, sh);
          if (lane >= sh) o += v;
        }
        o -= c;
        for (int w0 = 0; w0 < T; w0 += kListWin) {
          const int w1 = min(T, w0 + kListWin);
          if (o < w1 && o + c > w0) {
            int e = o;
            auto put = [&](int row) {
              if (e >= w0 && e < w1) list[e - w0] = (uint16_t)row;
              ++e;
            };
            if (full) {
              put(t6 + base / 64);
            } else {
              for (uint64_t m = f16; m; m &= m - 1) put(t4 + (base + __ffsll((long long)m) - 1) / 16);
              for (uint64_t m = f4; m; m &= m - 1) put(t2 + (base + __ffsll((long long)m) - 1) / 4);
              for (uint64_t m = f1; m; m &= m - 1) put(base + __ffsll((long long)m) - 1);
            }
          }
          const int n = w1 - w0;
          for (int t = lane; t < 4 * P; t += 32) list[n + t] = (uint16_t)sent;
          __syncwarp();
          for (int e2 = grp; e2 < n; e2 += 4 * P) {
            const int i0 = list[e2], i1 = list[e2 + P], i2 = list[e2 + 2 * P], i3 = list[e2 + 3 * P];
            acc |= bs[i0 * G + lig] | bs[i1 * G + lig] | bs[i2 * G + lig] | bs[i3 * G + lig];
          }
          __syncwarp();
        }
      }
    }
    if (q == nbat - 1) {
      uint64_t r = acc;
#pragma unroll
      for (int o = G; o < 32; o <<= 1) r |= __shfl_xor_sync(0xffffffffu, r, o);
      const int m = gw + i * gstride;
      const int64_t n = n0 + lane;
      if (lane < G && n < d.Nw) {
        uint64_t* c = d.C + (b * d.M + m) * d.Nw + n;
        if (d.atomic) {
          if (r) atomicOr((unsigned long long*)c, (unsigned long long)r);
        } else {
          *c = r;
        }
      }
    }
  }
}

}  // namespace

namespace {

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// Shared memory of one CTA: the tables plus the warps' lists, their counters
// and the mbarrier, within the 227 KB a CTA may opt into.
constexpr size_t kSmemLimit = 227 * 1024 - 2048;  // the kernel's static shared memory stays out
constexpr size_t kListBytes = (size_t)(kRowOrThreads / 32) * kListCap * 2 + 16 +
                              (size_t)(kRowOrThreads / 32) * 4;

size_t table_bytes(int64_t staged, int Nt) { return (size_t)rowor_table_rows(staged) * Nt * 8; }

}  // namespace

EncodeTiledFn tensor_map_encoder() { return encode_fn(); }

cudaError_t smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> set;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = set[{fn, dev}];
  if (bytes <= have) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

void rowor_plan(RowOrDesc& d, int64_t target_ctas) {
  const bool tma_ok = (d.Nw % 2 == 0) && (reinterpret_cast<uintptr_t>(d.B) % 16 == 0) &&
                      (d.nbatch * d.K < (1ll << 31)) && encode_fn() != nullptr;
  auto staged_of = [&](int64_t kc, bool tma) { return tma ? (kc + 255) / 256 * 256 : kc; };
  // the widest power-of-two tile (<= 32 words, <= the row): a row of A is
  // split into blocks and listed once per tile, so wide tiles cut that work
  // (32-word tiles took the chain's 2048^3 joins from 19.3 to 16.0 us per
  // launch against 8-word tiles over the whole K range).  When the whole K
  // range does not fit next to it, K is split into chunks whose results are
  // OR-ed into C (cleared beforehand).
  int Nt = 1;
  while (Nt < 32 && Nt < d.Nw) Nt <<= 1;
  d.Nt = Nt;
  d.use_tma = (tma_ok && Nt % 2 == 0) ? 1 : 0;
  const int64_t step = d.use_tma ? 256 : 64;
  if (table_bytes(staged_of(d.K, d.use_tma), Nt) + kListBytes <= kSmemLimit) {
    d.Kc = (int32_t)d.K;
  } else {
    int64_t kc = step;
    while (table_bytes(kc + step, Nt) + kListBytes <= kSmemLimit) kc += step;
    d.Kc = (int32_t)kc;
  }
  d.n_tiles = (d.Nw + Nt - 1) / Nt;
  d.k_chunks = (d.K + d.Kc - 1) / d.Kc;
  d.atomic = d.k_chunks > 1 ? 1 : 0;
  const int64_t base = d.nbatch * d.n_tiles * d.k_chunks;
  const int64_t target = std::max<int64_t>(1, target_ctas);
  // round down: a launch of more CTAs than SMs (one CTA fits an SM) would run
  // a short second wave and nearly double its time
  int64_t splits = target / base;
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, (d.M + 15) / 16));
  d.rows_per_split = (d.M + splits - 1) / splits;
  d.row_splits = (d.M + d.rows_per_split - 1) / d.rows_per_split;
}

size_t rowor_smem_bytes(const RowOrDesc& d) {
  const int64_t staged = d.use_tma ? ((int64_t)d.Kc + 255) / 256 * 256 : d.Kc;
  return table_bytes(staged, d.Nt) + kListBytes;
}

int64_t rowor_ctas(const RowOrDesc& d) { return d.nbatch * d.n_tiles * d.k_chunks * d.row_splits; }

cudaError_t rowor_encode_map(const RowOrDesc& d, CUtensorMap* map) {
  memset(map, 0, sizeof *map);
  if (!d.use_tma) return cudaSuccess;
  const cuuint64_t dims[2] = {(cuuint64_t)d.Nw, (cuuint64_t)(d.nbatch * d.K)};
  const cuuint64_t strides[1] = {(cuuint64_t)d.Nw * 8};
  const cuuint32_t box[2] = {(cuuint32_t)d.Nt, 256u};
  const cuuint32_t estr[2] = {1u, 1u};
  CUresult r = encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t*>(d.B), dims,
                           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Failure-path check of the bounded waits: one thread waits on an mbarrier
// that nothing arrives at, gives up after limit_ns as every wait of the
// contraction kernels does, and sets the error word.
__global__ void wait_selftest_kernel(int* err, long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (!mbar_wait(&bar, 0, limit_ns)) atomicExch(err, 1);
}

cudaError_t launch_wait_selftest(int* err, long long limit_ns, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(err, limit_ns);
  return cudaGetLastError();
}

cudaError_t launch_rowor(const RowOrDesc* d_descs, const CUtensorMap* d_maps,
                         const int64_t* d_cta0, int nprob, int64_t grid, size_t smem, int Nt,
                         cudaStream_t s) {
  if (nprob <= 0 || grid <= 0) return cudaSuccess;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  // programmatic dependent launch: CTAs may start on SMs the previous kernel
  // has left and set up while it finishes (the kernel waits before any data)
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kRowOrThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
#define PA_ROWOR(GG)                                                                         \
  do {                                                                                       \
    smem_limit(reinterpret_cast<const void*>(rowor_tile_kernel<GG>), smem);                  \
    cudaLaunchKernelEx(&cfg, rowor_tile_kernel<GG>, d_descs, d_maps, d_cta0, nprob);         \
  } while (0)
  switch (Nt) {
    case 1: PA_ROWOR(1); break;
    case 2: PA_ROWOR(2); break;
    case 4: PA_ROWOR(4); break;
    case 8: PA_ROWOR(8); break;
    case 16: PA_ROWOR(16); break;
    default: PA_ROWOR(32); break;
  }
#undef PA_ROWOR
  return cudaGetLastError();
}

// -------------------------------------------------------------- popcount
__global__ void popcount_kernel(const uint64_t* __restrict__ w, int64_t n,
                                unsigned long long* __restrict__ out) {
  unsigned long long c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c += (unsigned long long)__popcll(w[i]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

void launch_popcount(const uint64_t* w, int64_t nwords, unsigned long long* out, cudaStream_t s) {
  if (nwords <= 0) return;
  int64_t blocks = (nwords + 255) / 256;
  if (blocks > 152 * 4) blocks = 152 * 4;
  popcount_kernel<<<(unsigned)blocks, 256, 0, s>>>(w, nwords, out);
}


}  // namespace pa
