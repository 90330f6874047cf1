// Contraction kernels: Eq. (GAM) of Sec. 3.3 for one two-array cluster (Sec. 3.5)
// over the Boolean semiring, on bit-packed arrays.
//
// After the planner has brought both operands into matrix form
//   A[b][m][k]  (k packed along rows)   and   B[b][k][n]  (n packed along rows),
// the cluster is C[b][m][n] = OR_k A[b][m][k] AND B[b][k][n], computed row-wise:
// row (b, m) of C is the OR of the rows B[b][k][:] selected by the set bits of
// row (b, m) of A.  Curve plots are sparse, so the work is proportional to the
// number of set bits of A times the packed width of B, not to M*K*N.
#include "pa_internal.h"

namespace pa {

// --------------------------------------------------------------- reshape
__global__ void reshape_kernel(const ReshapeDesc d) {
  const int64_t total = d.out_nrows * d.out_row_words;
  const int outer = d.out_ndim - d.out_inner;
  int64_t red_total = 1;
  for (int q = 0; q < d.nred; ++q) red_total *= d.red_res[q];
  for (int64_t ow = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; ow < total;
       ow += (int64_t)gridDim.x * blockDim.x) {
    const int64_t orow = ow / d.out_row_words, w = ow % d.out_row_words;
    int64_t brow = 0, bcol = 0, rest = orow;
    for (int a = outer - 1; a >= 0; --a) {
      const int64_t v = rest % d.out_res[a];
      rest /= d.out_res[a];
      brow += v * d.row_stride[a];
      bcol += v * d.col_stride[a];
    }
    uint64_t word = 0;
    if (d.word_mode) {
      // columns map 1:1: OR whole input words over the reduced axes
      int64_t cnt[2 * kMaxDim] = {};
      int64_t rr = brow;
      for (int64_t s = 0; s < red_total; ++s) {
        word |= d.in[rr * d.in_row_words + w];
        for (int q = d.nred - 1; q >= 0; --q) {
          rr += d.red_row_stride[q];
          if (++cnt[q] < d.red_res[q]) break;
          rr -= d.red_row_stride[q] * d.red_res[q];
          cnt[q] = 0;
        }
      }
    } else {
      for (int b = 0; b < 64; ++b) {
        const int64_t ocol = w * 64 + b;
        if (ocol >= d.out_rowlen) break;
        int64_t rr = brow, cc = bcol, rest2 = ocol;
        for (int a = d.out_ndim - 1; a >= outer; --a) {
          const int64_t v = rest2 % d.out_res[a];
          rest2 /= d.out_res[a];
          rr += v * d.row_stride[a];
          cc += v * d.col_stride[a];
        }
        int64_t cnt[2 * kMaxDim] = {};
        uint64_t bit = 0;
        for (int64_t s = 0; s < red_total && !bit; ++s) {
          bit = (d.in[rr * d.in_row_words + (cc >> 6)] >> (cc & 63)) & 1ull;
          for (int q = d.nred - 1; q >= 0; --q) {
            rr += d.red_row_stride[q];
            cc += d.red_col_stride[q];
            if (++cnt[q] < d.red_res[q]) break;
            rr -= d.red_row_stride[q] * d.red_res[q];
            cc -= d.red_col_stride[q] * d.red_res[q];
            cnt[q] = 0;
          }
        }
        word |= bit << b;
      }
    }
    d.out[ow] = word;
  }
}

void launch_reshape(const ReshapeDesc& d, cudaStream_t s) {
  const int64_t total = d.out_nrows * d.out_row_words;
  if (total <= 0) return;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  reshape_kernel<<<(unsigned)blocks, 256, 0, s>>>(d);
}

// ---------------------------------------------------------------- row-OR
// Lanes form groups of G (a power of two <= 32).  A group owns one task
// (output row, k-chunk, n-chunk); lane l of the group accumulates the words
// n = n0 + l + G*j, j < NJ, of that row.  The A words of the task are read by
// the group together and their set bits walked with ffs.
template <int G, int NJ>
__global__ void __launch_bounds__(256) rowor_kernel(const RowOrDesc d) {
  const int lane = threadIdx.x & 31;
  const int grp = lane / G, lig = lane % G;
  constexpr int kGroups = 32 / G;
  const int64_t nrows = d.nbatch * d.M;
  const int64_t ntasks = nrows * d.nkchunks * d.nnchunks;
  const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // lanes of one group run in lockstep (same task, same loop bounds), so the
  // group's own mask suffices for its shuffles
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
  for (int64_t t = warp_global * kGroups + grp; t < ntasks; t += nwarps * kGroups) {
    const int64_t nc = t % d.nnchunks;
    const int64_t t2 = t / d.nnchunks;
    const int64_t kc = t2 % d.nkchunks;
    const int64_t row = t2 / d.nkchunks;
    const int64_t b = row / d.M;
    const uint64_t* __restrict__ arow = d.A + row * d.a_row_words;
    const uint64_t* __restrict__ bmat = d.B + b * d.K * d.Nw;
    const int64_t n0 = nc * (int64_t)(G * NJ);
    uint64_t acc[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = 0;
    const int64_t kw0 = kc * d.kchunk_words;
    const int64_t kw1 = min(kw0 + d.kchunk_words, d.a_row_words);
    for (int64_t kb = kw0; kb < kw1; kb += G) {
      // the group loads up to G words of A at once, then walks them in turn
      const int64_t myk = kb + lig;
      const uint64_t mw = (myk < kw1) ? __ldg(arow + myk) : 0ull;
      const int cnt = (int)min((int64_t)G, kw1 - kb);
      for (int q = 0; q < cnt; ++q) {
        uint64_t aw = __shfl_sync(gmask, mw, grp * G + q);
        while (aw) {
          const int bit = __ffsll((long long)aw) - 1;
          aw &= aw - 1;
          const int64_t k = (kb + q) * 64 + bit;
          if (k >= d.K) break;  // padding bits of a caller's array are ignored
          const uint64_t* __restrict__ brow = bmat + k * d.Nw;
#pragma unroll
          for (int j = 0; j < NJ; ++j) {
            const int64_t n = n0 + lig + (int64_t)G * j;
            if (n < d.Nw) acc[j] |= __ldg(brow + n);
          }
        }
      }
    }
    uint64_t* crow = d.C + row * d.Nw;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
      const int64_t n = n0 + lig + (int64_t)G * j;
      if (n < d.Nw) {
        if (d.atomic) {
          if (acc[j]) atomicOr((unsigned long long*)(crow + n), (unsigned long long)acc[j]);
        } else {
          crow[n] = acc[j];
        }
      }
    }
  }
}

void launch_rowor(const RowOrDesc& d, cudaStream_t s) {
  const int64_t nrows = d.nbatch * d.M;
  if (nrows <= 0 || d.Nw <= 0) return;
  int G = 1;
  while (G < 32 && G < d.Nw) G <<= 1;
  int NJ = 1;
  if (d.Nw > 32) NJ = (d.Nw >= 256) ? 8 : (d.Nw >= 128 ? 4 : (d.Nw >= 64 ? 2 : 1));
  const int64_t groups = nrows * d.nkchunks * d.nnchunks;
  const int64_t warps = (groups + (32 / G) - 1) / (32 / G);
  int64_t blocks = (warps + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  const unsigned gb = (unsigned)blocks;
#define PA_ROWOR(GG, NN) rowor_kernel<GG, NN><<<gb, 256, 0, s>>>(d)
  switch (G) {
    case 1: PA_ROWOR(1, 1); break;
    case 2: PA_ROWOR(2, 1); break;
    case 4: PA_ROWOR(4, 1); break;
    case 8: PA_ROWOR(8, 1); break;
    case 16: PA_ROWOR(16, 1); break;
    default:
      switch (NJ) {
        case 1: PA_ROWOR(32, 1); break;
        case 2: PA_ROWOR(32, 2); break;
        case 4: PA_ROWOR(32, 4); break;
        default: PA_ROWOR(32, 8); break;
      }
  }
#undef PA_ROWOR
}

// Number of words of one output row handled by one task for this shape.
int64_t rowor_chunk_words(int64_t Nw) {
  int G = 1;
  while (G < 32 && G < Nw) G <<= 1;
  int NJ = 1;
  if (Nw > 32) NJ = (Nw >= 256) ? 8 : (Nw >= 128 ? 4 : (Nw >= 64 ? 2 : 1));
  return (int64_t)G * NJ;
}

// ------------------------------------------------------------------- AND
__global__ void and_kernel(const uint64_t* __restrict__ a, const uint64_t* __restrict__ b,
                           uint64_t* __restrict__ c, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    c[i] = a[i] & b[i];
}

void launch_and(const uint64_t* a, const uint64_t* b, uint64_t* c, int64_t nwords,
                cudaStream_t s) {
  if (nwords <= 0) return;
  int64_t blocks = (nwords + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  and_kernel<<<(unsigned)blocks, 256, 0, s>>>(a, b, c, nwords);
}

}  // namespace pa
