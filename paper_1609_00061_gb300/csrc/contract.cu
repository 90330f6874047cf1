// Contraction kernels: Eq. (GAM) of Sec. 3.3 for one two-array cluster (Sec. 3.5)
// over the Boolean semiring, on bit-packed arrays.
//
// After the planner has brought both operands into matrix form
//   A[b][m][k]  (k packed along rows)   and   B[b][k][n]  (n packed along rows),
// the cluster is C[b][m][n] = OR_k A[b][m][k] AND B[b][k][n], computed row-wise:
// row (b, m) of C is the OR of the rows B[b][k][:] selected by the set bits of
// row (b, m) of A.  Curve plots are sparse, so the work is proportional to the
// number of set bits of A times the packed width of B, not to M*K*N.
#include <cuda.h>
#include <string.h>

#include <algorithm>

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
// One CTA owns the tile B[b][k0 .. k0+Kc)[n0 .. n0+Nt) in shared memory, staged
// by the Tensor Memory Accelerator (2-D boxes of 256 rows x Nt words) when the
// row pitch allows it, else by plain loads, followed by an all-zero sentinel
// row.  Each warp then takes one output row at a time:
//   1. its lanes load up to 32 words of the row's A bits for this K range,
//      count their set bits and prefix-sum the counts across the warp;
//   2. every lane writes the tile-row indices of its set bits into the warp's
//      list in shared memory (bits past the tile point at the sentinel);
//   3. the warp splits into 32/Nt groups of Nt lanes; group g ORs tile rows
//      list[g], list[g + 32/Nt], ... (four loads in flight per lane), lane l of
//      a group holding word n0 + l;
//   4. the groups' words are OR-ed together with shuffles and stored.
namespace {

constexpr int kRowOrThreads = 512;
constexpr int kListCap = 32 * 64 + 128;  // one batch of 32 A words, plus sentinel padding

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
  uint16_t* lists = reinterpret_cast<uint16_t*>(bs + (staged + 1) * G);
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
    for (int idx = tid; idx < kc_len * G; idx += blockDim.x) {
      const int r = idx / G, c = idx % G;
      const int64_t n = n0 + c;
      bs[idx] = (n < d.Nw) ? __ldg(d.B + (b * d.K + k0 + r) * d.Nw + n) : 0ull;
    }
  }
  if (tid < G) bs[(size_t)kc_len * G + tid] = 0ull;  // sentinel row
  __syncthreads();

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
      // list of the set bits (tile-row indices), in any order
      const int c = __popcll(a);
      int off = c ? atomicAdd(wcount, c) : 0;
      const int base = (kw0 + q * 32 + lane) * 64 - (int)k0;
      while (a) {
        const int bit = __ffsll((long long)a) - 1;
        a &= a - 1;
        const int ix = base + bit;
        list[off++] = (uint16_t)(ix < kc_len ? ix : kc_len);
      }
      __syncwarp();
      const int T = *wcount;
      // pad to a whole number of rounds with the sentinel row (4P entries,
      // which is more than one per lane when the groups are narrow)
      for (int t = lane; t < 4 * P; t += 32) list[T + t] = (uint16_t)kc_len;
      __syncwarp();
      for (int e = grp; e < T; e += 4 * P) {
        const int i0 = list[e], i1 = list[e + P], i2 = list[e + 2 * P], i3 = list[e + 3 * P];
        acc |= bs[i0 * G + lig] | bs[i1 * G + lig] | bs[i2 * G + lig] | bs[i3 * G + lig];
      }
      __syncwarp();
      if (lane == 0) {
        *wcount = 0;
        if (d.stat) atomicAdd(d.stat, (unsigned long long)T * G);
      }
      __syncwarp();
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

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

constexpr size_t kTileBudget = 156 * 1024;  // shared bytes for one B tile (the lists take 68 KB more)

}  // namespace

void rowor_plan(RowOrDesc& d, int64_t target_ctas) {
  // widest power-of-two tile (<= 32 words, <= the row) whose K range fits the budget
  int nt_max = 1;
  while (nt_max < 32 && nt_max < d.Nw) nt_max <<= 1;
  int Nt = nt_max;
  while (Nt > 2 && (size_t)(d.K + 1) * Nt * 8 > kTileBudget) Nt >>= 1;
  d.Nt = Nt;
  int64_t kc = (int64_t)(kTileBudget / ((size_t)Nt * 8)) - 1;
  const bool tma_ok = (d.Nw % 2 == 0) && (Nt % 2 == 0) &&
                      (reinterpret_cast<uintptr_t>(d.B) % 16 == 0) &&
                      (d.nbatch * d.K < (1ll << 31)) && encode_fn() != nullptr;
  d.use_tma = tma_ok ? 1 : 0;
  if (tma_ok) {
    // the staged rows are whole 256-row boxes, plus the sentinel row
    d.Kc = (int32_t)(((d.K + 255) / 256 * 256 <= kc) ? d.K : std::max<int64_t>(256, kc / 256 * 256));
  } else {
    d.Kc = (int32_t)((d.K <= kc) ? d.K : std::max<int64_t>(64, kc / 64 * 64));
  }
  d.n_tiles = (d.Nw + Nt - 1) / Nt;
  d.k_chunks = (d.K + d.Kc - 1) / d.Kc;
  d.atomic = d.k_chunks > 1 ? 1 : 0;
  const int64_t base = d.nbatch * d.n_tiles * d.k_chunks;
  const int64_t target = std::max<int64_t>(1, target_ctas);
  int64_t splits = (target + base - 1) / base;
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, (d.M + 15) / 16));
  d.rows_per_split = (d.M + splits - 1) / splits;
  d.row_splits = (d.M + d.rows_per_split - 1) / d.rows_per_split;
}

size_t rowor_smem_bytes(const RowOrDesc& d) {
  const int64_t rows = d.use_tma ? ((int64_t)d.Kc + 255) / 256 * 256 : d.Kc;
  return (size_t)(rows + 1) * d.Nt * 8 + (size_t)(kRowOrThreads / 32) * kListCap * 2 + 16 +
         (size_t)(kRowOrThreads / 32) * 4;
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

cudaError_t launch_rowor(const RowOrDesc* d_descs, const CUtensorMap* d_maps,
                         const int64_t* d_cta0, int nprob, int64_t grid, size_t smem, int Nt,
                         cudaStream_t s) {
  if (nprob <= 0 || grid <= 0) return cudaSuccess;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
#define PA_ROWOR(GG)                                                                         \
  do {                                                                                       \
    cudaFuncSetAttribute(rowor_tile_kernel<GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         (int)smem);                                                         \
    rowor_tile_kernel<GG><<<(unsigned)grid, kRowOrThreads, smem, s>>>(d_descs, d_maps, d_cta0, \
                                                                     nprob);                 \
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
