// Tensor-core path of the Boolean contraction (Eq. GAM of Sec. 3.3 for one
// cluster of Sec. 3.5): C[b][m][n] = OR_k A[b][m][k] AND B[b][k][n] computed as
// the 0/1 matrix product sum_k A[b][m][k] * B[b][k][n] on the 5th-generation
// tensor cores, then thresholded at > 0.
//
// Exactness: the operands hold only 0.0 and 1.0 (exact in E4M3), every product
// is 0 or 1 and the FP32 accumulator only ever adds non-negative values, so the
// sum is positive exactly when some product is 1 (a positive FP32 sum can round
// but never back to zero).  The result bits are therefore the Boolean product
// for any K.
//
// Data path: each operand is expanded once from its bit-packed row-OR layout
// into E4M3 bytes, K-major (A as [b][m][k]: unpack_rows_kernel; B as
// [b][n][k]: unpack_transpose_kernel, through 64 x 64 bit transposes in
// registers).  mma_bool_kernel stages 128-byte-wide K slices of both with TMA
// (128-byte swizzle) into a 4-deep ring, one elected thread issues
// tcgen05.mma kind::f8f6f4 (M = 128, N = BN, K = 32 per instruction) into a
// TMEM accumulator of 128 lanes x BN FP32 columns, and four epilogue warps read
// it back with tcgen05.ld, compare with zero and store bit-packed rows.  A
// product with few output tiles and a long K splits K over several CTAs per
// tile, whose bits are OR-ed into C (cleared beforehand): partial sums combine
// by OR because each is positive exactly when one of its products is.  Every
// wait on an mbarrier is bounded (about 1 s); on expiry the kernel sets the
// error word, finishes without storing and frees its TMEM.  (Expanding inside
// the contraction kernel instead re-expands every A tile once per column tile
// and every B tile once per row tile, and measured 2.4x slower.)
#include <cuda.h>
#include <string.h>

#include <algorithm>

#include "pa_internal.h"

namespace pa {

namespace {

constexpr int kMmaBM = 128;                   // rows of A per tile (TMEM lanes)
constexpr int kMmaBK = 128;                   // K bytes per stage = one 128-byte swizzle row
constexpr int kMmaStages = 4;
constexpr int kMmaATile = kMmaBM * kMmaBK;    // 16 KB
constexpr int kMmaMaxBN = 256;
constexpr int kMmaStageMax = kMmaATile + kMmaMaxBN * kMmaBK;  // 48 KB
constexpr int kMmaTmemCols = 256;
constexpr int kMmaThreads = 256;
constexpr size_t kMmaSmem = (size_t)kMmaStages * kMmaStageMax + 1024 + 256;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Wait for phase `parity` of an mbarrier, giving up after about one second.
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  for (long long it = 0; it < (1ll << 26); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > 2000000000ll) return false;
  }
  return false;
}

// Shared-memory matrix descriptor of a K-major operand tile in the canonical
// 128-byte swizzled layout: 8-row x 128-byte atoms stacked every 1024 bytes
// (stride byte offset), descriptor version 1, swizzle mode 2 (128 B).  The
// leading byte offset is unused because a stage is exactly one atom wide in K.
__device__ __forceinline__ uint64_t sw128_kmajor_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::f8f6f4: FP32 accumulator (bits 4-5 = 1),
// A and B E4M3 (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__device__ __forceinline__ uint32_t f8_idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
        "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
        "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

// 16 bits -> 16 bytes: byte j = E4M3 1.0 (0x38) when bit j is set, else 0.
// For a nibble n, n * 0x00204081 places bit j of n at bit 8j (the four shifted
// copies occupy disjoint bit ranges, so nothing carries); masking keeps those
// bits and the final multiply turns each 0/1 byte into 0/0x38.
__device__ __forceinline__ uint32_t expand4(uint32_t n) {
  return ((n * 0x00204081u) & 0x01010101u) * 0x38u;
}
__device__ __forceinline__ uint4 expand16(uint32_t bits) {
  return make_uint4(expand4(bits & 0xFu), expand4((bits >> 4) & 0xFu), expand4((bits >> 8) & 0xFu),
                    expand4((bits >> 12) & 0xFu));
}

// In-register transpose of a 64 x 64 bit block held by one warp: lane l holds
// rows l (lo) and l + 32 (hi), bit c of a row being column c; afterwards lane
// l holds columns l and l + 32.  Recursive block swap: for block size s the
// rows r and r + s (r & s == 0) exchange the columns c + s of row r with the
// columns c of row r + s (c & s == 0).
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

// A operand: out[r][64 w .. 64 w + 63] = E4M3 bytes of word w of bit row r
// (zero past the row's words).  One thread per input word; a warp's 32 words
// are written as 128 16-byte chunks, four stores of 512 contiguous bytes each
// (chunk c takes its 16 bits from the word of lane c / 4 by a shuffle).
// Problem blockIdx.y of the table.
__global__ void unpack_rows_kernel(const MmaDesc* __restrict__ descs) {
  const MmaDesc& d = descs[blockIdx.y];
  const uint64_t* __restrict__ in = d.A;
  uint8_t* __restrict__ out = d.Ab;
  const int64_t rows = d.nbatch * d.M, row_words = d.a_row_words, Kp = d.Kp;
  const int64_t wpr = Kp / 64;  // output words of 64 bytes per row (even)
  const int64_t total = rows * wpr;
  const int lane = threadIdx.x & 31;
  // the trip count is the same for every lane of a warp (total rounded up to
  // whole warps), so the shuffles and ballots see all 32 lanes
  const int64_t total_w = (total + 31) / 32 * 32;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total_w;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t word = 0;
    int64_t r = 0, w = 0;
    if (i < total) {
      r = i / wpr;
      w = i - r * wpr;
      word = w < row_words ? __ldg(in + r * row_words + w) : 0ull;
    }
    // chunk c = 32 j + lane of the warp's 128 is bits 16 (c % 4) .. of the
    // word of lane c / 4; it lands at byte 16 c past the warp's first output
    // byte, since the warp's words are consecutive in the output
    const int64_t i0 = i - lane;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 32 * j + lane;
      const uint64_t src = __shfl_sync(0xffffffffu, word, c >> 2);
      if (i0 + (c >> 2) < total)
        reinterpret_cast<uint4*>(out)[(i0 * 64 + 16 * (int64_t)c) / 16] =
            expand16((uint32_t)(src >> ((c & 3) * 16)) & 0xFFFFu);
    }
    // occupancy: the lanes whose word holds a set bit OR their (row tile,
    // K block) bits together per bitmap word, and one lane per word issues
    // the atomic (a warp covering one row of K <= 4096 issues one), skipped
    // when the bits are already set: every row of a tile sets the same bits,
    // and same-address atomics queue at L2
    if (d.occ_a) {
      const bool nzl = word != 0;
      const uint32_t nz = __ballot_sync(0xffffffffu, nzl);
      if (nzl) {
        const int64_t tile = (r / d.M) * d.m_tiles + (r % d.M) / 128, kb = w / 2;
        const int64_t widx = tile * d.kb_words + kb / 32;
        const uint32_t peers = __match_any_sync(nz, (unsigned long long)widx);
        const uint32_t bits = __reduce_or_sync(peers, 1u << (kb % 32));
        if (lane == __ffs(peers) - 1) {
          uint32_t* o = d.occ_a + widx;
          if ((__ldcg(o) & bits) != bits) atomicOr(o, bits);
        }
      }
    }
  }
}

// B operand: in [nb][K][Nw] bits (N packed) -> out [nb][N][Kp] bytes
// (K-major).  One warp per 64 x 64 bit block (batch, 64 K rows, 64 columns):
// lanes load K rows l and l + 32 and transpose in registers (lane l then holds
// columns l and l + 32, 64 K bits each); the 64 output rows of 64 bytes are
// written 8 rows per instruction, 4 lanes per row, words passed by shuffles.
// K rows >= K give zeros.
// Problem blockIdx.y of the table.
__global__ void unpack_transpose_kernel(const MmaDesc* __restrict__ descs) {
  // the contraction launch that follows may start its set-up now; it waits
  // for this grid to finish before it reads anything written here
  asm volatile("griddepcontrol.launch_dependents;");
  const MmaDesc& d = descs[blockIdx.y];
  const uint64_t* __restrict__ in = d.B;
  uint8_t* __restrict__ out = d.Bb;
  const int64_t nb = d.nbatch, K = d.K, N = d.N, Nw = d.Nw, Kp = d.Kp;
  const int lane = threadIdx.x & 31;
  const int64_t kblk = Kp / 64, nblk = Nw;
  const int64_t total = nb * kblk * nblk;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < total;
       it += nwarps) {
    const int64_t nbk = it % nblk, rest = it / nblk;
    const int64_t kb = rest % kblk, b = rest / kblk;
    const int64_t k0 = kb * 64 + lane;
    const uint64_t* src = in + b * K * Nw + nbk;
    uint64_t lo = k0 < K ? __ldg(src + k0 * Nw) : 0ull;
    uint64_t hi = k0 + 32 < K ? __ldg(src + (k0 + 32) * Nw) : 0ull;
    // a 64 x 64 block lies inside one (column tile, K block) pair
    if (d.occ_b && __any_sync(0xffffffffu, (lo | hi) != 0ull) && lane == 0) {
      const int64_t nt = (nbk * 64) / d.BN, kblock = (kb * 64) / 128;
      uint32_t* o = d.occ_b + (b * d.n_tiles + nt) * d.kb_words + kblock / 32;
      const uint32_t bit = 1u << (kblock % 32);
      if (!(__ldcg(o) & bit)) atomicOr(o, bit);
    }
    transpose64(lo, hi, lane);
    uint8_t* dst = out + (b * N) * Kp + kb * 64;
    const int sub = lane >> 2, c = lane & 3;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int r = 8 * (j & 3) + sub;  // row within the half
      const uint64_t v = __shfl_sync(0xffffffffu, j < 4 ? lo : hi, r);
      const int64_t n = nbk * 64 + (j < 4 ? 0 : 32) + r;
      if (n < N)
        *reinterpret_cast<uint4*>(dst + n * Kp + c * 16) =
            expand16((uint32_t)(v >> (16 * c)) & 0xFFFFu);
    }
  }
}

// One CTA per (problem, batch, 128-row tile of A, BN-column tile of B).
// Warp 0 lane 0: TMA producer.  Warp 1 lane 0: MMA issuer.  Warp 2: TMEM
// allocation.  Warps 4-7: epilogue (warp 4 + j reads TMEM lanes 32j..32j+31).
//
// Start-up: the launch may begin while the expansion kernel that writes the
// operands and occupancy bitmaps is still running (programmatic dependent
// launch).  Thread 0 reads the descriptor, initialises the barriers and
// signals the other warps through a named barrier, then waits for the
// expansion to finish (griddepcontrol.wait) and issues its first copies at
// once, while warp 2 allocates TMEM; no role reads the operands, the bitmaps
// or C before its own griddepcontrol.wait.
__global__ void __launch_bounds__(kMmaThreads, 1)
mma_bool_kernel(const MmaDesc* __restrict__ descs, const CUtensorMap* __restrict__ maps,
                const int64_t* __restrict__ cta0s, int nprob) {
  extern __shared__ uint8_t mma_raw[];
  uint8_t* smem =
      reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(mma_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)kMmaStages * kMmaStageMax);
  uint64_t* empty = full + kMmaStages;
  uint64_t* accum = empty + kMmaStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accum + 1);
  volatile int* sfail = reinterpret_cast<volatile int*>(tslot + 1);
  int* sp = const_cast<int*>(sfail) + 1;
  __shared__ MmaDesc sd;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t tmem = 0;  // warps 1-7 (the producer never touches TMEM)

  if (warp == 0) {
    if (lane == 0) {
      int lo = 0, hi = nprob - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cta0s[mid] <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
      }
      *sp = lo;
      sd = descs[lo];
      for (int s = 0; s < kMmaStages; ++s) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[s])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&empty[s])) : "memory");
      }
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(accum)) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      *sfail = 0;
    }
    __syncwarp();
    // descriptor, barriers and failure word are ready for warps 1-7
    asm volatile("bar.arrive 1, %0;" ::"r"(kMmaThreads) : "memory");
  } else {
    if (warp == 2) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       smem_addr(tslot)),
                   "r"(kMmaTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    asm volatile("bar.sync 1, %0;" ::"r"(kMmaThreads) : "memory");
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem = *tslot;
  }
  const int p = *sp;
  const MmaDesc& d = sd;
  int64_t t = (int64_t)blockIdx.x - cta0s[p];
  const int kc = (int)(t % d.ksplit);
  t /= d.ksplit;
  const int64_t nt = t % d.n_tiles;
  t /= d.n_tiles;
  const int64_t mt = t % d.m_tiles;
  const int64_t b = t / d.m_tiles;
  const int BN = d.BN;
  const int stage_bytes = kMmaATile + BN * kMmaBK;
  const int nk = (int)(d.Kp / kMmaBK);
  // the K blocks where both this CTA's A row tile and B column tile hold a set
  // bit (every block when the problem has no occupancy bitmaps); producer and
  // issuer walk the same sequence, the j-th active block using ring slot j
  const uint32_t* occa = d.occ_a ? d.occ_a + (b * d.m_tiles + mt) * d.kb_words : nullptr;
  const uint32_t* occb = d.occ_b ? d.occ_b + (b * d.n_tiles + nt) * d.kb_words : nullptr;
  // this CTA's K blocks [kb0, kb1) and the bitmap words that hold them
  const int kb0 = kc * d.kchunk, kb1 = min(nk, kb0 + d.kchunk);
  const int w0 = kb0 / 32, w1 = (kb1 + 31) / 32;
  const bool split = d.ksplit > 1;
  auto active = [&](int w) -> uint32_t {
    uint32_t m = 0xffffffffu;
    if (occa) m &= __ldcg(occa + w);
    if (occb) m &= __ldcg(occb + w);
    const int lo = max(kb0 - 32 * w, 0), hi = min(kb1 - 32 * w, 32);
    if (hi <= lo) return 0u;
    m &= (hi == 32 ? 0xffffffffu : (1u << hi) - 1u) & ~((1u << lo) - 1u);
    return m;
  };

  // the operands, the bitmaps and C belong to the expansion kernel until it
  // has finished: each role waits for it (griddepcontrol.wait) right before
  // its first access to them
  if (warp == 0) {
    if (lane == 0) {
      const CUtensorMap* ma = maps + 2 * p;
      const CUtensorMap* mb = ma + 1;
      // the tensor maps were written to global memory by a copy before the launch
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(ma) : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(mb) : "memory");
      asm volatile("griddepcontrol.wait;" ::: "memory");
      int j = 0;
      bool failed = false;
      for (int w = w0; w < w1 && !failed; ++w) {
        for (uint32_t m = active(w); m; m &= m - 1) {
          const int k = w * 32 + __ffs(m) - 1;
          const int s = j % kMmaStages;
          const uint32_t ph = (uint32_t)(j / kMmaStages) & 1u;
          if (j >= kMmaStages && !bar_wait(&empty[s], ph ^ 1u)) {
            *sfail = 1;
            failed = true;
            break;
          }
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                           smem_addr(&full[s])),
                       "r"(stage_bytes)
                       : "memory");
          const uint32_t dst_a = smem_addr(smem + (size_t)s * kMmaStageMax);
          const uint32_t dst_b = dst_a + kMmaATile;
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst_a),
              "l"(reinterpret_cast<uint64_t>(ma)), "r"(k * kMmaBK), "r"((int)(mt * kMmaBM)),
              "r"((int)b), "r"(smem_addr(&full[s]))
              : "memory");
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst_b),
              "l"(reinterpret_cast<uint64_t>(mb)), "r"(k * kMmaBK), "r"((int)(nt * BN)),
              "r"((int)b), "r"(smem_addr(&full[s]))
              : "memory");
          ++j;
        }
      }
      // after a failure anywhere, wait (bounded) for the copies still in
      // flight before the CTA's shared memory is released
      if (*sfail)
        for (int q = j > kMmaStages ? j - kMmaStages : 0; q < j; ++q)
          bar_wait(&full[q % kMmaStages], (uint32_t)(q / kMmaStages) & 1u);
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      asm volatile("griddepcontrol.wait;" ::: "memory");
      const uint32_t idesc = f8_idesc(kMmaBM, BN);
      int j = 0;
      bool failed = false;
      for (int w = w0; w < w1 && !failed; ++w) {
        for (uint32_t m = active(w); m; m &= m - 1) {
          const int s = j % kMmaStages;
          const uint32_t ph = (uint32_t)(j / kMmaStages) & 1u;
          if (!bar_wait(&full[s], ph)) {
            *sfail = 1;
            failed = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_addr(smem + (size_t)s * kMmaStageMax), b0 = a0 + kMmaATile;
#pragma unroll
          for (int kk = 0; kk < kMmaBK / 32; ++kk) {
            const uint64_t ad = sw128_kmajor_desc(a0 + kk * 32), bd = sw128_kmajor_desc(b0 + kk * 32);
            const uint32_t acc = (j > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  smem_addr(&empty[s]))
              : "memory");
          ++j;
        }
      }
      // arrives once every MMA issued above has completed (also on failure)
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_addr(accum))
          : "memory");
    }
    __syncwarp();
  } else if (warp >= 4) {
    const int ew = warp - 4;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // no K block in common: nothing was accumulated, every sum is zero
    // (decided while the products run)
    bool none = true;
    for (int w = w0; w < w1 && none; ++w) none = (active(w) == 0);
    const bool ok = bar_wait(accum, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // with K split, a CTA that summed nothing leaves C as it is (other CTAs
    // OR their bits into the same words)
    const bool store = ok && !*sfail && !(split && none);
    const int64_t m = mt * kMmaBM + ew * 32 + lane;
    // up to 128 columns per round: every TMEM load of the round is in flight
    // before the one wait
    const int G = BN < 128 ? BN : 128;
    for (int c0 = 0; c0 < BN; c0 += G) {
      uint32_t v[128];
      const uint32_t ta = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)c0;
      if (none) {
#pragma unroll
        for (int q = 0; q < 128; ++q) v[q] = 0u;
      } else {
        tmem_ld32(ta, v);
        tmem_ld32(ta + 32u, v + 32);
        if (G == 128) {
          tmem_ld32(ta + 64u, v + 64);
          tmem_ld32(ta + 96u, v + 96);
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h * 64 >= G) break;
        const uint32_t* vh = v + 64 * h;
        const int c = (c0 >> 6) + h;  // 64-column chunk of the tile
        if (d.counts) {
          // counting semiring: every sum is an integer <= K <= 2^24, exact in
          // FP32.  The warp's 32 rows x 64 counts go through shared memory (the
          // operand ring is idle once every product is done; rows padded to 65
          // words against bank conflicts) so that each store writes 32
          // consecutive counts of one row.
          if (store) {
            uint32_t* st = reinterpret_cast<uint32_t*>(smem) + ew * (32 * 65);
#pragma unroll
            for (int q = 0; q < 64; ++q) st[lane * 65 + q] = (uint32_t)__uint_as_float(vh[q]);
            __syncwarp();
            const int64_t n0 = nt * BN + c * 64;
            for (int rr = 0; rr < 32; ++rr) {
              const int64_t mm = mt * kMmaBM + ew * 32 + rr;
              if (mm >= d.M) break;
              uint32_t* row = d.counts + (b * d.M + mm) * d.N;
              if (n0 + lane < d.N) row[n0 + lane] = st[rr * 65 + lane];
              if (n0 + 32 + lane < d.N) row[n0 + 32 + lane] = st[rr * 65 + 32 + lane];
            }
            __syncwarp();
          }
          continue;
        }
        uint64_t word = 0;
#pragma unroll
        for (int q = 0; q < 64; ++q) word |= (uint64_t)(__uint_as_float(vh[q]) > 0.0f) << q;
        const int64_t w = nt * (BN / 64) + c;
        if (store && m < d.M && w < d.Nw) {
          const int64_t rem = d.N - w * 64;
          if (rem < 64) word &= (1ull << rem) - 1ull;
          uint64_t* dst = d.C + (b * d.M + m) * d.Nw + w;
          if (!split) *dst = word;
          else if (word) atomicOr(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)word);
        }
      }
    }
    if (!ok && lane == 0) atomicExch(d.err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 2) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kMmaTmemCols)
                 : "memory");
  }
  if (threadIdx.x == 0 && *sfail) atomicExch(d.err, 1);
}

// Random bits for autotuning: bit j of word i is set when the SplitMix64 mix
// of (seed, 64 i + j) falls below density * 2^64; bits of column >= valid in
// each row of row_words words stay zero.
__global__ void random_bits_kernel(uint64_t* __restrict__ w, int64_t nwords, int64_t row_words,
                                   int64_t valid, double density, uint64_t seed) {
  const uint64_t thr = density >= 1.0 ? ~0ull : (uint64_t)(density * 18446744073709551616.0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col0 = (i % row_words) * 64;
    uint64_t word = 0;
    for (int j = 0; j < 64 && col0 + j < valid; ++j) {
      uint64_t z = seed + (uint64_t)(i * 64 + j) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      word |= (uint64_t)(z < thr) << j;
    }
    w[i] = word;
  }
}

// ext and stride are device arrays of ndim entries (in the call's blob)
__global__ void permute_u32_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                   int ndim, const int64_t* __restrict__ ext,
                                   const int64_t* __restrict__ stride, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t rest = i, src = 0;
    for (int a = ndim - 1; a >= 0; --a) {
      const int64_t e = __ldg(ext + a);
      const int64_t q = rest % e;
      rest /= e;
      src += q * __ldg(stride + a);
    }
    out[i] = in[src];
  }
}

}  // namespace

void launch_permute_u32(const uint32_t* in, uint32_t* out, int ndim, const int64_t* d_ext,
                        const int64_t* d_stride, int64_t total, cudaStream_t s) {
  if (total <= 0) return;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  permute_u32_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, out, ndim, d_ext, d_stride, total);
}

void launch_random_bits(uint64_t* w, int64_t nwords, int64_t row_words, int64_t valid,
                        double density, uint64_t seed, cudaStream_t s) {
  if (nwords <= 0) return;
  int64_t blocks = (nwords + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  random_bits_kernel<<<(unsigned)blocks, 256, 0, s>>>(w, nwords, row_words, valid, density, seed);
}

void mma_plan(MmaDesc& d) {
  d.BN = d.N <= 64 ? 64 : d.N <= 128 ? 128 : 256;
  d.Nw = (d.N + 63) / 64;
  d.Kp = (d.K + kMmaBK - 1) / kMmaBK * kMmaBK;
  d.m_tiles = (d.M + kMmaBM - 1) / kMmaBM;
  d.n_tiles = (d.N + d.BN - 1) / d.BN;
  const int64_t nk = d.Kp / kMmaBK;
  d.kb_words = (nk + 31) / 32;
  // Few output tiles and a long K (a cluster that sums many variables into a
  // small result) would leave most SMs idle: split K over up to one CTA per
  // SM, each with at least 8 K blocks.  Only for the Boolean product, whose
  // partial results combine by OR.
  d.ksplit = 1;
  d.kchunk = (int32_t)nk;
  const int64_t tiles = d.nbatch * d.m_tiles * d.n_tiles;
  if (!d.counts && tiles < 152) {
    const int64_t want = std::min<int64_t>(152 / tiles, nk / 8);
    if (want > 1) {
      const int64_t chunk = (nk + want - 1) / want;
      d.kchunk = (int32_t)chunk;
      d.ksplit = (int32_t)((nk + chunk - 1) / chunk);
    }
  }
}

int64_t mma_occ_words(const MmaDesc& d) {
  return d.nbatch * (d.m_tiles + d.n_tiles) * d.kb_words;
}

int64_t mma_ctas(const MmaDesc& d) { return d.nbatch * d.m_tiles * d.n_tiles * d.ksplit; }

size_t mma_smem_bytes() { return kMmaSmem; }

cudaError_t mma_encode_maps(const MmaDesc& d, CUtensorMap* maps2) {
  memset(maps2, 0, 2 * sizeof(CUtensorMap));
  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  const int64_t rows[2] = {d.M, d.N};
  const uint8_t* base[2] = {d.Ab, d.Bb};
  const cuuint32_t box_rows[2] = {(cuuint32_t)kMmaBM, (cuuint32_t)d.BN};
  for (int i = 0; i < 2; ++i) {
    const cuuint64_t dims[3] = {(cuuint64_t)d.Kp, (cuuint64_t)rows[i], (cuuint64_t)d.nbatch};
    const cuuint64_t strides[2] = {(cuuint64_t)d.Kp, (cuuint64_t)(d.Kp * rows[i])};
    const cuuint32_t box[3] = {(cuuint32_t)kMmaBK, box_rows[i], 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = enc(&maps2[i], CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(base[i]), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

int64_t unpack_blocks_a(const MmaDesc& d) {
  return std::min<int64_t>((d.nbatch * d.M * (d.Kp / 64) + 255) / 256, 152 * 16);
}

int64_t unpack_blocks_b(const MmaDesc& d) {
  return std::min<int64_t>((d.nbatch * (d.Kp / 64) * d.Nw + 7) / 8, 152 * 16);
}

void launch_unpack(const MmaDesc* d_descs, int nprob, int64_t blocks_a, int64_t blocks_b,
                   cudaStream_t s) {
  if (nprob <= 0) return;
  // the expansion kernels use no shared memory; asking for the largest
  // shared-memory carveout anyway keeps the SMs in the configuration the
  // contraction kernel that follows needs, so that no reconfiguration sits
  // between the two launches
  static bool carveout = [] {
    cudaFuncSetAttribute(reinterpret_cast<const void*>(unpack_rows_kernel),
                         cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    cudaFuncSetAttribute(reinterpret_cast<const void*>(unpack_transpose_kernel),
                         cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    return true;
  }();
  (void)carveout;
  if (blocks_a > 0) unpack_rows_kernel<<<dim3((unsigned)blocks_a, (unsigned)nprob), 256, 0, s>>>(d_descs);
  if (blocks_b > 0)
    unpack_transpose_kernel<<<dim3((unsigned)blocks_b, (unsigned)nprob), 256, 0, s>>>(d_descs);
}

cudaError_t launch_mma(const MmaDesc* d_descs, const CUtensorMap* d_maps, const int64_t* d_cta0,
                       int nprob, int64_t grid, cudaStream_t s) {
  if (nprob <= 0 || grid <= 0) return cudaSuccess;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  smem_limit(reinterpret_cast<const void*>(mma_bool_kernel), kMmaSmem);
  // programmatic dependent launch: the set-up overlaps the expansion kernel
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kMmaThreads);
  cfg.dynamicSmemBytes = kMmaSmem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, mma_bool_kernel, d_descs, d_maps, d_cta0, nprob);
}

}  // namespace pa
