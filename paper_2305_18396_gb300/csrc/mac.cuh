// mac.cuh -- the slot-wise multiply-accumulate of Algorithm 1 step 3 (NTT domain):
// operand layout, arithmetic helpers and the block body shared by the single, batched and
// multi-product launches.
#pragma once

#include "async.cuh"
#include "he_common.cuh"

namespace he {

// Operand word of the multiply-accumulate: a residue v < 2^50 stored pre-split as
// v mod 2^25 in the low half and floor(v / 2^25) in the high half.
__device__ __forceinline__ u64 split_word(u64 v) { return (v & ((1ull << 25) - 1)) | ((v >> 25) << 32); }

// Slot-wise multiply-accumulate (Algorithm 1 step 3 in the NTT domain).  For each
// prime l and slot s the outputs form a small matrix product over the k-blocks J:
//   out[r][I] = sum_J ct[r][J] * pt[I][J],   r = (Lb, component c) rows, I columns.
//
// Operand layout ("slot-chunked"): both the NTT of the input ciphertexts and the
// encoded weights store, for every row (resp. column), prime and chunk of 32 slots, the
// 32-slot vectors of all nJ k-blocks contiguously:
//   word ((row * L + l) * (N / 32) + s / 32) * nJ * 32 + J * 32 + s % 32.
// A block owns one 32-slot chunk of one prime and a (kRows x kCols) output tile.  Per
// stage, a producer warp streams JB consecutive k-blocks of every operand row of the tile
// into shared memory -- one 1-D bulk copy (TMA) of JB * 256 contiguous bytes per row --
// completing on the stage's mbarrier; STAGES stages are in flight.  Each consumer thread
// owns one slot and a TM x TN register tile.  Operands < 2^50 are stored split, x = x0 + 2^25 x1
// (split_word), and multiplied Karatsuba-style: three mad.wide.u32 per slot product into lo / mid / hi
// 64-bit columns (no carries for nJ <= 4096), reduced once per output at the end.
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s: a copy that never lands is an error

// Operands arrive pre-split (split_word): halves of the word, plus their sum for Karatsuba.
__device__ __forceinline__ void split25(u64 w, u32& a0, u32& a1, u32& as) {
  a0 = (u32)w;
  a1 = (u32)(w >> 32);
  as = a0 + a1;
}

// Where the multiply-accumulate writes component c of (global) output ciphertext g:
// base[c] + g * ct_stride[c] + l * N + slot.
struct OutPlace {
  u64* base[2];
  u64 ct_stride[2];
};

// acc += a * b with a 32 x 32 -> 64-bit product (one mad.wide.u32).
__device__ __forceinline__ void mad_wide(u64& acc, u32 a, u32 b) {
  asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}

__host__ __device__ constexpr u64 chunked_index(u64 row, u32 J, u32 l, u32 s, u32 nJ, u32 L, u32 N) {
  return ((row * L + l) * (N >> 5) + (s >> 5)) * (u64)nJ * 32 + (u64)J * 32 + (s & 31);
}

template <int TM, int TN, int WR, int WC, int JB, int STAGES>
struct MacCfg {
  static constexpr int kTM = TM, kTN = TN, kWR = WR, kWC = WC, kJB = JB, kStages = STAGES;
  static constexpr int kRows = TM * WR, kCols = TN * WC;
  static constexpr int kThreads = 32 * WR * WC;
  static constexpr int kStageWords = (kRows + kCols) * JB * 32;
  static constexpr size_t kSmemBytes = (size_t)STAGES * kStageWords * sizeof(u64);
};

// One block's share of a product: the 32-slot chunk `chunk` of prime l and the output
// tile with first row r0 and first column c0 (ct0 = global index of the product's first
// output ciphertext, for the output placement; shared memory: the caller's dynamic
// buffer of M::kSmemBytes bytes).  Warp-specialized: the block has M::kThreads consumer
// threads plus one producer warp (the last).  The producer streams the stages (waiting on a stage's "empty"
// barrier before refilling it); each consumer warp waits on the stage's "full" barrier
// itself, computes, and releases the stage by arriving on "empty" (count = consumer warps).
// No block-wide barrier after set-up.  Every wait is bounded and warp-uniform; a warp that
// gives up records the error flag and leaves, which in turn makes the others' waits expire.
template <class M>
__device__ __forceinline__ void mac_tile_ws(const u64* __restrict__ ctN, const u64* __restrict__ pt,
                                            const OutPlace& out, u64 ct0, u32 nI, u32 nJ, u32 nLb, u32 r0, u32 c0,
                                            u32 chunk, u32 l, int* err, const Consts& C, u64* sm) {
  __shared__ __align__(8) uint64_t full[M::kStages], empty[M::kStages];
  constexpr int TM = M::kTM, TN = M::kTN, JB = M::kJB, ST = M::kStages;
  constexpr u32 kConsumers = M::kWR * M::kWC;

  const u32 N = C.N, L = C.L;
  const PrimeConsts P = C.p[l];
  const u32 rows = 2 * nLb;
  const u32 nrows = min((u32)M::kRows, rows - r0), ncols = min((u32)M::kCols, nI - c0);
  const u32 nstages = (nJ + JB - 1) / JB;
  const u32 warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int st = 0; st < ST; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], kConsumers);
    }
    mbar_init_fence();
  }
  __syncthreads();

  if (warp == kConsumers) {  // producer warp
    u32 issued = 0;
    for (u32 i = 0; i < nstages; ++i) {
      const u32 st = i % ST;
      if (i >= (u32)ST && !mbar_wait_warp(&empty[st], ((i / ST) - 1) & 1, kWaitLimitNs)) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      const u32 J0 = i * JB, jb = min((u32)JB, nJ - J0);
      const u32 bytes = jb * 32 * sizeof(u64);
      if (lane == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&full[st], (nrows + ncols) * bytes);
      }
      __syncwarp();
      u64* stage = sm + st * M::kStageWords;
      for (u32 t = lane; t < nrows + ncols; t += 32) {
        const bool is_row = t < nrows;
        const u64* src = is_row ? ctN + chunked_index(r0 + t, J0, l, chunk << 5, nJ, L, N)
                                : pt + chunked_index(c0 + (t - nrows), J0, l, chunk << 5, nJ, L, N);
        u64* dst = stage + (is_row ? t : M::kRows + (t - nrows)) * (JB * 32);
        bulk_copy_g2s(dst, src, bytes, &full[st]);
      }
      issued = i + 1;
    }
    // before leaving, let the copies of the last stages land (bounded): the block's shared
    // memory must not be released with copies in flight
    for (u32 i = issued > (u32)ST ? issued - ST : 0; i < issued; ++i)
      mbar_wait_warp(&full[i % ST], (i / ST) & 1, kWaitLimitNs);
    return;
  }

  const u32 wr = warp % M::kWR, wc = warp / M::kWR;
  u64 lo[TM][TN], mid[TM][TN], hi[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) lo[a][b] = mid[a][b] = hi[a][b] = 0;

  for (u32 i = 0; i < nstages; ++i) {
    const u32 st = i % ST;
    if (!mbar_wait_warp(&full[st], (i / ST) & 1, kWaitLimitNs)) {
      if (lane == 0) atomicExch(err, 1);
      return;
    }
    const u64* stage = sm + st * M::kStageWords;
    const u32 jb = min((u32)JB, nJ - i * JB);
    const u64* prow = stage + (M::kRows + wc * TN) * (JB * 32) + lane;
    const u64* crow = stage + (wr * TM) * (JB * 32) + lane;
    auto kblock = [&](u32 jj) {
      u32 p0[TN], p1[TN], ps[TN];
#pragma unroll
      for (int b = 0; b < TN; ++b) split25(prow[b * (JB * 32) + jj * 32], p0[b], p1[b], ps[b]);
#pragma unroll
      for (int a = 0; a < TM; ++a) {
        u32 x0, x1, xs;
        split25(crow[a * (JB * 32) + jj * 32], x0, x1, xs);
#pragma unroll
        for (int b = 0; b < TN; ++b) {
          mad_wide(lo[a][b], x0, p0[b]);
          mad_wide(hi[a][b], x1, p1[b]);
          mad_wide(mid[a][b], xs, ps[b]);
        }
      }
    };
    if (jb == (u32)JB) {
#pragma unroll
      for (int jj = 0; jj < JB; ++jj) kblock(jj);
    } else {
      for (u32 jj = 0; jj < jb; ++jj) kblock(jj);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }

  const u32 s = (chunk << 5) + lane;
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const u32 r = r0 + wr * TM + a;
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const u32 I = c0 + wc * TN + b;
      if (r < rows && I < nI) {
        const u64 cross = mid[a][b] - lo[a][b] - hi[a][b];  // sum of x0 y1 + x1 y0
        u64 v = reduce_word(lo[a][b], P);
        v = add_mod(v, csub(mul_shoup(cross, P.r25, P.r25_sh, P.q), P.q), P.q);
        v = add_mod(v, csub(mul_shoup(hi[a][b], P.r50, P.r50_sh, P.q), P.q), P.q);
        const u32 c = r & 1;
        out.base[c][(ct0 + (u64)(r >> 1) * nI + I) * out.ct_stride[c] + (u64)l * N + s] = v;
      }
    }
  }
}

// The configuration the library launches.
// The launched configuration: 4 x 2 register tiles, 2 x 4 consumer warps (8 x 8 output
// tile), 8 k-blocks per stage, 3 stages (96 KB of shared memory, 2 blocks per SM).
// Measured on the BERT-base layer (ms per layer): 3 stages 3.218, 2 stages 3.273,
// 4 k-blocks x 4 stages 3.558, 8 x 4 tiles with 3 blocks per SM 3.291.  The macros let a
// build try another configuration (-DHE_MAC_TM=... etc.).
#ifndef HE_MAC_TM
#define HE_MAC_TM 4
#define HE_MAC_TN 2
#define HE_MAC_WR 2
#define HE_MAC_WC 4
#define HE_MAC_JB 8
#define HE_MAC_ST 3
#endif
#ifndef HE_MAC_MINB
#define HE_MAC_MINB 2
#endif
using MacProd = MacCfg<HE_MAC_TM, HE_MAC_TN, HE_MAC_WR, HE_MAC_WC, HE_MAC_JB, HE_MAC_ST>;
constexpr int kMacMinBlocks = HE_MAC_MINB;

}  // namespace he
