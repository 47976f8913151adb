// mac_tcr.cuh -- the slot-wise multiply-accumulate of Algorithm 1 step 3 for coset products
// with few k-blocks (nJ <= 64), on the tcgen05 tensor cores with the roles of the operands
// swapped relative to mac_tc.cuh.
//
// Same exact method as mac_tc.cuh (balanced base-256 digits, exact in bf16; the 49 digit
// products folded onto 13 diagonal accumulators by TMEM column offsets; f32 sums that stay
// exact integers; recombination mod q_l by tc_combine4), but the MMA's M dimension holds 128
// operand rows of the inputs (rows (2 Lb + c) G + g of a coset product) and its N dimension
// the 7 digit planes of 16 weight rows.  A product with few k-blocks has one accumulation
// round per output, so its cost is the recombination: with the weight rows on M (mac_tc.cuh)
// a product of 32 or 64 weight rows leaves three or two of the four TMEM lane quadrants --
// and the SM sub-partitions that read them -- without work, and it would need more weight
// rows per block (k_b larger, more outputs) to fill the tile.  Here the inputs fill M
// (a coset product has 2 nLb G >= 128 rows per slot whenever G >= 64) for any nI.
//
// A work unit is one prime l, one slot s and 128 input rows; it splits those rows' words
// (all of their k-blocks, at most 4 stages of 16) into digit planes once, in shared memory,
// then streams every 16-row tile of the weights past them: per weight tile and stage, 7
// MMAs (M = 128 input rows, plane a; N = 7 weight planes x 16 rows; K = 16 k-blocks) into
// one of two TMEM accumulator sets, so the recombination of one weight tile overlaps the
// MMAs of the next.
//
// Layouts.  Inputs: the coset stage-tiled layout of mac_tc.cuh (128 rows of one (l, s,
// stage) are 16 KB contiguous).  Weights ("row-major digit tiles"): for prime l, slot s,
// weight-row tile t (16 rows) and stage js, one B operand tile of 112 rows (plane b, row i:
// row 16 b + i) x 16 k-blocks, K-major no-swizzle (tc::tile_offset(16 b + i, j, 32, 2)),
// 3584 bytes, tiles in (l, s, t, js) order, zero past the product's rows and k-blocks.
#pragma once

#include "mac_tc.cuh"

namespace he {

constexpr u32 kTcrM = 128;                 // input rows per unit (MMA M)
constexpr u32 kTcrI = 16;                  // weight rows per tile
constexpr u32 kTcrMaxStages = 4;           // k-blocks per product at most 64
constexpr u32 kTcrBStages = 8;             // weight tiles in flight
constexpr u32 kTcrRawStages = 4;           // raw input stages in flight (a unit's at most 4 load together)
constexpr u32 kTcrSplitWarps = 4;
constexpr u32 kTcrEpiWarps = 8;            // two per TMEM lane quadrant, 8 weight rows each
constexpr u32 kTcrEpi0 = 2 + kTcrSplitWarps;
constexpr u32 kTcrThreads = 32 * (kTcrEpi0 + kTcrEpiWarps);  // 448
constexpr u32 kTcrPlaneBytes = kTcrM * kTcJB * 2;           // one digit plane of the unit's rows: 4 KB
constexpr u32 kTcrABytes = kTcPlanes * kTcrPlaneBytes;      // a stage's 7 planes: 28 KB
constexpr u32 kTcrRawBytes = kTcrM * kTcRawRow;             // a stage's raw words: 16 KB
constexpr u32 kTcrBBytes = kTcPlanes * kTcrI * kTcJB * 2;   // one weight tile: 3584 bytes
constexpr u32 kTcrSmem =
    kTcrMaxStages * kTcrABytes + kTcrRawStages * kTcrRawBytes + kTcrBBytes * kTcrBStages + kTcZBytes + 128;
static_assert(kTcrSmem <= 227 * 1024, "row-major tensor-core MAC shared memory above the per-block limit");

__host__ __device__ inline u32 tcr_tiles_I(u32 nI) { return (nI + kTcrI - 1) / kTcrI; }
__host__ __device__ inline u32 tcr_tiles_R(u32 R) { return (R + kTcrM - 1) / kTcrM; }
__host__ __device__ constexpr u64 tcr_weight_words(u32 nI, u32 nJ, u32 L, u32 S) {
  return (u64)L * S * ((nI + kTcrI - 1) / kTcrI) * tc_stages(nJ) * (kTcrBBytes / 8);
}
__host__ __device__ constexpr u64 tcr_weight_offset(u32 t, u32 l, u32 s, u32 js, u32 nIt, u32 nS, u32 S) {
  return ((((u64)l * S + s) * nIt + t) * nS + js) * kTcrBBytes;
}
// Units of one product: input-row tiles fastest (the units of one slot share its weights in
// L2), then slots, then primes.
__host__ __device__ inline u64 tcr_units(u32 S, u32 L, u32 R) { return (u64)L * S * tcr_tiles_R(R); }

struct TcrWork {
  const u64* ctN;      // inputs' coset transforms (stage-tiled)
  const uint8_t* ptd;  // row-major digit tiles of the weights
  u64* acc;            // sums: output o, component c, prime l at acc + ((o 2 + c) L + l) 2N + g S + s
  u64 ct0;
  u32 nI, nJ, r0, s, l, S, R, logG;
};

__device__ __forceinline__ void tcr_unit(u64 u, u32 S, u32 R, TcrWork& w) {
  const u32 nRt = tcr_tiles_R(R);
  w.r0 = (u32)(u % nRt) * kTcrM;
  u /= nRt;
  w.s = (u32)(u % S);
  w.l = (u32)(u / S);
  w.S = S;
  w.R = R;
}

struct TcrShared {
  uint64_t raw_full[kTcrRawStages], raw_empty[kTcrRawStages], a_full[kTcrMaxStages], a_free;
  uint64_t b_full[kTcrBStages], b_empty[kTcrBStages];
  uint64_t acc_full[2], acc_empty[2], done;
  uint32_t tmem;
  int abort;
};

// One block per SM: work units blockIdx.x, blockIdx.x + gridDim.x, ... < total, each
// described by get(g, w).  smem: the caller's dynamic buffer of kTcrSmem bytes.
template <class GetWork>
__device__ __forceinline__ void mac_tcr_run(const GetWork& get, u64 total, int* err, const Consts& C, uint8_t* smem,
                                            TcrShared& sh) {
  uint8_t* const Ad = smem;                                         // [stage][plane][128 x 16] digits
  uint8_t* const Raw = Ad + kTcrMaxStages * kTcrABytes;             // [kTcrRawStages][128 rows x 128 bytes]
  uint8_t* const Bt = Raw + kTcrRawStages * kTcrRawBytes;           // [kTcrBStages][3584]
  uint8_t* const Zt = Bt + kTcrBBytes * kTcrBStages;                // 96 zero rows
  const u32 warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 N = C.N;

  if (threadIdx.x == 0) {
    for (u32 b = 0; b < kTcrRawStages; ++b) {
      mbar_init(&sh.raw_full[b], 1);
      mbar_init(&sh.raw_empty[b], kTcrSplitWarps);
    }
    for (u32 b = 0; b < 2; ++b) {
      mbar_init(&sh.acc_full[b], 1);
      mbar_init(&sh.acc_empty[b], kTcrEpiWarps);
    }
    for (u32 b = 0; b < kTcrMaxStages; ++b) mbar_init(&sh.a_full[b], kTcrSplitWarps);
    mbar_init(&sh.a_free, 1);
    for (u32 b = 0; b < kTcrBStages; ++b) {
      mbar_init(&sh.b_full[b], 1);
      mbar_init(&sh.b_empty[b], 1);
    }
    mbar_init(&sh.done, 1);
    sh.abort = 0;
    mbar_init_fence();
  }
  for (u32 i = threadIdx.x; i < kTcZBytes / 16; i += blockDim.x) reinterpret_cast<uint4*>(Zt)[i] = make_uint4(0, 0, 0, 0);
  tc::fence_smem_to_async();
  if (warp == 1) tc::tmem_alloc(&sh.tmem, kTcCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = sh.tmem;
  volatile int* abort_flag = &sh.abort;
  auto give_up = [&]() {
    if (lane == 0) {
      atomicExch(err, 1);
      *abort_flag = 1;
    }
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    u32 rc = 0, bc = 0;  // raw stages and weight tiles issued
    bool ok = true;
    for (u64 g = blockIdx.x; ok && g < total && !*abort_flag; g += gridDim.x) {
      TcrWork w;
      get(g, w);
      const u32 nS = tc_stages(w.nJ), nIt = tcr_tiles_I(w.nI), nc = min(kTcrM, w.R - w.r0);
      for (u32 js = 0; ok && js < nS; ++js, ++rc) {
        const u32 b = rc % kTcrRawStages;
        if (rc >= kTcrRawStages &&
            !mbar_wait_warp(&sh.raw_empty[b], ((rc / kTcrRawStages) - 1) & 1, kWaitLimitNs)) {
          give_up();
          ok = false;
          break;
        }
        if (lane == 0) {
          fence_proxy_async_smem();
          mbar_arrive_expect_tx(&sh.raw_full[b], nc * kTcRawRow);
          bulk_copy_g2s(Raw + b * kTcrRawBytes, w.ctN + tc_index(w.r0, js * kTcJB, w.l, w.s, w.R, nS, w.S),
                        nc * kTcRawRow, &sh.raw_full[b]);
        }
        __syncwarp();
      }
      for (u32 t = 0; ok && t < nIt; ++t)
        for (u32 js = 0; js < nS; ++js, ++bc) {
          const u32 b = bc % kTcrBStages;
          if (bc >= kTcrBStages &&
              !mbar_wait_warp(&sh.b_empty[b], ((bc / kTcrBStages) - 1) & 1, kWaitLimitNs)) {
            give_up();
            ok = false;
            break;
          }
          if (lane == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&sh.b_full[b], kTcrBBytes);
            bulk_copy_g2s(Bt + b * kTcrBBytes, w.ptd + tcr_weight_offset(t, w.l, w.s, js, nIt, nS, w.S), kTcrBBytes,
                          &sh.b_full[b]);
          }
          __syncwarp();
        }
    }
    // copies still in flight must land before the block's shared memory is released
    for (u32 k = rc > kTcrRawStages ? rc - kTcrRawStages : 0; k < rc; ++k)
      mbar_wait_warp(&sh.raw_full[k % kTcrRawStages], (k / kTcrRawStages) & 1, kWaitLimitNs);
    for (u32 k = bc > kTcrBStages ? bc - kTcrBStages : 0; k < bc; ++k)
      mbar_wait_warp(&sh.b_full[k % kTcrBStages], (k / kTcrBStages) & 1, kWaitLimitNs);
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issue
    const uint32_t id_main = tc::idesc_bf16_f32(kTcrM, kTcPlanes * kTcrI);
    const uint32_t id_zero = tc::idesc_bf16_f32(kTcrM, (kTcDiag - kTcPlanes) * kTcrI);
    u32 bc = 0, rnd = 0;
    u32 acnt[kTcrMaxStages] = {0, 0, 0, 0};  // completed phases of a_full[js] (units with more than js stages)
    bool ok = true;
    for (u64 g = blockIdx.x; ok && g < total && !*abort_flag; g += gridDim.x) {
      TcrWork w;
      get(g, w);
      const u32 nS = tc_stages(w.nJ), nIt = tcr_tiles_I(w.nI);
      for (u32 t = 0; ok && t < nIt; ++t, ++rnd) {
        const u32 set = rnd & 1;
        if (rnd >= 2 && !mbar_wait_warp(&sh.acc_empty[set], ((rnd >> 1) - 1) & 1, kWaitLimitNs)) {
          give_up();
          ok = false;
          break;
        }
        for (u32 js = 0; js < nS; ++js, ++bc) {
          const u32 b = bc % kTcrBStages;
          if ((t == 0 && !mbar_wait_warp(&sh.a_full[js], acnt[js] & 1, kWaitLimitNs)) ||  // the unit's digits are split
              !mbar_wait_warp(&sh.b_full[b], (bc / kTcrBStages) & 1, kWaitLimitNs)) {  // the weight tile landed
            give_up();
            ok = false;
            break;
          }
          tc::fence_after_sync();
          if (lane == 0) {
            const uint32_t d = tmem + set * kTcSetCols;
            const uint64_t bdesc = tc::smem_desc(Bt + b * kTcrBBytes, 128, 256);
#pragma unroll
            for (u32 a = 0; a < kTcPlanes; ++a) {
              const uint64_t adesc = tc::smem_desc(Ad + js * kTcrABytes + a * kTcrPlaneBytes, 128, 256);
              tc::mma_bf16(d + a * kTcrI, adesc, bdesc, id_main, (a > 0 || js > 0) ? 1u : 0u);
              if (a == 0 && js == 0)  // diagonals 7-12 start from zero
                tc::mma_bf16(d + kTcPlanes * kTcrI, adesc, tc::smem_desc(Zt, 128, 256), id_zero, 0u);
            }
            tc::commit(&sh.b_empty[b]);
          }
          __syncwarp();
        }
        if (!ok) break;
        if (lane == 0) tc::commit(&sh.acc_full[set]);
        __syncwarp();
      }
      if (!ok) break;
      for (u32 js = 0; js < nS; ++js) ++acnt[js];
      if (lane == 0) tc::commit(&sh.a_free);  // the unit's digit planes may be overwritten
      __syncwarp();
    }
    if (lane == 0) tc::commit(&sh.done);  // every MMA issued has completed once this arrives
    __syncwarp();
    mbar_wait_warp(&sh.done, 0, kWaitLimitNs);
  } else if (warp < kTcrEpi0) {
    // ---------------------------------------------------------------- input digit planes
    const u32 sw = warp - 2;  // split warp: rows 32 sw .. 32 sw + 31, both octets of 8 k-blocks
    u32 rc = 0, unit = 0;
    bool ok = true;
    for (u64 g = blockIdx.x; ok && g < total && !*abort_flag; g += gridDim.x, ++unit) {
      TcrWork w;
      get(g, w);
      const u32 nS = tc_stages(w.nJ), nc = min(kTcrM, w.R - w.r0);
      if (unit > 0 && !mbar_wait_warp(&sh.a_free, (unit - 1) & 1, kWaitLimitNs)) {  // the last unit's MMAs are done
        give_up();
        ok = false;
        break;
      }
      for (u32 js = 0; js < nS; ++js, ++rc) {
        const u32 b = rc % kTcrRawStages, jb = min(kTcJB, w.nJ - js * kTcJB);
        if (!mbar_wait_warp(&sh.raw_full[b], (rc / kTcrRawStages) & 1, kWaitLimitNs)) {
          give_up();
          ok = false;
          break;
        }
        uint8_t* const dst = Ad + js * kTcrABytes;
#pragma unroll
        for (u32 o = 0; o < 2; ++o) {
          const u32 row = 32 * sw + lane;
          if (row < nc) {
            const uint8_t* src = Raw + b * kTcrRawBytes + row * kTcRawRow;
            u64 u[8];
#pragma unroll
            for (int h = 0; h < 4; ++h) {  // chunk 4 o + h of the row sits at position (4 o + h + row) mod 8
              const uint4 x = *reinterpret_cast<const uint4*>(src + 16 * ((4 * o + h + row) & 7));
              u[2 * h] = (u64)x.x | ((u64)x.y << 32);
              u[2 * h + 1] = (u64)x.z | ((u64)x.w << 32);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              if (8 * o + k >= jb) u[k] = 0;  // k-blocks past the product's last: zero digits
              u[k] += 0x0080808080808080ull;
            }
#pragma unroll
            for (int p = 0; p < (int)kTcPlanes; ++p)
              *reinterpret_cast<uint4*>(dst + p * kTcrPlaneBytes + tc::tile_offset(row, 8 * o, kTcJB * 2, 2)) =
                  digit_plane(u, p);
          }
        }
        tc::fence_smem_to_async();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&sh.raw_empty[b]);
          mbar_arrive(&sh.a_full[js]);
        }
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const u32 q = warp & 3;                    // TMEM lane quadrant: input rows 32 q .. 32 q + 31
    const u32 ih = (warp - kTcrEpi0) >> 2;     // weight rows 8 ih .. 8 ih + 7 of each tile
    u32 rnd = 0;
    bool ok = true;
    for (u64 g = blockIdx.x; ok && g < total && !*abort_flag; g += gridDim.x) {
      TcrWork w;
      get(g, w);
      const u32 nIt = tcr_tiles_I(w.nI);
      const PrimeConsts P = C.p[w.l];
      u32 clo[kTcDiag], chi[kTcDiag];  // 256^d mod q_l in 32-bit halves
#pragma unroll
      for (u32 d = 0; d < kTcDiag; ++d) {
        clo[d] = P.pw256_lo[d];
        chi[d] = P.pw256_hi[d];
      }
      const u32 row = w.r0 + 32 * q + lane, G = 1u << w.logG;
      const bool row_ok = row < w.R;
      const u32 rcomp = row >> w.logG, gco = row & (G - 1);
      const bool small = w.nJ <= 2 * kTcJB;  // |D_d| <= 7 * 32 * 2^14 < 2^22
      for (u32 t = 0; t < nIt; ++t, ++rnd) {
        const u32 set = rnd & 1;
        if (!mbar_wait_warp(&sh.acc_full[set], (rnd >> 1) & 1, kWaitLimitNs)) {
          give_up();
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const u32 I0 = t * kTcrI + 8 * ih;
        const bool live = w.r0 + 32 * q < w.R && I0 < w.nI;
        const uint32_t tbase = tmem + set * kTcSetCols + ((32 * q) << 16);
#pragma unroll
        for (u32 h4 = 0; h4 < 2; ++h4) {
          if (!live) break;
          uint32_t v[13][4];
#pragma unroll
          for (u32 d = 0; d < kTcDiag; ++d) tc::ld_32x32b_x4(tbase + d * kTcrI + 8 * ih + 4 * h4, v[d]);
          tc::wait_ld();
          u64 x[4];
          if (small) tc_combine4<true>(v, clo, chi, P, x);
          else tc_combine4<false>(v, clo, chi, P, x);
          if (row_ok) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const u32 I = I0 + 4 * h4 + r;
              if (I < w.nI)
                w.acc[(((w.ct0 + (u64)(rcomp >> 1) * w.nI + I) * 2 + (rcomp & 1)) * C.L + w.l) * (2ull * N) +
                      (u64)gco * w.S + w.s] = x[r];
            }
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.acc_empty[set]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTcCols);
  }
}

}  // namespace he
