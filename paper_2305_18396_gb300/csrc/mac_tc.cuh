// mac_tc.cuh -- the slot-wise multiply-accumulate of Algorithm 1 step 3 (NTT domain) on the
// tcgen05 tensor cores, exact.
//
// For prime l and slot s the outputs of a product form a small matrix product over the
// k-blocks J:  out[r][I] = sum_J ct[r][J] * pt[I][J]  (mod q_l),  r = (Lb, component) rows,
// I = weight-block columns, values < q_l < 2^50.
//
// Exact split.  Every residue v is written in balanced base-256 digits,
//   v = sum_{a<7} d_a 256^a,  d_a in [-128, 127]  (the bytes of v + 0x0080808080808080,
//   each minus 128),
// and each digit is exact in bf16.  With A_a the digit planes of the weights and B_b those
// of the ciphertext rows, out = sum_{a,b} 256^(a+b) sum_J A_a[I][J] B_b[r][J].  Products of
// digits are at most 2^14 in magnitude and a diagonal a + b = d collects at most 7 of them
// per k-block, so its f32 sum over 128 k-blocks stays below 7 * 128 * 2^14 < 2^24: every
// partial sum is an exact integer.  After each round of 128 k-blocks the 13 diagonal sums
// are converted to integers, combined with their powers of 256 and reduced mod q_l.
//
// Diagonal folding.  The B planes of one stage are stacked along the MMA's N dimension,
// row b * 16 + r for plane b and ciphertext row r (N = 112), and the MMA of weight plane a
// (M = 128 weight rows, K = 16 k-blocks) writes TMEM columns a * 16 + (b * 16 + r): the
// accumulator of diagonal d sits at columns d * 16 .. d * 16 + 15 (13 x 16 = 208 columns),
// and each MMA adds its plane products onto the right diagonals.  7 MMAs per stage of 16
// k-blocks; the first stage of a round overwrites (diagonals 0-6 by plane 0, diagonals 7-12
// by an MMA against a zero tile).
//
// Operand layout ("stage-tiled"): plain residues (no split); for prime l, slot s and stage
// js (k-blocks 16 js .. 16 js + 15) the 16 words of every operand row (weight block I,
// resp. input row (Lb, c)) are 128 contiguous bytes, rows back to back:
//   word ((((l N + s) nS + js) rows + row) 16 + chunk 2 + (J & 1),
//   chunk = ((J & 15) / 2 + row) mod 8   (the 16-byte chunks rotated by the row),
// nS = ceil(nJ / 16) stages, `rows` = nI for the weights and 2 nLb for the inputs.  A stage
// of a block's 128 weight rows (16 ciphertext rows) is then one contiguous 16 KB (2 KB)
// bulk copy, and the rotation keeps the digit split's shared-memory reads free of bank
// conflicts.  A block works on kTcSlots consecutive slots of one prime, one tile of 128
// weight rows and one tile of 16 ciphertext rows; per stage a producer warp copies the two
// tiles into shared memory, four warps split them into digit planes (bf16, the K-major
// no-swizzle layout of tcgen05.cuh), one thread issues the MMAs, and the same four warps
// read the accumulators back after each round.
#pragma once

#include <cuda_bf16.h>

#include "async.cuh"
#include "he_common.cuh"
#include "mac.cuh"
#include "tcgen05.cuh"

namespace he {

constexpr u32 kTcM = 128;        // weight rows per block (MMA M)
constexpr u32 kTcR = 16;         // ciphertext rows per block
constexpr u32 kTcPlanes = 7;     // balanced base-256 digits of a 50-bit residue
constexpr u32 kTcDiag = 13;      // diagonals a + b
constexpr u32 kTcJB = 16;        // k-blocks per stage (one MMA K step)
constexpr u32 kTcRound = 8;      // stages per exact accumulation round (128 k-blocks)
constexpr u32 kTcSlots = 4;      // consecutive slots per block
constexpr u32 kTcThreads = 192;  // warp 0 producer, warp 1 MMA, warps 2-5 digits + epilogue
constexpr u32 kTcCols = 256;     // TMEM columns per block (208 used); two blocks per SM
constexpr u32 kTcRawRow = kTcJB * 8;                          // bytes per staged operand row
constexpr u32 kTcRawBytes = (kTcM + kTcR) * kTcRawRow;        // one raw stage
constexpr u32 kTcAKBytes = kTcPlanes * kTcJB * 2;             // K bytes per weight row (7 planes)
constexpr u32 kTcABytes = kTcM * kTcAKBytes;                  // weight digit tile
constexpr u32 kTcBBytes = kTcPlanes * kTcR * kTcJB * 2;       // ciphertext digit tile (112 rows)
constexpr u32 kTcZBytes = (kTcDiag - kTcPlanes) * kTcR * kTcJB * 2;  // zero tile (96 rows)
constexpr u32 kTcSmem = 2 * kTcRawBytes + 2 * kTcABytes + 2 * kTcBBytes + kTcZBytes + 128;

// Stages of 16 k-blocks per slot, and words of an operand with `rows` rows in the
// stage-tiled layout (all primes and slots).
__host__ __device__ constexpr u32 tc_stages(u32 nJ) { return (nJ + kTcJB - 1) / kTcJB; }
__host__ __device__ constexpr u64 tc_words(u32 rows, u32 nJ, u32 L, u32 N) {
  return (u64)L * N * tc_stages(nJ) * rows * kTcJB;
}

__host__ __device__ constexpr u64 tc_index(u32 row, u32 J, u32 l, u32 s, u32 rows, u32 nS, u32 N) {
  return ((((u64)l * N + s) * nS + (J >> 4)) * rows + row) * kTcJB + ((((J & 15) >> 1) + row) & 7) * 2 + (J & 1);
}

// x mod q for a signed 64-bit x (|x| < 2^63).
__device__ __forceinline__ u64 smod(long long x, const PrimeConsts& P) {
  const u64 m = reduce_word(x < 0 ? (u64)(-x) : (u64)x, P);
  return (x < 0 && m) ? P.q - m : m;
}

__device__ __forceinline__ int f32_to_s32(uint32_t bits) {
  int r;
  asm("cvt.rni.s32.f32 %0, %1;" : "=r"(r) : "f"(__uint_as_float(bits)));
  return r;
}

// Digit plane p of the 8 residues w[0..7] as 8 bf16 (16 bytes): byte p of w + 0x0080808080808080,
// placed into the float 2^23 + byte (one byte permute), minus 2^23 + 128.
__device__ __forceinline__ uint4 digit_plane(const u64 (&u)[8], int p) {
  uint32_t h[4];
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    const uint32_t src0 = p < 4 ? (uint32_t)u[j] : (uint32_t)(u[j] >> 32);
    const uint32_t src1 = p < 4 ? (uint32_t)u[j + 1] : (uint32_t)(u[j + 1] >> 32);
    const uint32_t sel = 0x7440u | (uint32_t)(p & 3);
    const float f0 = __uint_as_float(__byte_perm(src0, 0x4B000000u, sel)) - 8388736.0f;
    const float f1 = __uint_as_float(__byte_perm(src1, 0x4B000000u, sel)) - 8388736.0f;
    __nv_bfloat162 b = __floats2bfloat162_rn(f0, f1);
    h[j >> 1] = *reinterpret_cast<uint32_t*>(&b);
  }
  return make_uint4(h[0], h[1], h[2], h[3]);
}

struct TcShared {
  uint64_t raw_full[2], raw_empty[2], limb_full[2], limb_empty[2], acc_full, acc_empty, done;
  uint32_t tmem;
  int abort;
};

// One block: slots s0 .. s0 + nslots - 1 of prime l, weight rows I0 .. I0 + 127 and output
// rows r0 .. r0 + 15 of one product.  ct0: index of the product's first output ciphertext
// in `out`.  smem: the caller's dynamic buffer of kTcSmem bytes (128-byte aligned).
__device__ __forceinline__ void mac_tc_block(const u64* __restrict__ ctN, const u64* __restrict__ pt,
                                             const OutPlace& out, u64 ct0, u32 nI, u32 nJ, u32 nLb, u32 I0, u32 r0,
                                             u32 s0, u32 nslots, u32 l, int* err, const Consts& C, uint8_t* smem,
                                             TcShared& sh) {
  // stage b: raw rows at raw0 + b kTcRawBytes, digit tiles at At0 + b kTcABytes, Bt0 + b kTcBBytes
  uint8_t* const raw0 = smem;
  uint8_t* const At0 = smem + 2 * kTcRawBytes;
  uint8_t* const Bt0 = At0 + 2 * kTcABytes;
  uint8_t* const Zt = Bt0 + 2 * kTcBBytes;
  const u32 warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 N = C.N, L = C.L;
  const PrimeConsts& P = C.p[l];
  const u32 R = 2 * nLb;
  const u32 nw = min(kTcM, nI - I0), nc = min(kTcR, R - r0);
  const u32 sps = tc_stages(nJ);  // stages per slot
  const u32 total = sps * nslots;

  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh.raw_full[b], 1);
      mbar_init(&sh.raw_empty[b], 4);
      mbar_init(&sh.limb_full[b], 4);
      mbar_init(&sh.limb_empty[b], 1);
    }
    mbar_init(&sh.acc_full, 1);
    mbar_init(&sh.acc_empty, 4);
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
    u32 issued = 0;
    for (u32 i = 0; i < total && !*abort_flag; ++i) {
      const u32 b = i & 1;
      if (i >= 2 && !mbar_wait_warp(&sh.raw_empty[b], ((i >> 1) - 1) & 1, kWaitLimitNs)) {
        give_up();
        break;
      }
      const u32 s = s0 + i / sps, J0 = (i % sps) * kTcJB;
      if (lane == 0) {  // two bulk copies: the block's weight rows and its ciphertext rows of this stage
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&sh.raw_full[b], (nw + nc) * kTcRawRow);
        bulk_copy_g2s(raw0 + b * kTcRawBytes, pt + tc_index(I0, J0, l, s, nI, sps, N), nw * kTcRawRow,
                      &sh.raw_full[b]);
        bulk_copy_g2s(raw0 + b * kTcRawBytes + kTcM * kTcRawRow, ctN + tc_index(r0, J0, l, s, R, sps, N),
                      nc * kTcRawRow, &sh.raw_full[b]);
      }
      __syncwarp();
      issued = i + 1;
    }
    // copies still in flight must land before the block's shared memory is released
    for (u32 i = issued > 2 ? issued - 2 : 0; i < issued; ++i)
      mbar_wait_warp(&sh.raw_full[i & 1], (i >> 1) & 1, kWaitLimitNs);
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issue
    const uint32_t id_main = tc::idesc_bf16_f32(kTcM, kTcPlanes * kTcR);
    const uint32_t id_zero = tc::idesc_bf16_f32(kTcM, (kTcDiag - kTcPlanes) * kTcR);
    u32 round = 0;
    for (u32 i = 0; i < total && !*abort_flag; ++i) {
      const u32 b = i & 1, j = i % sps;
      const bool first = (j % kTcRound) == 0, last = (j == sps - 1) || ((j + 1) % kTcRound == 0);
      if (first && round > 0 && !mbar_wait_warp(&sh.acc_empty, (round - 1) & 1, kWaitLimitNs)) {
        give_up();
        break;
      }
      if (!mbar_wait_warp(&sh.limb_full[b], (i >> 1) & 1, kWaitLimitNs)) {
        give_up();
        break;
      }
      tc::fence_after_sync();
      if (lane == 0) {
        const uint64_t bdesc = tc::smem_desc(Bt0 + b * kTcBBytes, 128, 256);
#pragma unroll
        for (u32 a = 0; a < kTcPlanes; ++a) {
          const uint64_t adesc = tc::smem_desc(At0 + b * kTcABytes + a * 256, 128, 8 * kTcAKBytes);
          tc::mma_bf16(tmem + a * kTcR, adesc, bdesc, id_main, (a > 0 || !first) ? 1u : 0u);
          if (a == 0 && first)
            tc::mma_bf16(tmem + kTcPlanes * kTcR, adesc, tc::smem_desc(Zt, 128, 256), id_zero, 0u);
        }
        tc::commit(&sh.limb_empty[b]);
        if (last) tc::commit(&sh.acc_full);
      }
      __syncwarp();
      if (last) ++round;
    }
    if (lane == 0) tc::commit(&sh.done);  // every MMA issued has completed once this arrives
    __syncwarp();
    mbar_wait_warp(&sh.done, 0, kWaitLimitNs);
  } else {
    // ---------------------------------------------------------------- digits + epilogue
    const u32 e = threadIdx.x - 64;          // 0 .. 127
    const u32 q = warp & 3;                  // TMEM lane quadrant this warp may read
    const u32 I = 32 * q + lane;             // weight row (TMEM lane) of this thread's outputs
    u64 acc[kTcR];
#pragma unroll
    for (u32 r = 0; r < kTcR; ++r) acc[r] = 0;
    u32 round = 0;
    for (u32 i = 0; i < total && !*abort_flag; ++i) {
      const u32 b = i & 1, j = i % sps, J0 = j * kTcJB;
      const u32 jb = min(kTcJB, nJ - J0);
      const bool last = (j == sps - 1) || ((j + 1) % kTcRound == 0);
      if (!mbar_wait_warp(&sh.raw_full[b], (i >> 1) & 1, kWaitLimitNs) ||
          (i >= 2 && !mbar_wait_warp(&sh.limb_empty[b], ((i >> 1) - 1) & 1, kWaitLimitNs))) {
        give_up();
        break;
      }
      // items: (weight row, octet of 8 k-blocks) then (ciphertext row, octet)
      for (u32 t = e; t < 2 * (kTcM + kTcR); t += 128) {
        const bool wrow = t < 2 * kTcM;
        const u32 row = wrow ? (t & (kTcM - 1)) : ((t - 2 * kTcM) & (kTcR - 1));
        const u32 o = wrow ? (t >> 7) : ((t - 2 * kTcM) >> 4);
        if (row >= (wrow ? nw : nc)) continue;  // padding rows only feed outputs nobody stores
        const uint8_t* src = raw0 + b * kTcRawBytes + (wrow ? row : kTcM + row) * kTcRawRow;
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
        for (int p = 0; p < (int)kTcPlanes; ++p) {
          const uint4 v = digit_plane(u, p);
          uint8_t* dst = wrow ? At0 + b * kTcABytes + tc::tile_offset(row, p * kTcJB + 8 * o, kTcAKBytes, 2)
                              : Bt0 + b * kTcBBytes + tc::tile_offset(p * kTcR + row, 8 * o, kTcJB * 2, 2);
          *reinterpret_cast<uint4*>(dst) = v;
        }
      }
      tc::fence_smem_to_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&sh.raw_empty[b]);
        mbar_arrive(&sh.limb_full[b]);
      }
      if (!last) continue;
      // ---- epilogue of a round: 13 diagonal sums per output -> exact integer -> mod q
      if (!mbar_wait_warp(&sh.acc_full, round & 1, kWaitLimitNs)) {
        give_up();
        break;
      }
      ++round;
      tc::fence_after_sync();
      const uint32_t tbase = tmem + ((32 * q) << 16);
#pragma unroll
      for (u32 hh = 0; hh < 2; ++hh) {  // output rows 8 hh .. 8 hh + 7
        u64 part[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) part[r] = 0;
#pragma unroll
        for (u32 g = 0; g < 3; ++g) {  // diagonals 0-3, 4-7, 8-12: weights 1, 2^32, 2^64
          const u32 d0 = 4 * g, nd = g == 2 ? 5 : 4;
          uint32_t v[5][8];
#pragma unroll
          for (u32 dd = 0; dd < nd; ++dd) tc::ld_32x32b_x8(tbase + (d0 + dd) * kTcR + 8 * hh, v[dd]);
          tc::wait_ld();
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            long long G = 0;
#pragma unroll
            for (u32 dd = 0; dd < nd; ++dd) G += (long long)f32_to_s32(v[dd][r]) << (8 * dd);
            const u64 gm = smod(G, P);
            const u64 w = g == 0 ? gm
                        : g == 1 ? csub(mul_shoup(gm, P.r32, P.r32_sh, P.q), P.q)
                                 : csub(mul_shoup(gm, P.r64, P.r64_sh, P.q), P.q);
            part[r] = add_mod(part[r], w, P.q);
          }
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[8 * hh + r] = add_mod(acc[8 * hh + r], part[r], P.q);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.acc_empty);
      if (j == sps - 1) {  // the slot is complete: store its outputs, restart the sums
        const u32 s = s0 + i / sps;
        if (I0 + I < nI) {
#pragma unroll
          for (u32 r = 0; r < kTcR; ++r) {
            const u32 row = r0 + r;
            if (row < R) {
              const u32 c = row & 1;
              out.base[c][(ct0 + (u64)(row >> 1) * nI + I0 + I) * out.ct_stride[c] + (u64)l * N + s] = acc[r];
            }
          }
        }
#pragma unroll
        for (u32 r = 0; r < kTcR; ++r) acc[r] = 0;
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

// Work units of one product in the tensor-core grid: ciphertext-row tiles fastest, then
// weight-row tiles, then groups of kTcSlots slots, then primes -- the units that share a
// slot's operands run together and re-read them from L2.
struct TcUnit {
  u32 I0, r0, s0, l;
};

__host__ __device__ inline u32 tc_tiles_I(u32 nI) { return (nI + kTcM - 1) / kTcM; }
__host__ __device__ inline u32 tc_tiles_R(u32 nLb) { return (2 * nLb + kTcR - 1) / kTcR; }
__host__ __device__ inline u64 tc_units(u32 N, u32 L, u32 nI, u32 nLb) {
  return (u64)L * (N / kTcSlots) * tc_tiles_I(nI) * tc_tiles_R(nLb);
}

__device__ __forceinline__ TcUnit tc_unit(u64 u, u32 N, u32 nI, u32 nLb) {
  const u32 nRt = tc_tiles_R(nLb), nIt = tc_tiles_I(nI);
  TcUnit t;
  t.r0 = (u32)(u % nRt) * kTcR;
  u /= nRt;
  t.I0 = (u32)(u % nIt) * kTcM;
  u /= nIt;
  t.s0 = (u32)(u % (N / kTcSlots)) * kTcSlots;
  t.l = (u32)(u / (N / kTcSlots));
  return t;
}

}  // namespace he
