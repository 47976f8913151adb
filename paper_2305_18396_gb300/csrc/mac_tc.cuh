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
// Operand layouts.  The encoded weights are stored split, as the bf16 digit planes the MMAs
// read ("digit tiles"): for prime l, slot s and stage js (k-blocks 16 js .. 16 js + 15) all
// weight rows I form one K-major no-swizzle tile of K = 7 planes x 16 k-blocks (element
// (I, 16 p + j) at tc::tile_offset(I, 16 p + j, 224, 2)), tiles back to back in (l, s, js)
// order, k-blocks past the product's last zero.  A work unit's 128 weight rows of a stage
// are then one contiguous bulk copy straight into the MMA's operand buffer, with no split
// on the SM (the weights are resident and encoded once; their digit form costs 14 bytes
// per residue instead of 8).  The NTT of the input ciphertexts keeps plain residues
// ("stage-tiled"): for prime l, slot s and stage js the 16 words of every input row
// (Lb, c) are 128 contiguous bytes, rows back to back,
//   word ((((l N + s) nS + js) rows + row) 16 + chunk 2 + (J & 1),
//   chunk = ((J & 15) / 2 + row) mod 8   (the 16-byte chunks rotated by the row),
// nS = ceil(nJ / 16), rows = 2 nLb (2 nLb G rows and 2D slots per prime for coset products,
// coset.cuh); two warps split a unit's 16 input rows into digit planes per stage (planes
// 0-3 and 4-6; the rotation keeps their shared-memory reads free of bank conflicts).
// A work unit is kTcSlots consecutive slots of one prime, one tile of 128 weight rows and
// one tile of 16 input rows; per stage a producer warp issues the two bulk copies, the two
// split warps convert the input rows, one thread issues the MMAs, and eight warps (two per
// TMEM lane quadrant, 8 output rows each) read the accumulators back after each round while
// the MMAs of the next round fill the other of two accumulator sets.  One block per SM
// works through its share of the launch's work units back to back, so the pipeline never
// drains between units.  Coset products of at most 64 k-blocks take mac_tcr.cuh instead.
#pragma once

#include <cuda_bf16.h>

#include "async.cuh"
#include "he_common.cuh"
#include "mac.cuh"
#include "tcgen05.cuh"

namespace he {

constexpr u32 kTcM = 128;          // weight rows per work unit (MMA M)
constexpr u32 kTcR = 16;           // ciphertext rows per work unit
constexpr u32 kTcPlanes = 7;       // balanced base-256 digits of a 50-bit residue
constexpr u32 kTcDiag = 13;        // diagonals a + b
constexpr u32 kTcJB = 16;          // k-blocks per stage (one MMA K step)
constexpr u32 kTcRound = 8;        // stages per exact accumulation round (128 k-blocks)
constexpr u32 kTcSlots = 4;        // consecutive slots per work unit (measured: 2.5% faster than 8 on the coset FC products, 16 slower)
constexpr u32 kTcStages = 6;       // stages in flight: 225 KB of shared memory (coset products, operands from L2: 2.4% faster than 4)
constexpr u32 kTcSplitWarps = 2;   // digit split of the input rows: planes 0-3 and 4-6
constexpr u32 kTcEpi0 = 2 + kTcSplitWarps;  // first epilogue warp
constexpr u32 kTcEpiWarps = 8;     // epilogue: two per TMEM lane quadrant (warp w reads quadrant w mod 4), 8 rows each
constexpr u32 kTcThreads = 32 * (kTcEpi0 + kTcEpiWarps);  // producer, MMA, digit split, epilogue: 384
constexpr u32 kTcCols = 512;       // TMEM: two accumulator sets of 13 x 16 columns, at 0 and 256
constexpr u32 kTcSetCols = 256;
constexpr u32 kTcRawRow = kTcJB * 8;                          // bytes per staged input row
constexpr u32 kTcRawBytes = kTcR * kTcRawRow;                 // one stage of input rows
constexpr u32 kTcAKBytes = kTcPlanes * kTcJB * 2;             // K bytes per weight row (7 planes)
constexpr u32 kTcGroupBytes = 8 * kTcAKBytes;                 // one 8-row group of a digit tile
constexpr u32 kTcABytes = kTcM * kTcAKBytes;                  // weight digit tile of a unit
constexpr u32 kTcBBytes = kTcPlanes * kTcR * kTcJB * 2;       // input digit tile (112 rows)
constexpr u32 kTcZBytes = (kTcDiag - kTcPlanes) * kTcR * kTcJB * 2;  // zero tile (96 rows)
constexpr u32 kTcAccBytes = kTcR * kTcM * 8;                // the epilogue's running sums mod q
constexpr u32 kTcStageBytes = kTcABytes + kTcRawBytes + kTcBBytes;
constexpr u32 kTcSmem = kTcStages * kTcStageBytes + kTcZBytes + kTcAccBytes + 128;
static_assert(kTcSmem <= 227 * 1024, "tensor-core MAC shared memory above the per-block limit");

// Stages of 16 k-blocks per slot; words of the inputs' NTT (`rows` rows, stage-tiled) and of
// the weights' digit tiles (nI rows) for all primes and slots.
__host__ __device__ constexpr u32 tc_stages(u32 nJ) { return (nJ + kTcJB - 1) / kTcJB; }
__host__ __device__ constexpr u64 tc_words(u32 rows, u32 nJ, u32 L, u32 N) {
  return (u64)L * N * tc_stages(nJ) * rows * kTcJB;
}
__host__ __device__ constexpr u64 tc_weight_words(u32 nI, u32 nJ, u32 L, u32 N) {
  return (u64)L * N * tc_stages(nJ) * ((nI + 7) / 8) * kTcGroupBytes / 8;
}

__host__ __device__ constexpr u64 tc_index(u32 row, u32 J, u32 l, u32 s, u32 rows, u32 nS, u32 N) {
  return ((((u64)l * N + s) * nS + (J >> 4)) * rows + row) * kTcJB + ((((J & 15) >> 1) + row) & 7) * 2 + (J & 1);
}

// Byte offset of the digit-tile group (8 weight rows from I0, a multiple of 8) of prime l,
// slot s and stage js; digit p of k-block j of row I0 + i sits at that offset plus
// tc::tile_offset(i, 16 p + j, 224, 2).
__host__ __device__ constexpr u64 tc_weight_offset(u32 I0, u32 l, u32 s, u32 js, u32 nI, u32 nS, u32 N) {
  return ((((u64)l * N + s) * nS + js) * ((nI + 7) / 8) + (I0 >> 3)) * kTcGroupBytes;
}

__device__ __forceinline__ int f32_to_s32(uint32_t bits) {
  int r;
  asm("cvt.rni.s32.f32 %0, %1;" : "=r"(r) : "f"(__uint_as_float(bits)));
  return r;
}

// The same for an exact integer of magnitude at most 2^22, on the add pipes instead of the
// conversion unit: x + 1.5 2^23 lies in [2^23, 2^24], where floats are the integers, so its
// bits are 0x4B400000 + x.
__device__ __forceinline__ int f32_small_to_s32(uint32_t bits) {
  return (int)(__float_as_uint(__fadd_rn(__uint_as_float(bits), 12582912.0f)) - 0x4B400000u);
}

// sum_d D_d 256^d mod q, less 2^24 sum_d 256^d, for four outputs (TMEM words v[d][r], exact
// f32 integers, |D_d| < 2^24; SMALL: |D_d| <= 2^22).  With D_d + 2^24 in [0, 2^25) and
// 256^d mod q = lo_d + 2^32 hi_d (hi_d = 0 below d = 4), A = sum (D_d + 2^24) lo_d < 2^61 and
// B = sum (D_d + 2^24) hi_d < 2^47 take one mad.wide each per diagonal, in two chains each
// (even and odd d) for instruction-level parallelism; A + 2^32 B is reduced once.
template <bool SMALL>
__device__ __forceinline__ void tc_combine4(const uint32_t (&v)[13][4], const u32 (&clo)[13], const u32 (&chi)[13],
                                            const PrimeConsts& P, u64 (&x)[4]) {
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    u64 A0 = 0, A1 = 0, B0 = 0, B1 = 0;
#pragma unroll
    for (int d = 0; d < 13; ++d) {
      const uint32_t D = (uint32_t)((SMALL ? f32_small_to_s32(v[d][r]) : f32_to_s32(v[d][r])) + (1 << 24));
      mad_wide(d & 1 ? A1 : A0, D, clo[d]);
      if (d >= 4) mad_wide(d & 1 ? B1 : B0, D, chi[d]);
    }
    const u64 y = reduce_word(A0 + A1, P) + csub(mul_shoup(B0 + B1, P.r32, P.r32_sh, P.q), P.q);  // [0, 2q)
    x[r] = sub_mod(csub(y, P.q), P.pw256_bias, P.q);
  }
}

// Digit p of u = v + 0x0080808080808080 (v < 2^50) as the bits of an exact f32: byte p of u
// placed into the float 2^23 + byte (one byte permute), minus 2^23 + 128.  Its bf16 is the
// high half of those bits (the digit has at most 8 significant bits).
__device__ __forceinline__ uint32_t digit_f32_bits(u64 u, int p) {
  const uint32_t src = p < 4 ? (uint32_t)u : (uint32_t)(u >> 32);
  return __float_as_uint(__uint_as_float(__byte_perm(src, 0x4B000000u, 0x7440u | (uint32_t)(p & 3))) - 8388736.0f);
}

// Digit plane p of the 8 offset residues u[0..7] as 8 bf16 (16 bytes).
__device__ __forceinline__ uint4 digit_plane(const u64 (&u)[8], int p) {
  uint32_t h[4];
#pragma unroll
  for (int j = 0; j < 8; j += 2) h[j >> 1] = __byte_perm(digit_f32_bits(u[j], p), digit_f32_bits(u[j + 1], p), 0x7632u);
  return make_uint4(h[0], h[1], h[2], h[3]);
}

struct TcShared {
  uint64_t full[kTcStages], conv[kTcStages], empty[kTcStages];
  uint64_t acc_full[2], acc_empty[2], done;
  uint32_t tmem;
  int abort;
};

// One work unit: slots s0 .. s0 + kTcSlots - 1 of prime l, weight rows I0 .. I0 + 127 and output
// rows r0 .. r0 + 15 of one product (input NTT ctN, weight digit tiles ptd; outputs `out`, the
// product's first output ciphertext at index ct0).
//
// Coset products (coset.cuh): each prime has S = 2D slots instead of N and the operand rows
// are (Lb, component, coset g), row = (2 Lb + c) G + g (R = 2 nLb G rows); acc != nullptr
// then receives the sums, output ciphertext o, component c, prime l at
// acc + ((o 2 + c) L + l) 2N + g S + s.
struct TcWork {
  const u64* ctN;
  const uint8_t* ptd;
  OutPlace out;
  u64* acc;
  u64 ct0;
  u32 nI, nJ, nLb, I0, r0, s0, l;
  u32 S, R, logG;  // slots per prime, operand rows, log2 of the cosets (coset products)
};

// Work units of one product: ciphertext-row tiles fastest, then weight-row tiles, then groups
// of kTcSlots slots, then primes -- the units that share a slot's operands run together and
// re-read them from L2.
// S slots per prime, R operand rows (2 nLb, or 2 nLb G for coset products).
__host__ __device__ inline u32 tc_tiles_I(u32 nI) { return (nI + kTcM - 1) / kTcM; }
__host__ __device__ inline u32 tc_tiles_R(u32 R) { return (R + kTcR - 1) / kTcR; }
__host__ __device__ inline u64 tc_units(u32 S, u32 L, u32 nI, u32 R) {
  return (u64)L * (S / kTcSlots) * tc_tiles_I(nI) * tc_tiles_R(R);
}

__device__ __forceinline__ void tc_unit(u64 u, u32 S, u32 nI, u32 R, TcWork& w) {
  const u32 nRt = tc_tiles_R(R), nIt = tc_tiles_I(nI);
  w.r0 = (u32)(u % nRt) * kTcR;
  u /= nRt;
  w.I0 = (u32)(u % nIt) * kTcM;
  u /= nIt;
  w.s0 = (u32)(u % (S / kTcSlots)) * kTcSlots;
  w.l = (u32)(u / (S / kTcSlots));
  w.S = S;
  w.R = R;
}

// One block per SM: work units blockIdx.x, blockIdx.x + gridDim.x, ... < total, each unit
// described by get(g, w) (the same sequence for every role).  smem: the caller's dynamic
// buffer of kTcSmem bytes (128-byte aligned).
template <class GetWork>
__device__ __forceinline__ void mac_tc_run(const GetWork& get, u64 total, int* err, const Consts& C, uint8_t* smem,
                                           TcShared& sh) {
  // stage b: weight digit tile at st0 + b kTcStageBytes, then the raw input rows, then the
  // input digit tile
  uint8_t* const st0 = smem;
  uint8_t* const Zt = smem + kTcStages * kTcStageBytes;
  u64* const accs = reinterpret_cast<u64*>(Zt + kTcZBytes);  // [output row r][epilogue thread]
  const u32 warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const u32 N = C.N;

  if (threadIdx.x == 0) {
    for (u32 b = 0; b < kTcStages; ++b) {
      mbar_init(&sh.full[b], 1);
      mbar_init(&sh.conv[b], kTcSplitWarps);
      mbar_init(&sh.empty[b], 1);
    }
    for (u32 b = 0; b < 2; ++b) {
      mbar_init(&sh.acc_full[b], 1);
      mbar_init(&sh.acc_empty[b], kTcEpiWarps);
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
    u32 i = 0;
    bool ok = true;
    for (u64 g = blockIdx.x; ok && g < total && !*abort_flag; g += gridDim.x) {
      TcWork w;
      get(g, w);
      const u32 sps = tc_stages(w.nJ), R = w.R;
      const u32 nw = min(kTcM, w.nI - w.I0), nc = min(kTcR, R - w.r0);
      for (u32 st = 0; st < kTcSlots * sps; ++st, ++i) {
        const u32 b = i % kTcStages;
        if (i >= kTcStages && !mbar_wait_warp(&sh.empty[b], ((i / kTcStages) - 1) & 1, kWaitLimitNs)) {
          give_up();
          ok = false;
          break;
        }
        const u32 s = w.s0 + st / sps, js = st % sps;
        if (lane == 0) {  // two bulk copies: the unit's weight digit rows and its raw input rows
          uint8_t* dst = st0 + b * kTcStageBytes;
          const u32 abytes = ((nw + 7) / 8) * kTcGroupBytes;
          fence_proxy_async_smem();
          mbar_arrive_expect_tx(&sh.full[b], abytes + nc * kTcRawRow);
          bulk_copy_g2s(dst, w.ptd + tc_weight_offset(w.I0, w.l, s, js, w.nI, sps, w.S), abytes, &sh.full[b]);
          bulk_copy_g2s(dst + kTcABytes, w.ctN + tc_index(w.r0, js * kTcJB, w.l, s, R, sps, w.S), nc * kTcRawRow,
                        &sh.full[b]);
        }
        __syncwarp();
      }
    }
    // copies still in flight must land before the block's shared memory is released
    for (u32 k = i > kTcStages ? i - kTcStages : 0; k < i; ++k)
      mbar_wait_warp(&sh.full[k % kTcStages], (k / kTcStages) & 1, kWaitLimitNs);
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issue
    const uint32_t id_main = tc::idesc_bf16_f32(kTcM, kTcPlanes * kTcR);
    const uint32_t id_zero = tc::idesc_bf16_f32(kTcM, (kTcDiag - kTcPlanes) * kTcR);
    u32 i = 0, round = 0;
    bool ok = true;
    for (u64 g = blockIdx.x; ok && g < total && !*abort_flag; g += gridDim.x) {
      TcWork w;
      get(g, w);
      const u32 sps = tc_stages(w.nJ);
      for (u32 st = 0; st < kTcSlots * sps; ++st, ++i) {
        const u32 j = st % sps, set = round & 1, b = i % kTcStages;
        const bool first = (j % kTcRound) == 0, last = (j == sps - 1) || ((j + 1) % kTcRound == 0);
        if ((first && round >= 2 && !mbar_wait_warp(&sh.acc_empty[set], ((round >> 1) - 1) & 1, kWaitLimitNs)) ||
            !mbar_wait_warp(&sh.full[b], (i / kTcStages) & 1, kWaitLimitNs) ||  // the weight tile landed
            !mbar_wait_warp(&sh.conv[b], (i / kTcStages) & 1, kWaitLimitNs)) {  // the input tile is split
          give_up();
          ok = false;
          break;
        }
        tc::fence_after_sync();
        if (lane == 0) {
          uint8_t* stage = st0 + b * kTcStageBytes;
          const uint32_t d = tmem + set * kTcSetCols;
          const uint64_t bdesc = tc::smem_desc(stage + kTcABytes + kTcRawBytes, 128, 256);
#pragma unroll
          for (u32 a = 0; a < kTcPlanes; ++a) {
            const uint64_t adesc = tc::smem_desc(stage + a * 256, 128, kTcGroupBytes);
            tc::mma_bf16(d + a * kTcR, adesc, bdesc, id_main, (a > 0 || !first) ? 1u : 0u);
            if (a == 0 && first) tc::mma_bf16(d + kTcPlanes * kTcR, adesc, tc::smem_desc(Zt, 128, 256), id_zero, 0u);
          }
          tc::commit(&sh.empty[b]);
          if (last) tc::commit(&sh.acc_full[set]);
        }
        __syncwarp();
        if (last) ++round;
      }
    }
    if (lane == 0) tc::commit(&sh.done);  // every MMA issued has completed once this arrives
    __syncwarp();
    mbar_wait_warp(&sh.done, 0, kWaitLimitNs);
  } else if (warp < kTcEpi0) {
    // ---------------------------------------------------------------- input digit planes
    const int p0 = warp == 2 ? 0 : 4, p1 = warp == 2 ? 4 : (int)kTcPlanes;  // this warp's planes
    u32 i = 0;
    bool ok = true;
    for (u64 g = blockIdx.x; ok && g < total && !*abort_flag; g += gridDim.x) {
      TcWork w;
      get(g, w);
      const u32 sps = tc_stages(w.nJ), nc = min(kTcR, w.R - w.r0);
      for (u32 st = 0; st < kTcSlots * sps; ++st, ++i) {
        const u32 b = i % kTcStages, jb = min(kTcJB, w.nJ - (st % sps) * kTcJB);
        if (!mbar_wait_warp(&sh.full[b], (i / kTcStages) & 1, kWaitLimitNs)) {
          give_up();
          ok = false;
          break;
        }
        uint8_t* stage = st0 + b * kTcStageBytes;
        const u32 row = lane & (kTcR - 1), o = lane >> 4;  // (input row, octet of 8 k-blocks)
        if (row < nc) {
          const uint8_t* src = stage + kTcABytes + row * kTcRawRow;
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
          uint8_t* bt = stage + kTcABytes + kTcRawBytes;
#pragma unroll
          for (int p = 0; p < (int)kTcPlanes; ++p)
            if (p >= p0 && p < p1)
              *reinterpret_cast<uint4*>(bt + tc::tile_offset(p * kTcR + row, 8 * o, kTcJB * 2, 2)) = digit_plane(u, p);
        }
        tc::fence_smem_to_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.conv[b]);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const u32 q = warp & 3;        // TMEM lane quadrant this warp may read
    const u32 I = 32 * q + lane;   // weight row (TMEM lane) of this thread's outputs
    const u32 rh = (warp - kTcEpi0) >> 2;  // output rows 8 rh .. 8 rh + 7
    u64* const acc = accs + I;     // acc[r * 128]: this thread's sum of output row r
    u32 round = 0;
    bool ok = true;
    for (u64 g = blockIdx.x; ok && g < total && !*abort_flag; g += gridDim.x) {
      TcWork w;
      get(g, w);
      const u32 sps = tc_stages(w.nJ), R = w.R, rounds = (sps + kTcRound - 1) / kTcRound;
      const PrimeConsts P = C.p[w.l];
      u32 clo[kTcDiag], chi[kTcDiag];  // 256^d mod q_l in 32-bit halves
#pragma unroll
      for (u32 d = 0; d < kTcDiag; ++d) {
        clo[d] = P.pw256_lo[d];
        chi[d] = P.pw256_hi[d];
      }
      for (u32 slot = 0; ok && slot < kTcSlots; ++slot) {
        for (u32 rd = 0; rd < rounds; ++rd, ++round) {
          const u32 set = round & 1;
          if (!mbar_wait_warp(&sh.acc_full[set], (round >> 1) & 1, kWaitLimitNs)) {
            give_up();
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t tbase = tmem + set * kTcSetCols + ((32 * q) << 16);
          // 13 diagonal sums per output -> sum_d D_d 256^d mod q (tc_combine4); a round of at
          // most 32 k-blocks keeps |D_d| <= 7 * 32 * 2^14 < 2^22
          const bool small_round = w.nJ - rd * kTcRound * kTcJB <= 2 * kTcJB;
          // a warp whose 32 weight rows or 8 output rows all lie past the product's skips
          // the work (it still waits and arrives, keeping the rounds in step)
          const bool live = w.I0 + 32 * q < w.nI && w.r0 + 8 * rh < R;
#pragma unroll
          for (u32 h4 = 0; h4 < kTcR / 8; ++h4) {
            if (!live) break;
            const u32 hh = 2 * rh + h4;  // rows 4 hh .. 4 hh + 3
            uint32_t v[13][4];
#pragma unroll
            for (u32 d = 0; d < kTcDiag; ++d) tc::ld_32x32b_x4(tbase + d * kTcR + 4 * hh, v[d]);
            tc::wait_ld();
            u64 x[4];
            if (small_round) tc_combine4<true>(v, clo, chi, P, x);
            else tc_combine4<false>(v, clo, chi, P, x);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              u64& a = acc[(4 * hh + r) * kTcM];
              a = rd ? add_mod(a, x[r], P.q) : x[r];
            }
          }
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh.acc_empty[set]);
        }
        if (!ok) break;
        const u32 s = w.s0 + slot;  // the slot is complete: store its outputs
        if (w.I0 + I < w.nI) {
          if (w.acc) {  // coset product: row (2 Lb + c) G + g
            const u32 G = 1u << w.logG;
#pragma unroll
            for (u32 r = 8 * rh; r < 8 * rh + 8; ++r) {
              const u32 row = w.r0 + r;
              if (row < R) {
                const u32 rc = row >> w.logG, g = row & (G - 1);
                w.acc[(((w.ct0 + (u64)(rc >> 1) * w.nI + w.I0 + I) * 2 + (rc & 1)) * C.L + w.l) * (2ull * N) +
                      (u64)g * w.S + s] = acc[r * kTcM];
              }
            }
          } else {
#pragma unroll
            for (u32 r = 8 * rh; r < 8 * rh + 8; ++r) {
              const u32 row = w.r0 + r;
              if (row < R) {
                const u32 c = row & 1;
                w.out.base[c][(w.ct0 + (u64)(row >> 1) * w.nI + w.I0 + I) * w.out.ct_stride[c] + (u64)w.l * N + s] =
                    acc[r * kTcM];
              }
            }
          }
        }
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
