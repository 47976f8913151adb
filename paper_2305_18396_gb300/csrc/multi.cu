// multi.cu -- one set of launches for a list of products of different shapes (different
// m, k, n, blockings, weights, output modes): the forward NTT of every product's inputs,
// the multiply-accumulate of every product, the inverse NTTs and the masks each run as a
// single grid over the union of all products' work.  A product descriptor table travels
// as a kernel parameter; each block finds its product by binary search over per-kernel
// prefix sums of block counts.
#include <algorithm>

#include "async.cuh"
#include "coset.cuh"
#include "kernels.h"
#include "mac.cuh"
#include "mac_tc.cuh"
#include "mac_tcr.cuh"
#include "multi.h"
#include "ntt.cuh"

namespace he {

namespace {

constexpr int kThreadsSmall = 256;

// Largest i with begin(i) <= b (items sorted by their prefix sums).
template <class F>
__device__ __forceinline__ u32 find_item(const MultiTable& T, u64 b, F begin) {
  u32 lo = 0, hi = T.count - 1;
  while (lo < hi) {
    const u32 mid = (lo + hi + 1) >> 1;
    if (begin(T.it[mid]) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The item's mask seed: its value, or the word it points to (a seed that a replayed CUDA
// graph takes fresh on every replay).
__device__ __forceinline__ u64 item_seed(const MultiItem& it) { return it.seed_dev ? *it.seed_dev : it.mask_seed; }
__device__ __forceinline__ u64 seg_seed(const MultiSeg& sg) { return sg.seed_dev ? *sg.seed_dev : sg.mask_seed; }

// The segment of a merged item that holds row-block Lb (the last with lb0 <= Lb).
__device__ __forceinline__ const MultiSeg& find_seg(const MultiTable& T, const MultiItem& it, u32 Lb) {
  u32 s = it.seg0;
  for (u32 k = 1; k < it.nseg; ++k)
    if (T.seg[it.seg0 + k].lb0 <= Lb) s = it.seg0 + k;
  return T.seg[s];
}

template <int LOGN, int LOGR>
__global__ void __launch_bounds__(NttShape<LOGN, LOGR>::T, NttShape<LOGN, LOGR>::kMinBlocks) k_fwd_multi_t(const __grid_constant__ MultiTable T,
                                                                   const __grid_constant__ Consts C) {
  using S = NttShape<LOGN, LOGR>;
  extern __shared__ u64 sm[];
  const u32 i = find_item(T, blockIdx.x, [](const MultiItem& x) { return x.fwd_begin; });
  const MultiItem& it = T.it[i];
  const u64 local = blockIdx.x - it.fwd_begin;
  const u32 l = local % C.L, c = (local / C.L) % 2;
  const u32 LbJ = (u32)(local / (2 * C.L));
  const u32 Lb = LbJ / it.nJ, J = LbJ % it.nJ;
  const u64* sp;
  if (it.nseg) {  // merged: the request's own input ciphertexts, wire format
    const MultiSeg& sg = find_seg(T, it, Lb);
    sp = sg.ct_in + ((((u64)(Lb - sg.lb0) * it.nJ + J) * 2 + c) * C.L + l) * S::N;
  } else {
    sp = it.ct_in + local * S::N;
  }
  const u64 row = (u64)Lb * 2 + c;
  if (it.tc) {
    const u32 nS = tc_stages(it.nJ), rows = 2 * it.nLb;
    ntt_forward_block<S>(sm, C.p[l], [&](u32 e) { return sp[e]; },
                         [&](u32 e, u64 v) { it.ctN[tc_index((u32)row, J, l, e, rows, nS, S::N)] = v; });
  } else {
    ntt_forward_block<S>(sm, C.p[l], [&](u32 e) { return sp[e]; },
                         [&](u32 e, u64 v) { it.ctN[chunked_index(row, J, l, e, it.nJ, C.L, S::N)] = split_word(v); });
  }
}

__global__ void __launch_bounds__(kThreadsSmall) k_fwd_multi_small(const __grid_constant__ MultiTable T,
                                                                   const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u32 i = find_item(T, blockIdx.x, [](const MultiItem& x) { return x.fwd_begin; });
  const MultiItem& it = T.it[i];
  const u64 local = blockIdx.x - it.fwd_begin;
  const u32 l = local % C.L, c = (local / C.L) % 2;
  const u32 LbJ = (u32)(local / (2 * C.L));
  const u32 Lb = LbJ / it.nJ, J = LbJ % it.nJ;
  for (u32 e = threadIdx.x; e < C.N; e += blockDim.x) sm[e] = it.ct_in[local * C.N + e];
  __syncthreads();
  ntt_forward_smem(sm, C.logN, C.p[l]);
  for (u32 e = threadIdx.x; e < C.N; e += blockDim.x)
    it.ctN[chunked_index((u64)Lb * 2 + c, J, l, e, it.nJ, C.L, C.N)] = split_word(sm[e]);
}

template <class M, int MINB>
__global__ void __launch_bounds__(M::kThreads + 32, MINB) k_mac_multi_t(const __grid_constant__ MultiTable T, int* err,
                                                                   const __grid_constant__ Consts C) {
  extern __shared__ __align__(128) u64 sm[];
  const u32 i = find_item(T, blockIdx.x, [](const MultiItem& x) { return x.mac_begin; });
  const MultiItem& it = T.it[i];
  const u64 local = blockIdx.x - it.mac_begin;
  const u32 chunks = C.N >> 5;
  const u32 tiles = it.tilesR * it.tilesC;
  const u32 tile = local % tiles;  // tile-fastest: a chunk's operand rows are reused from L2
  const u64 rest = local / tiles;
  const u32 chunk = rest % chunks, l = (u32)(rest / chunks);
  const u32 r0 = (tile % it.tilesR) * M::kRows, c0 = (tile / it.tilesR) * M::kCols;
  const u64 N = C.N, L = C.L;
  OutPlace out;
  if (it.nseg) {  // merged: both components to the workspace, NTT domain
    out.base[0] = it.c0_ntt;
    out.base[1] = it.c1_ntt;
    out.ct_stride[0] = out.ct_stride[1] = L * N;
  } else if (it.compact) {
    const u64 Nc = N >> it.logkb;
    out.base[0] = it.c0_ntt;
    out.ct_stride[0] = L * N;
    out.base[1] = it.out + L * Nc;
    out.ct_stride[1] = L * (Nc + N);
  } else {
    out.base[0] = it.out;
    out.base[1] = it.out + L * N;
    out.ct_stride[0] = out.ct_stride[1] = 2 * L * N;
  }
  mac_tile_ws<M>(it.ctN, it.pt, out, 0, it.nI, it.nJ, it.nLb, r0, c0, chunk, l, err, C, sm);
}

// The tensor-core multiply-accumulate (mac_tc.cuh) over the products flagged tc: one block
// per SM works through the launch's work units (product, prime, slot group, weight-row tile,
// row tile) back to back; each unit's product is found by its offset tc_begin.
__global__ void __launch_bounds__(kTcThreads, 1) k_mac_tc_multi(const __grid_constant__ MultiTable T, u64 total,
                                                               int* err, const __grid_constant__ Consts C) {
  extern __shared__ __align__(128) uint8_t smem_tc[];
  __shared__ TcShared sh;
  auto get = [&](u64 g, TcWork& w) {
    const u32 i = find_item(T, g, [](const MultiItem& x) { return x.tc_begin; });
    const MultiItem& it = T.it[i];
    const u64 N = C.N, L = C.L;
    if (it.coset) {  // rows (2 Lb + c) G + g, 2D slots per prime, sums to acc
      const u32 logG = C.logN - it.logD;
      tc_unit(g - it.tc_begin, 2u << it.logD, it.nI, (2 * it.nLb) << logG, w);
      w.acc = it.acc;
      w.logG = logG;
    } else {
      tc_unit(g - it.tc_begin, C.N, it.nI, 2 * it.nLb, w);
      w.acc = nullptr;
      w.logG = 0;
    }
    w.ctN = it.ctN;
    w.ptd = reinterpret_cast<const uint8_t*>(it.pt);
    w.ct0 = 0;
    w.nI = it.nI;
    w.nJ = it.nJ;
    w.nLb = it.nLb;
    if (it.nseg) {  // merged: both components to the workspace, NTT domain
      w.out.base[0] = it.c0_ntt;
      w.out.base[1] = it.c1_ntt;
      w.out.ct_stride[0] = w.out.ct_stride[1] = L * N;
    } else if (it.compact) {
      const u64 Nc = N >> it.logkb;
      w.out.base[0] = it.c0_ntt;
      w.out.ct_stride[0] = L * N;
      w.out.base[1] = it.out + L * Nc;
      w.out.ct_stride[1] = L * (Nc + N);
    } else {
      w.out.base[0] = it.out;
      w.out.base[1] = it.out + L * N;
      w.out.ct_stride[0] = w.out.ct_stride[1] = 2 * L * N;
    }
  };
  mac_tc_run(get, total, err, C, smem_tc, sh);
}

// ---------------------------------------------------------------- coset products
//
// Resident blocks per SM asked of the compiler: two for blocks of at most 256 threads (128
// registers each), else one.
template <int LOGN>
constexpr int kCosetMinBlocks = NttShape<LOGN, 4>::T <= 256 ? 2 : 1;
//
// One block of S::T = N / 16 threads per polynomial (S = NttShape<log2 N, 4>); products with
// D <= 32 take the register-blocked transforms of coset.cuh (S::kSmemWords words of shared
// memory), larger D the shared-memory forms (2N words).

// Forward coset transform (coset.cuh) of one input polynomial of a coset item: the first
// log2 G NTT stages, then the zero-padded length-2D transform of each coset, into the
// stage-tiled operand layout of the tensor-core multiply-accumulate (rows (2 Lb + c) G + g,
// 2D slots per prime).
template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN, 4>::T, kCosetMinBlocks<LOGN>) k_coset_fwd_multi_t(const __grid_constant__ MultiTable T,
                                                                          const __grid_constant__ Consts C) {
  using S = NttShape<LOGN, 4>;
  extern __shared__ u64 sm[];
  const u32 i = find_item(T, blockIdx.x, [](const MultiItem& x) { return x.cfwd_begin; });
  const MultiItem& it = T.it[i];
  const u64 local = blockIdx.x - it.cfwd_begin;
  const u32 N = S::N, l = local % C.L, c = (local / C.L) % 2;
  const u32 LbJ = (u32)(local / (2 * C.L));
  const u32 Lb = LbJ / it.nJ, J = LbJ % it.nJ;
  const u64* sp;
  if (it.nseg) {  // merged: the request's own input ciphertexts, wire format
    const MultiSeg& sg = find_seg(T, it, Lb);
    sp = sg.ct_in + ((((u64)(Lb - sg.lb0) * it.nJ + J) * 2 + c) * C.L + l) * N;
  } else {
    sp = it.ct_in + local * N;
  }
  const PrimeConsts P = C.p[l];
  const u32 logD = it.logD, logG = LOGN - logD;
  const u32 S2 = 2u << logD, R = (2 * it.nLb) << logG, nS = tc_stages(it.nJ), row0 = (Lb * 2 + c) << logG;
  u64* dst = it.ctN;
  auto load = [&](u32 e) { return sp[e]; };
  auto store = [&](u32 g, u32 slot, u64 v) { dst[tc_index(row0 + g, J, l, slot, R, nS, S2)] = v; };
  switch (logD) {
    case 3: coset_forward_fast<S, 3>(sm, P, load, store); break;
    case 4: coset_forward_fast<S, 4>(sm, P, load, store); break;
    case 5: coset_forward_fast<S, 5>(sm, P, load, store); break;
    case 6: coset_forward_passes<S, 6>(sm, sm + S::kSmemWords, P, load, store); break;
    case 7: coset_forward_passes<S, 7>(sm, sm + S::kSmemWords, P, load, store); break;
    default: {
      u64* A = sm;
      u64* B = sm + N;
      for (u32 e = threadIdx.x; e < N; e += blockDim.x) A[e] = sp[e];
      __syncthreads();
      coset_head_fwd(A, LOGN, logG, P);
      coset_tail_fwd(A, B, LOGN, logD, P, store);
    }
  }
}

// Inverse coset transform of one output component (o, c, l) of a coset item: its 2N sums
// from acc, the inverse length-2D transforms, the fold, the inverse of the first log2 G
// stages; c0 is re-masked (Algorithm 1 step 3) and, for compact products, kept only at the
// decoded coefficients (Sec. 3.1.3).
template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN, 4>::T, kCosetMinBlocks<LOGN>) k_coset_inv_multi_t(const __grid_constant__ MultiTable T,
                                                                          const __grid_constant__ Consts C) {
  using S = NttShape<LOGN, 4>;
  extern __shared__ u64 sm[];
  const u32 i = find_item(T, blockIdx.x, [](const MultiItem& x) { return x.cinv_begin; });
  const MultiItem& it = T.it[i];
  const u64 local = blockIdx.x - it.cinv_begin;
  const u32 N = S::N, L = C.L, l = local % L, c = (local / L) % 2;
  const u64 o = local / (2 * L);
  const PrimeConsts P = C.p[l];
  const u32 logD = it.logD, D = 1u << logD;
  const u64* src = it.acc + local * 2 * (u64)N;
  u64* base;
  u64 seed, oo = o;
  if (it.nseg) {  // merged: the request's compact output, seed and output index
    const MultiSeg& sg = find_seg(T, it, (u32)(o / it.nI));
    oo = o - (u64)sg.lb0 * it.nI;
    base = sg.out + oo * L * ((N >> it.logkb) + N);
    seed = seg_seed(sg);
  } else {
    base = it.out + o * (it.compact ? L * ((N >> it.logkb) + N) : 2ull * L * N);
    seed = item_seed(it);
  }
  const bool compact = it.compact || it.nseg;
  const u32 Nc = N >> it.logkb, kbm = (1u << it.logkb) - 1;
  // coefficient e of this component (v in [0, q)): re-mask c0, keep what the output holds
  auto emit = [&](u32 e, u64 v) {
    if (c == 0) {
      if (compact && (e & kbm) != kbm) return;
      const u64 sv = lo64(draw(seed, e, (u32)oo, kDomainMask, 0)) & C.tmask;
      v = sub_mod(v, delta_residue(sv, C, P), P.q);
      if (compact) base[(u64)l * Nc + (e >> it.logkb)] = v;
      else base[(u64)l * N + e] = v;
    } else {
      base[(compact ? (u64)L * Nc : (u64)L * N) + (u64)l * N + e] = v;
    }
  };
  switch (logD) {
    case 3: coset_inverse_fast<S, 3>(sm, P, src, emit); break;
    case 4: coset_inverse_fast<S, 4>(sm, P, src, emit); break;
    case 5: coset_inverse_fast<S, 5>(sm, P, src, emit); break;
    case 6: coset_inverse_passes<S, 6>(sm, sm + S::kSmemWords, P, src, emit); break;
    case 7: coset_inverse_passes<S, 7>(sm, sm + S::kSmemWords, P, src, emit); break;
    default: {
      u64* A = sm;
      u64* B = sm + N;
      for (u32 e = threadIdx.x; e < 2 * N; e += blockDim.x) {
        const u32 g = e >> (logD + 1), pos = e & (2 * D - 1);
        (pos < D ? A : B)[g * D + (pos & (D - 1))] = src[e];
      }
      __syncthreads();
      coset_inverse(A, B, LOGN, logD, P);
      for (u32 e = threadIdx.x; e < N; e += blockDim.x) emit(e, csub(A[e], P.q));
    }
  }
}

// Weights of coset products: block b transforms up to G weight blocks of one (batch item,
// prime) at once -- the G blocks of D coefficients of the tail transform are G different
// weight blocks here -- and writes each one's 2D slots as bf16 digit tiles (mac_tc.cuh).
template <int LOGN>
__global__ void __launch_bounds__(NttShape<LOGN, 4>::T, kCosetMinBlocks<LOGN>) k_coset_encode_t(const u64* W, u32 k, u32 n, Blk b, u32 nI,
                                                                       u32 nJ, u32 logD, u32 tcr, u64* pt,
                                                                       const __grid_constant__ Consts C) {
  using S = NttShape<LOGN, 4>;
  extern __shared__ u64 sm[];
  const u32 N = S::N, logG = LOGN - logD, D = 1u << logD, G = 1u << logG, S2 = 2u << logD;
  const u32 per = nI * nJ, bpl = (per + G - 1) / G;  // weight blocks and blocks of the grid per (item, prime)
  const u32 il = blockIdx.x / bpl, first = (blockIdx.x % bpl) * G;
  const u32 item = il / C.L, l = il % C.L;
  const PrimeConsts P = C.p[l];
  W += (u64)item * k * n;
  uint8_t* const ptd =
      reinterpret_cast<uint8_t*>(pt + (u64)item * (tcr ? tcr_weight_words(nI, nJ, C.L, S2) : tc_weight_words(nI, nJ, C.L, S2)));
  const u32 nk = b.n_b * b.k_b, nS = tc_stages(nJ);
  const u64 half_t = (C.tmask >> 1) + 1;
  const bool fast = logD <= (u32)kCosetPassMaxLogD;  // the padded layout of the register forms
  for (u32 e = threadIdx.x; e < N; e += blockDim.x) {
    const u32 wb = first + (e >> logD), p = e & (D - 1);
    u64 v = 0;
    if (wb < per && p < nk) {  // pi_A: coefficient p = i k_b + k_b - 1 - j of block (I, J)
      const u32 I = wb / nJ, J = wb % nJ;
      const u32 ii = p / b.k_b, jj = b.k_b - 1 - p % b.k_b;
      const u32 row = J * b.k_b + jj, col = I * b.n_b + ii;
      if (row < k && col < n) {
        const u64 w = W[(u64)row * n + col] & C.tmask;
        v = w >= half_t ? P.q - (C.tmask + 1 - w) : w;  // centred lift [-t/2, t/2)
      }
    }
    sm[fast ? S::pad(e) : e] = v;
  }
  __syncthreads();
  auto store = [&](u32 g, u32 slot, u64 v) {
    const u32 wb = first + g;
    if (wb >= per) return;
    const u32 I = wb / nJ, J = wb % nJ;
    const u64 u = v + 0x0080808080808080ull;
    if (tcr) {  // row-major digit tile (mac_tcr.cuh): row 16 b + i of weight tile I / 16
      uint8_t* tile = ptd + tcr_weight_offset(I >> 4, l, slot, J >> 4, tcr_tiles_I(nI), nS, S2);
#pragma unroll
      for (int q = 0; q < (int)kTcPlanes; ++q)
        *reinterpret_cast<uint16_t*>(tile + tc::tile_offset(kTcrI * q + (I & 15), J & 15, kTcJB * 2, 2)) =
            (uint16_t)(digit_f32_bits(u, q) >> 16);
      return;
    }
    uint8_t* grp = ptd + tc_weight_offset(I & ~7u, l, slot, J >> 4, nI, nS, S2);
#pragma unroll
    for (int q = 0; q < (int)kTcPlanes; ++q)
      *reinterpret_cast<uint16_t*>(grp + tc::tile_offset(I & 7, kTcJB * q + (J & 15), kTcAKBytes, 2)) =
          (uint16_t)(digit_f32_bits(u, q) >> 16);
  };
  switch (logD) {
    case 3: coset_tail_regs<S, 3>(sm, P, store); break;
    case 4: coset_tail_regs<S, 4>(sm, P, store); break;
    case 5: coset_tail_regs<S, 5>(sm, P, store); break;
    case 6: coset_tail_both<S, 6>(sm, sm + S::kSmemWords, P, store); break;
    case 7: coset_tail_both<S, 7>(sm, sm + S::kSmemWords, P, store); break;
    default: coset_tail_fwd(sm, sm + N, LOGN, logD, P, store);
  }
}

#define HE_COSET_LOGNS(X) X(9) X(10) X(11) X(12) X(13)

// Shared-memory bytes of the coset grids: the most any coset item of the table needs.
// Shared-memory words of a coset transform of one polynomial with cosets of 2^logD.
__host__ __device__ inline u32 coset_words(u32 N, u32 logD) {
  const u32 padded = N + (N >> 4);
  return logD <= (u32)kCosetFastMaxLogD ? padded : logD <= (u32)kCosetPassMaxLogD ? 2 * padded : 2 * N;
}

size_t coset_smem(const Consts& C, const MultiTable& T) {
  u32 words = 0;
  for (u32 i = 0; i < T.count; ++i)
    if (T.it[i].coset) words = max(words, coset_words(C.N, T.it[i].logD));
  return (size_t)words * sizeof(u64);
}

// The row-major tensor-core multiply-accumulate (mac_tcr.cuh) over the items flagged tcr:
// one block per SM works through their units (product, prime, slot, 128 input rows).
__global__ void __launch_bounds__(kTcrThreads, 1) k_mac_tcr_multi(const __grid_constant__ MultiTable T, u64 total,
                                                                 int* err, const __grid_constant__ Consts C) {
  extern __shared__ __align__(128) uint8_t smem_tcr[];
  __shared__ TcrShared sh;
  auto get = [&](u64 g, TcrWork& w) {
    const u32 i = find_item(T, g, [](const MultiItem& x) { return x.tcr_begin; });
    const MultiItem& it = T.it[i];
    const u32 logG = C.logN - it.logD;
    tcr_unit(g - it.tcr_begin, 2u << it.logD, (2 * it.nLb) << logG, w);
    w.ctN = it.ctN;
    w.ptd = reinterpret_cast<const uint8_t*>(it.pt);
    w.acc = it.acc;
    w.ct0 = 0;
    w.nI = it.nI;
    w.nJ = it.nJ;
    w.logG = logG;
  };
  mac_tcr_run(get, total, err, C, smem_tcr, sh);
}

// Inverse NTT of block b of the inverse grid: compact products transform their c1
// polynomials in place; full products transform every output polynomial and re-mask c0.
template <class S>
__device__ __forceinline__ void inv_block(const MultiTable& T, const Consts& C, u64 b, u64* sm) {
  const u32 i = find_item(T, b, [](const MultiItem& x) { return x.inv_begin; });
  const MultiItem& it = T.it[i];
  const u64 local = b - it.inv_begin;
  const u64 N = S::N, L = C.L;
  const u32 l = local % L;
  if (it.nseg) {  // merged: c1 from the workspace to the request's compact output
    const u64 Nc = N >> it.logkb, o = local / L;
    const MultiSeg& sg = find_seg(T, it, (u32)(o / it.nI));
    const u64* src = it.c1_ntt + o * L * N + l * N;
    u64* d = sg.out + (o - (u64)sg.lb0 * it.nI) * L * (Nc + N) + L * Nc + l * N;
    ntt_inverse_block<S>(sm, C.p[l], [&](u32 e) { return src[e]; }, [&](u32 e, u64 v) { d[e] = v; });
  } else if (it.compact) {
    const u64 Nc = N >> it.logkb;
    u64* d = it.out + (local / L) * L * (Nc + N) + L * Nc + l * N;
    ntt_inverse_block<S>(sm, C.p[l], [&](u32 e) { return d[e]; }, [&](u32 e, u64 v) { d[e] = v; });
  } else {
    const u32 c = (local / L) % 2;
    const u32 o = (u32)(local / (2 * L));
    const PrimeConsts P = C.p[l];
    u64* d = it.out + local * N;
    const u64 seed = item_seed(it);
    ntt_inverse_block<S>(sm, P, [&](u32 e) { return d[e]; }, [&](u32 e, u64 v) {
      if (c == 0) {
        const u64 sv = lo64(draw(seed, e, o, kDomainMask, 0)) & C.tmask;
        v = sub_mod(v, delta_residue(sv, C, P), P.q);
      }
      d[e] = v;
    });
  }
}

// Pruned inverse NTT + mask of c0 for block b of the c0 grid (one block per (o, l) of the
// compact products).
__device__ __forceinline__ void c0_block(const MultiTable& T, const Consts& C, u64 b, u64* sm) {
  const u32 i = find_item(T, b, [](const MultiItem& x) { return x.c0_begin; });
  const MultiItem& it = T.it[i];
  const u64 local = b - it.c0_begin;
  const u64 N = C.N, L = C.L, Nc = N >> it.logkb;
  const u32 l = local % L;
  const u32 o = (u32)(local / L);
  if (it.nseg) {  // merged: the request's output and seed, its own output index
    const MultiSeg& sg = find_seg(T, it, o / it.nI);
    const u32 ol = o - sg.lb0 * it.nI;
    ntt_inverse_c0_targets(it.c0_ntt + local * N, sg.out + (u64)ol * L * (Nc + N) + l * Nc, it.logkb, seg_seed(sg), ol,
                           l, C, sm);
    return;
  }
  ntt_inverse_c0_targets(it.c0_ntt + local * N, it.out + (u64)o * L * (Nc + N) + l * Nc, it.logkb, item_seed(it), o, l,
                         C, sm);
}

template <int LOGN, int LOGR>
__global__ void __launch_bounds__(NttShape<LOGN, LOGR>::T, NttShape<LOGN, LOGR>::kMinBlocks) k_inv_multi_t(const __grid_constant__ MultiTable T,
                                                                   const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  inv_block<NttShape<LOGN, LOGR>>(T, C, blockIdx.x, sm);
}

// The c1 inverse NTTs and the pruned c0 transforms are independent: one grid runs both,
// blocks [0, inv_blocks) the former and the rest the latter, so neither drains alone.
template <int LOGN, int LOGR>
__global__ void __launch_bounds__(NttShape<LOGN, LOGR>::T, NttShape<LOGN, LOGR>::kMinBlocks) k_inv_c0_multi_t(
    const __grid_constant__ MultiTable T, const __grid_constant__ Consts C, u64 inv_blocks) {
  extern __shared__ u64 sm[];
  if (blockIdx.x < inv_blocks) inv_block<NttShape<LOGN, LOGR>>(T, C, blockIdx.x, sm);
  else c0_block(T, C, blockIdx.x - inv_blocks, sm);
}

__global__ void __launch_bounds__(kThreadsSmall) k_inv_multi_small(const __grid_constant__ MultiTable T,
                                                                   const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u32 i = find_item(T, blockIdx.x, [](const MultiItem& x) { return x.inv_begin; });
  const MultiItem& it = T.it[i];
  const u64 local = blockIdx.x - it.inv_begin;
  const u64 N = C.N, L = C.L;
  const u32 l = local % L;
  const PrimeConsts P = C.p[l];
  u64* d;
  u32 c = 1, o = 0;
  if (it.compact) {
    const u64 Nc = N >> it.logkb;
    d = it.out + (local / L) * L * (Nc + N) + L * Nc + l * N;
  } else {
    c = (local / L) % 2;
    o = (u32)(local / (2 * L));
    d = it.out + local * N;
  }
  const u64 seed = item_seed(it);
  for (u32 e = threadIdx.x; e < N; e += blockDim.x) sm[e] = d[e];
  __syncthreads();
  ntt_inverse_smem(sm, C.logN, P);
  for (u32 e = threadIdx.x; e < N; e += blockDim.x) {
    u64 v = sm[e];
    if (c == 0) {
      const u64 sv = lo64(draw(seed, e, o, kDomainMask, 0)) & C.tmask;
      v = sub_mod(v, delta_residue(sv, C, P), P.q);
    }
    d[e] = v;
  }
}

// Pruned inverse NTT + mask of c0 for the compact products (one block per (o, l)).
__global__ void __launch_bounds__(kThreadsSmall) k_c0_multi(const __grid_constant__ MultiTable T,
                                                            const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  c0_block(T, C, blockIdx.x, sm);
}

// KERNEL<LOGN, LOGR> for the context's (log N, radix); a pair that is not built is an error.
#define HE_MULTI_CASE(LN, LR, KERNEL, GRID, ST, ...)                                                               \
  case HE_NTT_KEY(LN, LR):                                                                                         \
    KERNEL<LN, LR><<<GRID, NttShape<LN, LR>::T, NttShape<LN, LR>::kSmemWords * sizeof(u64), ST>>>(__VA_ARGS__);    \
    break;
#define HE_MULTI_DISPATCH(KERNEL, GRID, ST, ...)                                                                   \
  switch (HE_NTT_KEY(C.logN, C.logR)) {                                                                            \
    HE_NTT_SHAPES(HE_MULTI_CASE, KERNEL, GRID, ST, __VA_ARGS__)                                                    \
    default: return cudaErrorInvalidValue;                                                                         \
  }

}  // namespace

cudaError_t configure_multi_kernels() {
  const int one = 8192 * (int)sizeof(u64);
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f, int bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  set((const void*)k_fwd_multi_small, one);
  set((const void*)k_inv_multi_small, one);
  set((const void*)k_c0_multi, 2 * one);
  set((const void*)k_mac_multi_t<MacProd, kMacMinBlocks>, (int)MacProd::kSmemBytes);
  set((const void*)k_mac_tc_multi, (int)kTcSmem);
  set((const void*)k_mac_tcr_multi, (int)kTcrSmem);
#define HE_SET_COSET(LN)                                                                      \
  set((const void*)k_coset_fwd_multi_t<LN>, 2 * ((1 << LN) + (1 << LN) / 16) * (int)sizeof(u64)); \
  set((const void*)k_coset_inv_multi_t<LN>, 2 * ((1 << LN) + (1 << LN) / 16) * (int)sizeof(u64)); \
  set((const void*)k_coset_encode_t<LN>, 2 * ((1 << LN) + (1 << LN) / 16) * (int)sizeof(u64));
  HE_COSET_LOGNS(HE_SET_COSET)
#undef HE_SET_COSET
  if (e == cudaSuccess)  // two blocks per SM need the largest shared-memory carveout
    e = cudaFuncSetAttribute((const void*)k_mac_tc_multi, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
#define HE_SET_MULTI(LN, LR, unused)                                                                   \
  set((const void*)k_fwd_multi_t<LN, LR>, NttShape<LN, LR>::kSmemWords * (int)sizeof(u64));            \
  set((const void*)k_inv_multi_t<LN, LR>, NttShape<LN, LR>::kSmemWords * (int)sizeof(u64));            \
  set((const void*)k_inv_c0_multi_t<LN, LR>, 2 * (1 << LN) * (int)sizeof(u64));
  HE_NTT_SHAPES(HE_SET_MULTI, 0)
#undef HE_SET_MULTI
  return e;
}

u32 mac_tile_rows() { return MacProd::kRows; }
u32 mac_tile_cols() { return MacProd::kCols; }

cudaError_t launch_fwd_multi(const Consts& C, const MultiTable& T, u64 blocks, cudaStream_t st) {
  if (!blocks) return cudaGetLastError();
  if (C.logN >= 9) {
    HE_MULTI_DISPATCH(k_fwd_multi_t, (unsigned)blocks, st, T, C)
  } else {
    k_fwd_multi_small<<<(unsigned)blocks, kThreadsSmall, C.N * sizeof(u64), st>>>(T, C);
  }
  return cudaGetLastError();
}

cudaError_t launch_mac_multi(const Consts& C, const MultiTable& T, u64 blocks, int* err, cudaStream_t st) {
  if (blocks)
    k_mac_multi_t<MacProd, kMacMinBlocks><<<(unsigned)blocks, MacProd::kThreads + 32, MacProd::kSmemBytes, st>>>(
        T, err, C);
  return cudaGetLastError();
}

cudaError_t launch_mac_tc_multi(const Consts& C, const MultiTable& T, u64 units, int* err, cudaStream_t st) {
  if (units) {
    const u64 grid = std::min<u64>(units, (u64)device_sms());
    k_mac_tc_multi<<<(unsigned)grid, kTcThreads, kTcSmem, st>>>(T, units, err, C);
  }
  return cudaGetLastError();
}

cudaError_t launch_mac_tcr_multi(const Consts& C, const MultiTable& T, u64 units, int* err, cudaStream_t st) {
  if (units) {
    const u64 grid = std::min<u64>(units, (u64)device_sms());
    k_mac_tcr_multi<<<(unsigned)grid, kTcrThreads, kTcrSmem, st>>>(T, units, err, C);
  }
  return cudaGetLastError();
}

cudaError_t launch_inv_multi(const Consts& C, const MultiTable& T, u64 blocks, cudaStream_t st) {
  if (!blocks) return cudaGetLastError();
  if (C.logN >= 9) {
    HE_MULTI_DISPATCH(k_inv_multi_t, (unsigned)blocks, st, T, C)
  } else {
    k_inv_multi_small<<<(unsigned)blocks, kThreadsSmall, C.N * sizeof(u64), st>>>(T, C);
  }
  return cudaGetLastError();
}

// One grid where the inverse transform's blocks are small (at most 256 threads, N <= 4096);
// at N = 8192 the inverse transform's 512-thread, 68 KB blocks would starve the c0 blocks
// (measured: 19% slower than two grids), and small rings use the simple kernels.
bool inv_c0_fused(const Consts& C) { return C.logN >= 9 && C.logN <= 12 && C.logN - C.logR <= 8; }

cudaError_t launch_inv_c0_multi(const Consts& C, const MultiTable& T, u64 inv_blocks, u64 c0_blocks, u32 c0_words,
                                cudaStream_t st) {
  if (!inv_c0_fused(C)) {
    cudaError_t e = launch_inv_multi(C, T, inv_blocks, st);
    return e == cudaSuccess ? launch_c0_multi(C, T, c0_blocks, c0_words, st) : e;
  }
  const u64 blocks = inv_blocks + c0_blocks;
  if (!blocks) return cudaGetLastError();
#define HE_INV_C0(LN, LR, unused)                                                                    \
  case HE_NTT_KEY(LN, LR): {                                                                         \
    using S = NttShape<LN, LR>;                                                                      \
    const u32 words = (u32)S::kSmemWords > c0_words ? (u32)S::kSmemWords : c0_words;                 \
    k_inv_c0_multi_t<LN, LR><<<(unsigned)blocks, S::T, (size_t)words * sizeof(u64), st>>>(T, C, inv_blocks); \
    break;                                                                                           \
  }
  switch (HE_NTT_KEY(C.logN, C.logR)) {
    HE_NTT_SHAPES(HE_INV_C0, 0)
    default: return cudaErrorInvalidValue;
  }
#undef HE_INV_C0
  return cudaGetLastError();
}

#define HE_COSET_CASE(LN, KERNEL, GRID, SMEM, ST, ...)                                                     \
  case LN:                                                                                                   \
    KERNEL<LN><<<GRID, NttShape<LN, 4>::T, SMEM, ST>>>(__VA_ARGS__);                                         \
    break;
#define HE_COSET_DISPATCH(KERNEL, GRID, SMEM, ST, ...)                                                       \
  switch (C.logN) {                                                                                          \
    HE_COSET_CASE(9, KERNEL, GRID, SMEM, ST, __VA_ARGS__)                                                    \
    HE_COSET_CASE(10, KERNEL, GRID, SMEM, ST, __VA_ARGS__)                                                   \
    HE_COSET_CASE(11, KERNEL, GRID, SMEM, ST, __VA_ARGS__)                                                   \
    HE_COSET_CASE(12, KERNEL, GRID, SMEM, ST, __VA_ARGS__)                                                   \
    HE_COSET_CASE(13, KERNEL, GRID, SMEM, ST, __VA_ARGS__)                                                   \
    default: return cudaErrorInvalidValue;                                                                   \
  }

cudaError_t launch_coset_fwd_multi(const Consts& C, const MultiTable& T, u64 blocks, cudaStream_t st) {
  if (!blocks) return cudaGetLastError();
  const size_t smem = coset_smem(C, T);
  HE_COSET_DISPATCH(k_coset_fwd_multi_t, (unsigned)blocks, smem, st, T, C)
  return cudaGetLastError();
}

cudaError_t launch_coset_inv_multi(const Consts& C, const MultiTable& T, u64 blocks, cudaStream_t st) {
  if (!blocks) return cudaGetLastError();
  const size_t smem = coset_smem(C, T);
  HE_COSET_DISPATCH(k_coset_inv_multi_t, (unsigned)blocks, smem, st, T, C)
  return cudaGetLastError();
}

cudaError_t launch_coset_encode_weights(const Consts& C, const u64* W, u32 k, u32 n, Blk b, u32 nI, u32 nJ, u32 batch,
                                        u32 tcr, u64* pt, cudaStream_t st) {
  const u32 logD = coset_logD(b.n_b * b.k_b);
  if (!nI || !nJ || !batch) return cudaGetLastError();
  if (C.logN < 9 || logD >= C.logN) return cudaErrorInvalidValue;
  const u32 S2 = 2u << logD, G = C.N >> logD;
  // digit tiles: k-blocks past the last and rows past nI must read as zero digits
  cudaError_t e = cudaMemsetAsync(
      pt, 0, 8ull * batch * (tcr ? tcr_weight_words(nI, nJ, C.L, S2) : tc_weight_words(nI, nJ, C.L, S2)), st);
  if (e != cudaSuccess) return e;
  const u64 blocks = (u64)batch * C.L * (((u64)nI * nJ + G - 1) / G);
  const size_t smem = (size_t)coset_words(C.N, logD) * sizeof(u64);
  HE_COSET_DISPATCH(k_coset_encode_t, (unsigned)blocks, smem, st, W, k, n, b, nI, nJ, logD, tcr, pt, C)
  return cudaGetLastError();
}

cudaError_t launch_c0_multi(const Consts& C, const MultiTable& T, u64 blocks, u32 c0_words, cudaStream_t st) {
  if (blocks) k_c0_multi<<<(unsigned)blocks, kThreadsSmall, (size_t)c0_words * sizeof(u64), st>>>(T, C);
  return cudaGetLastError();
}

}  // namespace he
