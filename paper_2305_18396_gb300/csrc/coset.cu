// coset.cu -- the kernels of the coset form (coset.cuh) in the multi-product launch: the
// forward transforms of coset products' inputs, the inverse transforms of their outputs
// (fold, mask, compact c0) and the encoding of their weights.  A translation unit of its
// own, compiled beside multi.cu.
#include <algorithm>

#include "coset.cuh"
#include "kernels.h"
#include "mac_tc.cuh"
#include "mac_tcr.cuh"
#include "multi.h"
#include "multi_items.cuh"
#include "ntt.cuh"

namespace he {

namespace {

// ---------------------------------------------------------------- coset products
//
// Resident blocks per SM asked of the compiler: two for blocks of at most 256 threads (128
// registers each), else one.
template <int LOGN>
constexpr int kCosetMinBlocks = NttShape<LOGN, 4>::T <= 256 ? 2 : 1;
// The register-blocked transforms are built for N = 4096 and 8192 (the rings the workloads
// use); smaller rings take the shared-memory forms (same results, less code to compile).
template <int LOGN>
constexpr bool kCosetRegisterForms = LOGN >= 12;
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
  switch (kCosetRegisterForms<LOGN> ? logD : 0u) {
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
  switch (kCosetRegisterForms<LOGN> ? logD : 0u) {
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
  const bool fast = kCosetRegisterForms<LOGN> && logD <= (u32)kCosetPassMaxLogD;  // padded layout of the register forms
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
  switch (kCosetRegisterForms<LOGN> ? logD : 0u) {
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
  if (N < 4096) return 2 * N;
  return logD <= (u32)kCosetFastMaxLogD ? padded : logD <= (u32)kCosetPassMaxLogD ? 2 * padded : 2 * N;
}

size_t coset_smem(const Consts& C, const MultiTable& T) {
  u32 words = 0;
  for (u32 i = 0; i < T.count; ++i)
    if (T.it[i].coset) words = max(words, coset_words(C.N, T.it[i].logD));
  return (size_t)words * sizeof(u64);
}

}  // namespace

cudaError_t configure_coset_kernels() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f, int bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
#define HE_SET_COSET(LN)                                                                      \
  set((const void*)k_coset_fwd_multi_t<LN>, 2 * ((1 << LN) + (1 << LN) / 16) * (int)sizeof(u64)); \
  set((const void*)k_coset_inv_multi_t<LN>, 2 * ((1 << LN) + (1 << LN) / 16) * (int)sizeof(u64)); \
  set((const void*)k_coset_encode_t<LN>, 2 * ((1 << LN) + (1 << LN) / 16) * (int)sizeof(u64));
  HE_COSET_LOGNS(HE_SET_COSET)
#undef HE_SET_COSET
  return e;
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

}  // namespace he
