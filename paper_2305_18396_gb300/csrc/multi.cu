// multi.cu -- one set of launches for a list of products of different shapes (different
// m, k, n, blockings, weights, output modes): the forward NTT of every product's inputs,
// the multiply-accumulate of every product, the inverse NTTs and the masks each run as a
// single grid over the union of all products' work.  A product descriptor table travels
// as a kernel parameter; each block finds its product by binary search over per-kernel
// prefix sums of block counts.
#include <algorithm>

#include "async.cuh"
#include "kernels.h"
#include "mac.cuh"
#include "mac_tc.cuh"
#include "mac_tcr.cuh"
#include "multi.h"
#include "multi_items.cuh"
#include "ntt.cuh"

namespace he {

namespace {

constexpr int kThreadsSmall = 256;

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
  if (e == cudaSuccess) e = configure_coset_kernels();
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

cudaError_t launch_c0_multi(const Consts& C, const MultiTable& T, u64 blocks, u32 c0_words, cudaStream_t st) {
  if (blocks) k_c0_multi<<<(unsigned)blocks, kThreadsSmall, (size_t)c0_words * sizeof(u64), st>>>(T, C);
  return cudaGetLastError();
}

}  // namespace he
