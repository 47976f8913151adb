// kernels.cu -- CUDA kernels of the GB300 HE library (sm_103a).
//
// Server hot path of Algorithm 1 (Sec. 3.1.1) on RNS BFV (Sec. 2.2):
//   k_encode_weights  pi_A of W^T blocks -> centred lift -> mod q_l -> NTT (resident)
//   k_ntt_forward     NTT of every input ciphertext polynomial (to workspace)
//   k_mac             slot-wise sum_J pt[I][J] * ct[Lb][J]: bulk-copy pipeline, Karatsuba lazy accumulation
//   k_intt_mask       inverse NTT of each output polynomial + re-mask of c0
// plus the test client (keygen / encrypt / decrypt / pack / unpack) and the
// server's unmask.  The polynomial product is NTT + slot-wise product + inverse
// NTT (footnote of Sec. 3.1.3).
#include <algorithm>
#include <mutex>

#include "async.cuh"
#include "kernels.h"
#include "mac.cuh"
#include "mac_tc.cuh"
#include "ntt.cuh"

namespace he {

__constant__ u64 c_gauss_cdt[2 * kGaussBound] = {
#include "gauss_cdt.inc"
};

constexpr int kNttThreads = 256;

// a * b mod q for a, b < q < 2^50 (128-bit product folded with 2^64 mod q).
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const PrimeConsts& P) {
  u64 lo = a * b, hi = __umul64hi(a, b);
  u64 r_hi = csub(mul_shoup(hi, P.r64, P.r64_sh, P.q), P.q);
  return add_mod(r_hi, reduce_word(lo, P), P.q);
}

__device__ __forceinline__ u64 signed_to_residue(long long v, u64 q) { return v >= 0 ? (u64)v : q - (u64)(-v); }

// ------------------------------------------------------------------ NTT of independent polys

// Polys laid out [npolys][N]; poly p uses prime p % L.
__global__ void __launch_bounds__(kNttThreads) k_ntt_forward(const u64* src, u64* dst,
                                                             const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  const PrimeConsts P = C.p[poly % C.L];
  const u64* s = src + poly * C.N;
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) sm[i] = s[i];
  __syncthreads();
  ntt_forward_smem(sm, C.logN, P);
  u64* d = dst + poly * C.N;
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) d[i] = sm[i];
}

__global__ void __launch_bounds__(kNttThreads) k_ntt_inverse(const u64* src, u64* dst,
                                                             const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  const PrimeConsts P = C.p[poly % C.L];
  const u64* s = src + poly * C.N;
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) sm[i] = s[i];
  __syncthreads();
  ntt_inverse_smem(sm, C.logN, P);
  u64* d = dst + poly * C.N;
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) d[i] = sm[i];
}

__global__ void __launch_bounds__(kNttThreads) k_poly_mul(const u64* a, const u64* b, u64* c,
                                                          const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  u64* sa = sm;
  u64* sb = sm + C.N;
  const u64 poly = blockIdx.x;
  const PrimeConsts P = C.p[poly % C.L];
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) {
    sa[i] = a[poly * C.N + i];
    sb[i] = b[poly * C.N + i];
  }
  __syncthreads();
  ntt_forward_smem(sa, C.logN, P);
  ntt_forward_smem(sb, C.logN, P);
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) sa[i] = mul_mod(sa[i], sb[i], P);
  __syncthreads();
  ntt_inverse_smem(sa, C.logN, P);
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) c[poly * C.N + i] = sa[i];
}

// Forward NTT of matmul inputs for N < 512 into the slot-chunked layout (see mac.cuh).


__global__ void __launch_bounds__(kNttThreads) k_ntt_forward_mm_small(const u64* src, u64* ctN, u32 nJ, u32 nLb,
                                                                      const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  const u64 item_polys = (u64)nLb * nJ * 2 * C.L;
  const u64 item = poly / item_polys, local = poly % item_polys;
  const u32 l = local % C.L;
  const u32 c = (local / C.L) % 2;
  const u32 LbJ = (u32)(local / (2 * C.L));
  const u32 Lb = LbJ / nJ, J = LbJ % nJ;
  const PrimeConsts P = C.p[l];
  u64* dst = ctN + item * item_polys * C.N;
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) sm[i] = src[poly * C.N + i];
  __syncthreads();
  ntt_forward_smem(sm, C.logN, P);
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x)
    dst[chunked_index((u64)Lb * 2 + c, J, l, i, nJ, C.L, C.N)] = split_word(sm[i]);
}

// Register-blocked versions for N >= 512 (blockDim = NttShape<LOGN, LOGR>::T).
template <int LOGN, int LOGR>
__global__ void __launch_bounds__(NttShape<LOGN, LOGR>::T, NttShape<LOGN, LOGR>::kMinBlocks) k_ntt_forward_t(const u64* src, u64* dst,
                                                                     const __grid_constant__ Consts C) {
  using S = NttShape<LOGN, LOGR>;
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  const PrimeConsts P = C.p[poly % C.L];
  const u64* s = src + poly * S::N;
  u64* d = dst + poly * S::N;
  ntt_forward_block<S>(sm, P, [&](u32 e) { return s[e]; }, [&](u32 e, u64 v) { d[e] = v; });
}

template <int LOGN, int LOGR>
__global__ void __launch_bounds__(NttShape<LOGN, LOGR>::T, NttShape<LOGN, LOGR>::kMinBlocks) k_ntt_inverse_t(const u64* src, u64* dst,
                                                                     const __grid_constant__ Consts C) {
  using S = NttShape<LOGN, LOGR>;
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  const PrimeConsts P = C.p[poly % C.L];
  const u64* s = src + poly * S::N;
  u64* d = dst + poly * S::N;
  ntt_inverse_block<S>(sm, P, [&](u32 e) { return s[e]; }, [&](u32 e, u64 v) { d[e] = v; });
}

// ------------------------------------------------------------------ test client

// sk[l][N] = NTT(s mod q_l), s_i = (u mod 3) - 1.
__global__ void __launch_bounds__(kNttThreads) k_keygen(u64 seed, u64* sk, const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u32 l = blockIdx.x;
  const PrimeConsts P = C.p[l];
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) {
    long long v = (long long)(lo64(draw(seed, i, 0, kDomainSecret, 0)) % 3ull) - 1;
    sm[i] = signed_to_residue(v, P.q);
  }
  __syncthreads();
  ntt_forward_smem(sm, C.logN, P);
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) sk[(u64)l * C.N + i] = sm[i];
}

__device__ __forceinline__ long long gauss_from_draw(u64 u) {
  long long v = -kGaussBound;
#pragma unroll
  for (int j = 0; j < 2 * kGaussBound; ++j) v += (u >= c_gauss_cdt[j]) ? 1 : 0;
  return v;
}

// One block per (ciphertext j, prime l): c1 = a, c0 = -a s + e + Delta(m).
__global__ void __launch_bounds__(kNttThreads) k_encrypt(const u64* sk, const u64* plain, u64 seed, u64* ct,
                                                         const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u32 j = blockIdx.x / C.L, l = blockIdx.x % C.L;
  const PrimeConsts P = C.p[l];
  const u64 N = C.N;
  u64* c0 = ct + ((u64)j * 2 * C.L + l) * N;
  u64* c1 = ct + ((u64)j * 2 * C.L + C.L + l) * N;
  for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
    uint4 w = draw(seed, i, j, kDomainUniform, l);
    u64 hi = csub(mul_shoup(hi64(w), P.r64, P.r64_sh, P.q), P.q);
    u64 a = add_mod(hi, reduce_word(lo64(w), P), P.q);
    c1[i] = a;
    sm[i] = a;
  }
  __syncthreads();
  ntt_forward_smem(sm, C.logN, P);
  for (u32 i = threadIdx.x; i < N; i += blockDim.x) sm[i] = mul_mod(sm[i], sk[(u64)l * N + i], P);
  __syncthreads();
  ntt_inverse_smem(sm, C.logN, P);
  for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
    long long e = gauss_from_draw(lo64(draw(seed, i, j, kDomainError, 0)));
    u64 m = plain[(u64)j * N + i] & C.tmask;
    u64 v = sub_mod(signed_to_residue(e, P.q), sm[i], P.q);
    c0[i] = add_mod(v, delta_residue(m, C, P), P.q);
  }
}

// One block per ciphertext: x_l = c0 + c1 s (all primes in shared memory), then
// m = round(t x / q) mod t via  t x / q = sum_l t y_l / q_l (mod t),
// y_l = x_l ((q / q_l)^{-1} mod q_l), with t / q_l as a 128-bit fraction.
__global__ void __launch_bounds__(kNttThreads) k_decrypt(const u64* sk, const u64* ct, u64* plain, int* budget,
                                                         const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  __shared__ u64 red[kNttThreads / 32];
  const u32 j = blockIdx.x;
  const u64 N = C.N;
  for (u32 l = 0; l < C.L; ++l) {
    const PrimeConsts P = C.p[l];
    u64* x = sm + (u64)l * N;
    const u64* c0 = ct + ((u64)j * 2 * C.L + l) * N;
    const u64* c1 = ct + ((u64)j * 2 * C.L + C.L + l) * N;
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) x[i] = c1[i];
    __syncthreads();
    ntt_forward_smem(x, C.logN, P);
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) x[i] = mul_mod(x[i], sk[(u64)l * N + i], P);
    __syncthreads();
    ntt_inverse_smem(x, C.logN, P);
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) x[i] = add_mod(x[i], c0[i], P.q);
    __syncthreads();
  }
  u64 worst = 0;
  for (u32 i = threadIdx.x; i < N; i += blockDim.x) {
    u64 ip = 0, fh = 0, fl = 0;  // integer part, fraction (2^-64 and 2^-128 words)
    for (u32 l = 0; l < C.L; ++l) {
      const PrimeConsts P = C.p[l];
      u64 y = csub(mul_shoup(sm[(u64)l * N + i], P.crt, P.crt_sh, P.q), P.q);
      u64 l1 = y * P.theta_lo, h1 = __umul64hi(y, P.theta_lo);
      u64 l2 = y * P.theta_hi, h2 = __umul64hi(y, P.theta_hi);
      u64 mid = l2 + h1;
      u64 carry = mid < l2 ? 1 : 0;
      ip += h2 + carry;
      u64 nfl = fl + l1;
      u64 c2 = nfl < fl ? 1 : 0;
      fl = nfl;
      u64 nfh = fh + mid;
      u64 c3 = nfh < fh ? 1 : 0;
      u64 nfh2 = nfh + c2;
      c3 += nfh2 < nfh ? 1 : 0;
      fh = nfh2;
      ip += c3;
    }
    u64 up = fh >> 63;
    plain[(u64)j * N + i] = (ip + up) & C.tmask;
    u64 d = up ? (0ull - fh) : fh;  // distance to the nearest integer, 2^-64 units
    worst = d > worst ? d : worst;
  }
  for (int off = 16; off; off >>= 1) {
    u64 o = __shfl_xor_sync(0xffffffffu, worst, off);
    worst = o > worst ? o : worst;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = worst;
  __syncthreads();
  if (threadIdx.x == 0 && budget) {
    for (u32 w = 1; w < blockDim.x / 32; ++w) worst = red[w] > worst ? red[w] : worst;
    int b = worst == 0 ? 63 : __clzll((long long)worst) - ((worst & (worst - 1)) ? 1 : 0);
    budget[j] = b;
  }
}

// pi_B: polys[Lb * nJ + J][l n_b k_b + j] = X[Lb m_b + l][J k_b + j].
__global__ void k_pack(const u64* X, u32 m, u32 k, Blk b, u32 nJ, u64 total, u64* polys,
                       const __grid_constant__ Consts C) {
  const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const u32 poly = (u32)(e >> C.logN), p = (u32)(e & (C.N - 1));
  const u32 Lb = poly / nJ, J = poly % nJ;
  const u32 nk = b.n_b * b.k_b;
  const u32 l = p / nk, j = p % nk;
  u64 v = 0;
  if (l < b.m_b && j < b.k_b) {
    u32 row = Lb * b.m_b + l, col = J * b.k_b + j;
    if (row < m && col < k) v = X[(u64)row * k + col] & C.tmask;
  }
  polys[e] = v;
}

// pi_C^{-1}: share[Lb m_b + l][I n_b + i] = dec[Lb nI + I][l n_b k_b + i k_b + k_b - 1].
__global__ void k_unpack(const u64* dec, u32 m, u32 n, Blk b, u32 nI, u64* share, const __grid_constant__ Consts C) {
  const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (u64)m * n) return;
  const u32 row = (u32)(e / n), col = (u32)(e % n);
  const u32 Lb = row / b.m_b, l = row % b.m_b, I = col / b.n_b, i = col % b.n_b;
  const u64 coef = (u64)l * b.n_b * b.k_b + (u64)i * b.k_b + b.k_b - 1;
  share[e] = dec[((u64)Lb * nI + I) * C.N + coef] & C.tmask;
}

// Server share pi_C^{-1}(s): the mask coefficient at the decode position.
__global__ void k_unmask(u64 seed, u32 m, u32 n, Blk b, u32 nI, u64* share, const __grid_constant__ Consts C) {
  const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (u64)m * n) return;
  const u32 row = (u32)(e / n), col = (u32)(e % n);
  const u32 Lb = row / b.m_b, l = row % b.m_b, I = col / b.n_b, i = col % b.n_b;
  const u32 coef = l * b.n_b * b.k_b + i * b.k_b + b.k_b - 1;
  share[e] = lo64(draw(seed, coef, Lb * nI + I, kDomainMask, 0)) & C.tmask;
}

// ------------------------------------------------------------------ server hot path

// pi_A: a_{I,J}[i k_b + k_b - 1 - j] = W[J k_b + j][I n_b + i], centred lift, mod q_l, NTT.
// pt layout [nI][nJ][L][N]; one block per (I, J, l).
__global__ void __launch_bounds__(kNttThreads) k_encode_weights(const u64* W, u32 k, u32 n, Blk b, u32 nI, u32 nJ, u64* pt,
                                                                const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u64 item_polys = (u64)nI * nJ * C.L;
  const u64 item = blockIdx.x / item_polys, poly = blockIdx.x % item_polys;
  W += item * k * n;
  pt += item * item_polys * C.N;
  const u32 l = poly % C.L;
  const u32 IJ = (u32)(poly / C.L);
  const u32 I = IJ / nJ, J = IJ % nJ;
  const PrimeConsts P = C.p[l];
  const u32 nk = b.n_b * b.k_b;
  const u64 half_t = (C.tmask >> 1) + 1;
  for (u32 p = threadIdx.x; p < C.N; p += blockDim.x) {
    u64 v = 0;
    if (p < nk) {
      u32 i = p / b.k_b, j = b.k_b - 1 - p % b.k_b;
      u32 row = J * b.k_b + j, col = I * b.n_b + i;
      if (row < k && col < n) {
        u64 w = W[(u64)row * n + col] & C.tmask;
        v = w >= half_t ? P.q - (C.tmask + 1 - w) : w;  // centred lift [-t/2, t/2)
      }
    }
    sm[p] = v;
  }
  __syncthreads();
  ntt_forward_smem(sm, C.logN, P);
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) pt[chunked_index(I, J, l, i, nJ, C.L, C.N)] = split_word(sm[i]);
}

template <int LOGN, int LOGR>
__global__ void __launch_bounds__(NttShape<LOGN, LOGR>::T, NttShape<LOGN, LOGR>::kMinBlocks) k_encode_weights_t(const u64* W, u32 k, u32 n, Blk b, u32 nI,
                                                                        u32 nJ, u32 tc, u64* pt, const __grid_constant__ Consts C) {
  using S = NttShape<LOGN, LOGR>;
  extern __shared__ u64 sm[];
  const u64 item_polys = (u64)nI * nJ * C.L;
  const u64 item = blockIdx.x / item_polys, poly = blockIdx.x % item_polys;
  const u32 nS = tc_stages(nJ);
  W += item * k * n;
  pt += item * (tc ? tc_weight_words(nI, nJ, C.L, S::N) : (u64)nI * nJ * C.L * S::N);
  const u32 l = poly % C.L;
  const u32 IJ = (u32)(poly / C.L);
  const u32 I = IJ / nJ, J = IJ % nJ;
  const PrimeConsts P = C.p[l];
  const u32 nk = b.n_b * b.k_b;
  const u64 half_t = (C.tmask >> 1) + 1;
  auto load = [&](u32 p) -> u64 {
    if (p >= nk) return 0;
    u32 i = p / b.k_b, j = b.k_b - 1 - p % b.k_b;
    u32 row = J * b.k_b + j, col = I * b.n_b + i;
    if (row >= k || col >= n) return 0;
    u64 w = W[(u64)row * n + col] & C.tmask;
    return w >= half_t ? P.q - (C.tmask + 1 - w) : w;  // centred lift [-t/2, t/2)
  };
  if (tc) {  // the weights' digit tiles (mac_tc.cuh): seven bf16 digits per residue
    uint8_t* const ptd = reinterpret_cast<uint8_t*>(pt);
    ntt_forward_block<S>(sm, P, load, [&](u32 e, u64 v) {
      const u64 u = v + 0x0080808080808080ull;
      uint8_t* grp = ptd + tc_weight_offset(I & ~7u, l, e, J >> 4, nI, nS, S::N);
#pragma unroll
      for (int p = 0; p < (int)kTcPlanes; ++p)
        *reinterpret_cast<uint16_t*>(grp + tc::tile_offset(I & 7, kTcJB * p + (J & 15), kTcAKBytes, 2)) =
            (uint16_t)(digit_f32_bits(u, p) >> 16);
    }, nk);
  }
  else
    ntt_forward_block<S>(sm, P, load,
                         [&](u32 e, u64 v) { pt[chunked_index(I, J, l, e, nJ, C.L, S::N)] = split_word(v); }, nk);
}

template <int LOGN, int LOGR>
__global__ void __launch_bounds__(NttShape<LOGN, LOGR>::T, NttShape<LOGN, LOGR>::kMinBlocks) k_intt_mask_t(u64* out, u64 out_cts, u64 seed,
                                                                   const __grid_constant__ Consts C) {
  using S = NttShape<LOGN, LOGR>;
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  const u64 item = poly / (out_cts * 2 * C.L);  // batch item: re-masked with seed + item
  seed += item;
  const u32 l = poly % C.L;
  const u32 c = (poly / C.L) % 2;
  const u32 o = (u32)((poly / (2 * C.L)) % out_cts);
  const PrimeConsts P = C.p[l];
  u64* d = out + poly * S::N;
  ntt_inverse_block<S>(sm, P, [&](u32 e) { return d[e]; }, [&](u32 e, u64 v) {
    if (c == 0) {
      u64 sv = lo64(draw(seed, e, o, kDomainMask, 0)) & C.tmask;
      v = sub_mod(v, delta_residue(sv, C, P), P.q);
    }
    d[e] = v;
  });
}

// Warp-specialized form (mac_tile_ws): M::kThreads consumer threads + one producer warp.
template <class M, int MINB>
__global__ void __launch_bounds__(M::kThreads + 32, MINB) k_mac_ws_t(const u64* __restrict__ ctN,
                                                                     const u64* __restrict__ pt, OutPlace out, u32 nI,
                                                                     u32 nJ, u32 nLb, u32 tilesR, int* err,
                                                                     const __grid_constant__ Consts C) {
  extern __shared__ __align__(128) u64 sm[];
  // tile-fastest: the blocks of one 32-slot chunk (all output tiles) run together, so the
  // operand rows of that chunk are re-read from L2 rather than DRAM
  const u32 tiles = tilesR * ((nI + M::kCols - 1) / M::kCols);
  const u32 tile = blockIdx.x % tiles;
  const u32 chunk = blockIdx.x / tiles;
  const u32 r0 = (tile % tilesR) * M::kRows, c0 = (tile / tilesR) * M::kCols;
  const u32 l = blockIdx.y % C.L;
  const u64 item = blockIdx.y / C.L;
  const u64 per_in = (u64)nLb * nJ * 2 * C.L * C.N, per_pt = (u64)nI * nJ * C.L * C.N;
  mac_tile_ws<M>(ctN + item * per_in, pt + item * per_pt, out, item * ((u64)nLb * nI), nI, nJ, nLb, r0, c0, chunk, l,
                 err, C, sm);
}

template <class M, int MINB>
cudaError_t launch_mac_ws_cfg(const Consts& C, const u64* ctN, const u64* pt, OutPlace out, u32 nI, u32 nJ, u32 nLb,
                              u32 batch, int* err, cudaStream_t st) {
  const u32 tilesR = (2 * nLb + M::kRows - 1) / M::kRows, tilesC = (nI + M::kCols - 1) / M::kCols;
  if ((u64)tilesR * tilesC * nJ * batch == 0) return cudaGetLastError();
  dim3 grid((unsigned)((u64)(C.N >> 5) * tilesR * tilesC), C.L * batch);
  k_mac_ws_t<M, MINB><<<grid, M::kThreads + 32, M::kSmemBytes, st>>>(ctN, pt, out, nI, nJ, nLb, tilesR, err, C);
  return cudaGetLastError();
}



// Forward NTT of the input ciphertexts of a product into the slot-chunked operand layout.
// Input poly p = ((Lb nJ + J) 2 + c) L + l of the wire format [Lb nJ + J][2][L][N].
template <int LOGN, int LOGR>
__global__ void __launch_bounds__(NttShape<LOGN, LOGR>::T, NttShape<LOGN, LOGR>::kMinBlocks) k_ntt_forward_mm_t(const u64* src, u64* ctN, u32 nJ, u32 nLb,
                                                                        u32 tc, const __grid_constant__ Consts C) {
  using S = NttShape<LOGN, LOGR>;
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  const u64 item_polys = (u64)nLb * nJ * 2 * C.L;
  const u64 item = poly / item_polys, local = poly % item_polys;
  const u32 l = local % C.L;
  const u32 c = (local / C.L) % 2;
  const u32 LbJ = (u32)(local / (2 * C.L));
  const u32 Lb = LbJ / nJ, J = LbJ % nJ;
  const PrimeConsts P = C.p[l];
  const u64* sp = src + poly * S::N;
  const u32 nS = tc_stages(nJ);
  u64* dst = ctN + item * (tc ? tc_words(2 * nLb, nJ, C.L, S::N) : (u64)nLb * nJ * 2 * C.L * S::N);
  const u64 row = (u64)Lb * 2 + c;
  if (tc)
    ntt_forward_block<S>(sm, P, [&](u32 e) { return sp[e]; },
                         [&](u32 e, u64 v) { dst[tc_index((u32)row, J, l, e, 2 * nLb, nS, S::N)] = v; });
  else
    ntt_forward_block<S>(sm, P, [&](u32 e) { return sp[e]; },
                         [&](u32 e, u64 v) { dst[chunked_index(row, J, l, e, nJ, C.L, S::N)] = split_word(v); });
}

// The tensor-core multiply-accumulate (mac_tc.cuh) of `batch` same-shape products: one block
// per SM works through units * batch work units (product-major).
__global__ void __launch_bounds__(kTcThreads, 1) k_mac_tc(const u64* __restrict__ ctN, const u64* __restrict__ pt,
                                                         OutPlace out, u32 nI, u32 nJ, u32 nLb, u64 units, u64 total,
                                                         int* err, const __grid_constant__ Consts C) {
  extern __shared__ __align__(128) uint8_t smem_tc[];
  __shared__ TcShared sh;
  const u64 per_in = tc_words(2 * nLb, nJ, C.L, C.N), per_pt = tc_weight_words(nI, nJ, C.L, C.N);
  auto get = [&](u64 g, TcWork& w) {
    const u64 item = g / units;
    tc_unit(g % units, C.N, nI, 2 * nLb, w);
    w.acc = nullptr;
    w.logG = 0;
    w.ctN = ctN + item * per_in;
    w.ptd = reinterpret_cast<const uint8_t*>(pt + item * per_pt);
    w.out = out;
    w.ct0 = item * ((u64)nLb * nI);
    w.nI = nI;
    w.nJ = nJ;
    w.nLb = nLb;
  };
  mac_tc_run(get, total, err, C, smem_tc, sh);
}

// Compact-output mode: inverse NTT of the c1 polynomials only, in place.  Ciphertext g's
// c1 for prime l sits at base + g * ct_stride + l * N.
template <int LOGN, int LOGR>
__global__ void __launch_bounds__(NttShape<LOGN, LOGR>::T, NttShape<LOGN, LOGR>::kMinBlocks) k_intt_c1_t(u64* base, u64 ct_stride,
                                                                 const __grid_constant__ Consts C) {
  using S = NttShape<LOGN, LOGR>;
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  u64* d = base + (poly / C.L) * ct_stride + (poly % C.L) * (u64)S::N;
  ntt_inverse_block<S>(sm, C.p[poly % C.L], [&](u32 e) { return d[e]; }, [&](u32 e, u64 v) { d[e] = v; });
}

__global__ void __launch_bounds__(kNttThreads) k_intt_c1_small(u64* base, u64 ct_stride,
                                                               const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  u64* d = base + (poly / C.L) * ct_stride + (poly % C.L) * (u64)C.N;
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) sm[i] = d[i];
  __syncthreads();
  ntt_inverse_smem(sm, C.logN, C.p[poly % C.L]);
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) d[i] = sm[i];
}

// Compact-output mode (Sec. 3.1.3, "Reducing the communication cost"): the client only
// decrypts the coefficients pi_C^{-1} reads, e = g k_b + k_b - 1, and decryption of
// coefficient e needs only (c0)_e; so c0 is inverse-transformed only at those e.  The
// Gentleman-Sande stages of span < k_b combine slots within groups of k_b; of their outputs
// only position k_b - 1 of each group feeds the wanted coefficients, so those stages keep
// one butterfly branch (k_b - 1 products per group), and the stages of span >= k_b run on
// the N / k_b surviving values.  The arithmetic on the kept branch is exactly that of the
// full inverse transform, so the kept coefficients are bit-identical to it.
// src: NTT-domain c0 of global ciphertext g, prime l at src + (g L + l) N.
// dst: compact c0 (N / k_b words per prime) at dst + g * ct_stride + l * (N / k_b); masked.
__global__ void __launch_bounds__(kNttThreads) k_intt_c0_targets(const u64* src, u64* dst, u64 ct_stride, u64 out_cts,
                                                                 u32 logkb, u64 seed, const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  const u32 l = poly % C.L;
  const u64 g_ct = poly / C.L;
  const u64 item = g_ct / out_cts;
  const u32 o = (u32)(g_ct % out_cts);
  ntt_inverse_c0_targets(src + poly * C.N, dst + g_ct * ct_stride + (u64)l * (C.N >> logkb), logkb, seed + item, o, l,
                         C, sm);
}

// One block per output polynomial (o, c, l): inverse NTT; for c = 0 subtract
// round(q s_i / t) where s_i is the mask of output o (Algorithm 1, step 3).
__global__ void __launch_bounds__(kNttThreads) k_intt_mask(u64* out, u64 out_cts, u64 seed,
                                                          const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  const u64 item = poly / (out_cts * 2 * C.L);  // batch item: re-masked with seed + item
  seed += item;
  const u32 l = poly % C.L;
  const u32 c = (poly / C.L) % 2;
  const u32 o = (u32)((poly / (2 * C.L)) % out_cts);
  const PrimeConsts P = C.p[l];
  u64* d = out + poly * C.N;
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) sm[i] = d[i];
  __syncthreads();
  ntt_inverse_smem(sm, C.logN, P);
  if (c == 0) {
    for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) {
      u64 sv = lo64(draw(seed, i, o, kDomainMask, 0)) & C.tmask;
      d[i] = sub_mod(sm[i], delta_residue(sv, C, P), P.q);
    }
  } else {
    for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) d[i] = sm[i];
  }
}

// ------------------------------------------------------------------ SM count of the current device

int device_sms() {
  static int cached[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
  if (!cached[dev]) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = sms > 0 ? sms : 1;
  }
  return cached[dev];
}

// ------------------------------------------------------------------ fixed scratch for he_matmul_noalloc

// File-scope device scratch used only by he_matmul_noalloc, for callers that cannot
// allocate device memory.  Every GPU that loads the library holds these bytes until
// the process exits.  Host code must not pass the symbol itself to a kernel (on the
// host it names a shadow variable, not device memory): it asks the runtime for the
// device address once per device, with that device current.
static __device__ __align__(256) u64 g_noalloc_scratch[kNoAllocScratchBytes / sizeof(u64)];

cudaError_t noalloc_scratch_address(int device, void** ptr) {
  static std::mutex mu;
  static void* addr[kMaxDevices] = {};
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // caller made `device` current
    if (e != cudaSuccess) return e;
    addr[device] = p;
  }
  *ptr = addr[device];
  return cudaSuccess;
}

// ------------------------------------------------------------------ launchers

static size_t poly_smem(const Consts& C) { return (size_t)C.N * sizeof(u64); }

// The attribute is per function and device, shared by every context: always raise it to the
// largest size any supported parameter set uses (N <= 8192, L * N <= 3 * 8192).
cudaError_t configure_kernels(const Consts&) {
  const int one = 8192 * (int)sizeof(u64), two = 2 * one, all = 3 * one;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f, int bytes) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  };
  set((const void*)k_ntt_forward, one);
  set((const void*)k_ntt_forward_mm_small, one);
  set((const void*)k_intt_c1_small, one);
  set((const void*)k_intt_c0_targets, two);
  set((const void*)k_ntt_inverse, one);
  set((const void*)k_poly_mul, two);
  set((const void*)k_keygen, one);
  set((const void*)k_encrypt, one);
  set((const void*)k_decrypt, all);
  set((const void*)k_encode_weights, one);
  set((const void*)k_intt_mask, one);
  set((const void*)k_mac_ws_t<MacProd, kMacMinBlocks>, (int)MacProd::kSmemBytes);
  set((const void*)k_mac_tc, (int)kTcSmem);
  if (e == cudaSuccess)  // two blocks per SM need the largest shared-memory carveout
    e = cudaFuncSetAttribute((const void*)k_mac_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
#define HE_SET_T(LN, LR, unused)                                                                    \
  {                                                                                                  \
    const int bytes = NttShape<LN, LR>::kSmemWords * (int)sizeof(u64);                               \
    set((const void*)k_ntt_forward_t<LN, LR>, bytes);                                                \
    set((const void*)k_ntt_inverse_t<LN, LR>, bytes);                                                \
    set((const void*)k_encode_weights_t<LN, LR>, bytes);                                             \
    set((const void*)k_ntt_forward_mm_t<LN, LR>, bytes);                                             \
    set((const void*)k_intt_mask_t<LN, LR>, bytes);                                                  \
    set((const void*)k_intt_c1_t<LN, LR>, bytes);                                                    \
  }
  HE_NTT_SHAPES(HE_SET_T, 0)
#undef HE_SET_T
  return e;
}

// Launch KERNEL<LOGN, LOGR> for the context's (log N, radix) with NttShape<LOGN, LOGR>
// threads and shared memory when N >= 512; a pair that is not built is an error.
#define HE_T_CASE(LN, LR, KERNEL, GRID, ST, ...)                                                          \
  case HE_NTT_KEY(LN, LR):                                                                                \
    KERNEL<LN, LR><<<GRID, NttShape<LN, LR>::T, NttShape<LN, LR>::kSmemWords * sizeof(u64), ST>>>(__VA_ARGS__); \
    break;
#define HE_DISPATCH_T(KERNEL, GRID, ST, ...)                                                              \
  switch (HE_NTT_KEY(C.logN, C.logR)) {                                                                   \
    HE_NTT_SHAPES(HE_T_CASE, KERNEL, GRID, ST, __VA_ARGS__)                                               \
    default: return cudaErrorInvalidValue;                                                                \
  }

cudaError_t launch_ntt_forward(const Consts& C, const u64* src, u64* dst, u64 npolys, cudaStream_t st) {
  if (!npolys) return cudaGetLastError();
  if (C.logN >= 9) {
    HE_DISPATCH_T(k_ntt_forward_t, (unsigned)npolys, st, src, dst, C)
  } else {
    k_ntt_forward<<<(unsigned)npolys, kNttThreads, poly_smem(C), st>>>(src, dst, C);
  }
  return cudaGetLastError();
}

cudaError_t launch_ntt_inverse(const Consts& C, const u64* src, u64* dst, u64 npolys, cudaStream_t st) {
  if (!npolys) return cudaGetLastError();
  if (C.logN >= 9) {
    HE_DISPATCH_T(k_ntt_inverse_t, (unsigned)npolys, st, src, dst, C)
  } else {
    k_ntt_inverse<<<(unsigned)npolys, kNttThreads, poly_smem(C), st>>>(src, dst, C);
  }
  return cudaGetLastError();
}

cudaError_t launch_poly_mul(const Consts& C, const u64* a, const u64* b, u64* c, u64 npolys, cudaStream_t st) {
  if (npolys) k_poly_mul<<<(unsigned)npolys, kNttThreads, 2 * poly_smem(C), st>>>(a, b, c, C);
  return cudaGetLastError();
}

cudaError_t launch_keygen(const Consts& C, u64 seed, u64* sk, cudaStream_t st) {
  k_keygen<<<C.L, kNttThreads, poly_smem(C), st>>>(seed, sk, C);
  return cudaGetLastError();
}

cudaError_t launch_encrypt(const Consts& C, const u64* sk, const u64* plain, u32 cnt, u64 seed, u64* ct,
                           cudaStream_t st) {
  if (cnt) k_encrypt<<<cnt * C.L, kNttThreads, poly_smem(C), st>>>(sk, plain, seed, ct, C);
  return cudaGetLastError();
}

cudaError_t launch_decrypt(const Consts& C, const u64* sk, const u64* ct, u32 cnt, u64* plain, int* budget,
                           cudaStream_t st) {
  if (cnt) k_decrypt<<<cnt, kNttThreads, C.L * poly_smem(C), st>>>(sk, ct, plain, budget, C);
  return cudaGetLastError();
}

cudaError_t launch_pack(const Consts& C, const u64* X, u32 m, u32 k, Blk b, u32 nJ, u32 nLb, u64* polys,
                        cudaStream_t st) {
  u64 total = (u64)nJ * nLb * C.N;
  if (total) k_pack<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(X, m, k, b, nJ, total, polys, C);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const Consts& C, const u64* dec, u32 m, u32 n, Blk b, u32 nI, u64* share,
                          cudaStream_t st) {
  u64 total = (u64)m * n;
  if (total) k_unpack<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(dec, m, n, b, nI, share, C);
  return cudaGetLastError();
}

// Pseudo-random data for timing runs (the autotuner): mode 0 fills residues mod q_l in the
// [..][L][N] layout (prime l = (e / N) mod L), mode 1 values in Z_t.
__global__ void k_fill_random(u64* dst, u64 words, u64 seed, int mode, const __grid_constant__ Consts C) {
  for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < words; e += (u64)gridDim.x * blockDim.x) {
    const u64 r = lo64(draw(seed, (u32)e, (u32)(e >> 32), kDomainFill, 0));
    dst[e] = mode == 0 ? r % C.p[(e / C.N) % C.L].q : r & C.tmask;
  }
}

cudaError_t launch_fill_random(const Consts& C, u64* dst, u64 words, u64 seed, int mode, cudaStream_t st) {
  if (words) k_fill_random<<<1216, 256, 0, st>>>(dst, words, seed, mode, C);
  return cudaGetLastError();
}

cudaError_t launch_unmask(const Consts& C, u64 seed, u32 m, u32 n, Blk b, u32 nI, u64* share, cudaStream_t st) {
  u64 total = (u64)m * n;
  if (total) k_unmask<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(seed, m, n, b, nI, share, C);
  return cudaGetLastError();
}

cudaError_t launch_encode_weights(const Consts& C, const u64* W, u32 k, u32 n, Blk b, u32 nI, u32 nJ, u32 batch,
                                  u32 tc, u64* pt, cudaStream_t st) {
  u64 polys = (u64)nI * nJ * C.L * batch;
  if (!polys) return cudaGetLastError();
  if (C.logN >= 9) {
    if (tc) {  // digit tiles: k-blocks past the last and rows past nI must read as zero digits
      cudaError_t e = cudaMemsetAsync(pt, 0, 8 * batch * tc_weight_words(nI, nJ, C.L, C.N), st);
      if (e != cudaSuccess) return e;
    }
    HE_DISPATCH_T(k_encode_weights_t, (unsigned)polys, st, W, k, n, b, nI, nJ, tc, pt, C)
  } else {
    if (tc) return cudaErrorInvalidValue;  // the tensor-core layout needs N >= 512
    k_encode_weights<<<(unsigned)polys, kNttThreads, poly_smem(C), st>>>(W, k, n, b, nI, nJ, pt, C);
  }
  return cudaGetLastError();
}


cudaError_t launch_mac(const Consts& C, const u64* ctN, const u64* pt, u64* out0, u64 stride0, u64* out1, u64 stride1,
                       u32 nI, u32 nJ, u32 nLb, u32 batch, int* err, cudaStream_t st) {
  OutPlace o;
  o.base[0] = out0;
  o.base[1] = out1;
  o.ct_stride[0] = stride0;
  o.ct_stride[1] = stride1;
  return launch_mac_ws_cfg<MacProd, kMacMinBlocks>(C, ctN, pt, o, nI, nJ, nLb, batch, err, st);
}

cudaError_t launch_mac_tc(const Consts& C, const u64* ctN, const u64* pt, u64* out0, u64 stride0, u64* out1,
                          u64 stride1, u32 nI, u32 nJ, u32 nLb, u32 batch, int* err, cudaStream_t st) {
  OutPlace o;
  o.base[0] = out0;
  o.base[1] = out1;
  o.ct_stride[0] = stride0;
  o.ct_stride[1] = stride1;
  const u64 units = tc_units(C.N, C.L, nI, 2 * nLb);
  if (!units || !nJ || !batch) return cudaGetLastError();
  if (C.logN < 9) return cudaErrorInvalidValue;
  const u64 total = units * batch, grid = std::min<u64>(total, (u64)device_sms());
  k_mac_tc<<<(unsigned)grid, kTcThreads, kTcSmem, st>>>(ctN, pt, o, nI, nJ, nLb, units, total, err, C);
  return cudaGetLastError();
}

cudaError_t launch_ntt_forward_mm(const Consts& C, const u64* ct_in, u64* ctN, u32 nJ, u32 nLb, u32 batch, u32 tc,
                                  cudaStream_t st) {
  const u64 polys = (u64)nLb * nJ * 2 * C.L * batch;
  if (!polys) return cudaGetLastError();
  if (C.logN >= 9) {
    HE_DISPATCH_T(k_ntt_forward_mm_t, (unsigned)polys, st, ct_in, ctN, nJ, nLb, tc, C)
  } else {
    if (tc) return cudaErrorInvalidValue;  // the tensor-core layout needs N >= 512
    k_ntt_forward_mm_small<<<(unsigned)polys, kNttThreads, poly_smem(C), st>>>(ct_in, ctN, nJ, nLb, C);
  }
  return cudaGetLastError();
}

cudaError_t launch_intt_mask(const Consts& C, u64* out, u64 out_cts, u32 batch, u64 seed, cudaStream_t st) {
  u64 polys = out_cts * 2 * C.L * batch;
  if (!polys) return cudaGetLastError();
  if (C.logN >= 9) {
    HE_DISPATCH_T(k_intt_mask_t, (unsigned)polys, st, out, out_cts, seed, C)
  } else {
    k_intt_mask<<<(unsigned)polys, kNttThreads, poly_smem(C), st>>>(out, out_cts, seed, C);
  }
  return cudaGetLastError();
}

}  // namespace he

namespace he {

cudaError_t launch_intt_c1(const Consts& C, u64* base, u64 ct_stride, u64 cts, cudaStream_t st) {
  const u64 polys = cts * C.L;
  if (!polys) return cudaGetLastError();
  if (C.logN >= 9) {
    HE_DISPATCH_T(k_intt_c1_t, (unsigned)polys, st, base, ct_stride, C)
  } else {
    k_intt_c1_small<<<(unsigned)polys, kNttThreads, poly_smem(C), st>>>(base, ct_stride, C);
  }
  return cudaGetLastError();
}

cudaError_t launch_intt_c0_targets(const Consts& C, const u64* src, u64* dst, u64 ct_stride, u64 out_cts, u32 batch,
                                   u32 logkb, u64 seed, cudaStream_t st) {
  const u64 polys = out_cts * batch * C.L;
  if (!polys) return cudaGetLastError();
  const size_t smem = (size_t)c0_smem_words(C.N, logkb) * sizeof(u64);
  k_intt_c0_targets<<<(unsigned)polys, kNttThreads, smem, st>>>(src, dst, ct_stride, out_cts, logkb, seed, C);
  return cudaGetLastError();
}

}  // namespace he

namespace he {

// Compact ciphertext [c0 at e = i k_b + k_b - 1: L x N/k_b][c1: L x N] -> full [2][L][N]
// with zeros at the c0 coefficients the compact form leaves out.
__global__ void k_expand_compact(const u64* src, u64 cnt, u32 logkb, u64* dst, const __grid_constant__ Consts C) {
  const u64 idx = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  const u64 N = C.N, L = C.L, Nc = N >> logkb;
  if (idx >= cnt * 2 * L * N) return;
  const u64 e = idx % N, l = (idx / N) % L, comp = (idx / (N * L)) % 2, g = idx / (2 * L * N);
  const u64* sct = src + g * L * (Nc + N);
  const u64 kb = 1ull << logkb;
  u64 v;
  if (comp == 1) v = sct[L * Nc + l * N + e];
  else v = (e % kb == kb - 1) ? sct[l * Nc + e / kb] : 0;
  dst[idx] = v;
}

cudaError_t launch_expand_compact(const Consts& C, const u64* src, u64 cnt, u32 logkb, u64* dst, cudaStream_t st) {
  const u64 total = cnt * 2 * C.L * C.N;
  if (total) k_expand_compact<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(src, cnt, logkb, dst, C);
  return cudaGetLastError();
}

// Wire-format check of he_ct_import: counts the words of cnt ciphertexts that are not
// below their prime and keeps the index of the first one (bad[0], bad[1]).  Per
// ciphertext: c0 with N >> logkb words per prime (all N for full ciphertexts, logkb = 0),
// then c1 with N words per prime.
__global__ void k_check_residues(const u64* ct, u64 cnt, u32 logkb, u64* bad, const __grid_constant__ Consts C) {
  const u64 N = C.N, L = C.L, Nc = N >> logkb, per = L * (Nc + N), total = cnt * per;
  for (u64 idx = (u64)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (u64)gridDim.x * blockDim.x) {
    const u64 w = idx % per;
    const u32 l = (u32)(w < L * Nc ? w / Nc : (w - L * Nc) / N);
    if (ct[idx] >= C.p[l].q) {
      atomicAdd((unsigned long long*)bad, 1ull);
      atomicMin((unsigned long long*)bad + 1, (unsigned long long)idx);
    }
  }
}

cudaError_t launch_check_residues(const Consts& C, const u64* ct, u64 cnt, u32 logkb, u64* bad, cudaStream_t st) {
  const u64 total = cnt * C.L * ((u64)(C.N >> logkb) + C.N);
  if (total) {
    const u64 blocks = std::min<u64>((total + 255) / 256, 152ull * 16);
    k_check_residues<<<(unsigned)blocks, 256, 0, st>>>(ct, cnt, logkb, bad, C);
  }
  return cudaGetLastError();
}

}  // namespace he

namespace he {

// Integer roofline probe: independent mad.wide.u32 chains (16 accumulators per thread,
// operands fixed per thread), the instruction the multiply-accumulate kernel is built on.
__global__ void __launch_bounds__(256) k_probe_mad_wide(u32 seed, int iters, u64* out) {
  u32 a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = (seed ^ (threadIdx.x * 2654435761u)) + 977u * i;
  const u32 b = seed | 1u;
  u64 acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < 16; ++i) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[i]) : "r"(a[i]), "r"(b));
  }
  u64 x = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) x ^= acc[i];
  out[(u64)blockIdx.x * blockDim.x + threadIdx.x] = x;
}

cudaError_t probe_mad_wide(int sms, u64* out, float* ms, cudaStream_t st) {
  const int blocks = sms * 8, iters = 2048;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  k_probe_mad_wide<<<blocks, 256, 0, st>>>(7u, 16, out);  // warm-up
  cudaEventRecord(e0, st);
  k_probe_mad_wide<<<blocks, 256, 0, st>>>(7u, iters, out);
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

}  // namespace he

namespace he {

// Failure-detection check: one thread waits, with the library's bounded wait, on an
// mbarrier that nothing arrives on; when the limit expires it records the error flag the
// host reads through he_device_status.  No copy is in flight and nothing else waits.
__global__ void k_wait_timeout_check(uint64_t limit_ns, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  mbar_init_fence();
  if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicExch(err, 1);
}

cudaError_t launch_wait_timeout_check(uint64_t limit_ns, int* err, cudaStream_t st) {
  k_wait_timeout_check<<<1, 32, 0, st>>>(limit_ns, err);
  return cudaGetLastError();
}

}  // namespace he
