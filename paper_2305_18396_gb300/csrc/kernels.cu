// kernels.cu -- CUDA kernels of the GB300 HE library (sm_103a).
//
// Server hot path of Algorithm 1 (Sec. 3.1.1) on RNS BFV (Sec. 2.2):
//   k_encode_weights  pi_A of W^T blocks -> centred lift -> mod q_l -> NTT (resident)
//   k_ntt_forward     NTT of every input ciphertext polynomial (to workspace)
//   k_mac             slot-wise sum_J pt[I][J] * ct[Lb][J], lazy 3-column accumulation
//   k_intt_mask       inverse NTT of each output polynomial + re-mask of c0
// plus the test client (keygen / encrypt / decrypt / pack / unpack) and the
// server's unmask.  The polynomial product is NTT + slot-wise product + inverse
// NTT (footnote of Sec. 3.1.3).
#include <mutex>

#include "kernels.h"
#include "ntt.cuh"

namespace he {

__constant__ u64 c_gauss_cdt[2 * kGaussBound] = {
#include "gauss_cdt.inc"
};

constexpr int kNttThreads = 256;
constexpr int kMacThreads = 128;
constexpr int kMacTI = 4;  // output blocks I per thread
constexpr int kMacTB = 2;  // output blocks Lb per thread (x 2 ciphertext components)

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
  const PrimeConsts& P = C.p[poly % C.L];
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
  const PrimeConsts& P = C.p[poly % C.L];
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
  const PrimeConsts& P = C.p[poly % C.L];
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

// ------------------------------------------------------------------ test client

// sk[l][N] = NTT(s mod q_l), s_i = (u mod 3) - 1.
__global__ void __launch_bounds__(kNttThreads) k_keygen(u64 seed, u64* sk, const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u32 l = blockIdx.x;
  const PrimeConsts& P = C.p[l];
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
  const PrimeConsts& P = C.p[l];
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
    const PrimeConsts& P = C.p[l];
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
      const PrimeConsts& P = C.p[l];
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
__global__ void __launch_bounds__(kNttThreads) k_encode_weights(const u64* W, u32 k, u32 n, Blk b, u32 nJ, u64* pt,
                                                                const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  const u32 l = poly % C.L;
  const u32 IJ = (u32)(poly / C.L);
  const u32 I = IJ / nJ, J = IJ % nJ;
  const PrimeConsts& P = C.p[l];
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
  u64* d = pt + poly * C.N;
  for (u32 i = threadIdx.x; i < C.N; i += blockDim.x) d[i] = sm[i];
}

// Slot-wise multiply-accumulate.  Each thread owns one slot s of prime l and a
// kMacTI x kMacTB tile of output blocks (both components).  Operands < 2^50
// are split as x = x0 + 2^26 x1 (x0 < 2^26, x1 < 2^24) and the products summed
// in three 64-bit columns (one mad.wide.u32 per partial product; no carries
// for nJ <= 4096), reduced once per output.
__global__ void __launch_bounds__(kMacThreads) k_mac(const u64* __restrict__ ctN, const u64* __restrict__ pt,
                                                     u64* __restrict__ out, u32 nI, u32 nJ, u32 nLb, u32 tilesI,
                                                     const __grid_constant__ Consts C) {
  const u32 chunks = (C.N + kMacThreads - 1) / kMacThreads;
  const u32 s = (blockIdx.x % chunks) * kMacThreads + threadIdx.x;
  if (s >= C.N) return;
  const u32 tile = blockIdx.x / chunks;
  const u32 l = blockIdx.y;
  const PrimeConsts& P = C.p[l];
  const u32 I0 = (tile % tilesI) * kMacTI;
  const u32 B0 = (tile / tilesI) * kMacTB;
  const u64 N = C.N, L = C.L;
  constexpr u32 M26 = (1u << 26) - 1;

  u64 acc[kMacTI][kMacTB][2][3];
#pragma unroll
  for (int a = 0; a < kMacTI; ++a)
#pragma unroll
    for (int bb = 0; bb < kMacTB; ++bb)
#pragma unroll
      for (int c = 0; c < 2; ++c) acc[a][bb][c][0] = acc[a][bb][c][1] = acc[a][bb][c][2] = 0;

  for (u32 J = 0; J < nJ; ++J) {
    u32 x0[kMacTI], x1[kMacTI];
#pragma unroll
    for (int a = 0; a < kMacTI; ++a) {
      u32 I = I0 + a;
      u64 v = I < nI ? __ldg(pt + (((u64)I * nJ + J) * L + l) * N + s) : 0;
      x0[a] = (u32)v & M26;
      x1[a] = (u32)(v >> 26);
    }
    u32 y0[kMacTB][2], y1[kMacTB][2];
#pragma unroll
    for (int bb = 0; bb < kMacTB; ++bb) {
      u32 Lb = B0 + bb;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        u64 v = Lb < nLb ? __ldg(ctN + ((((u64)Lb * nJ + J) * 2 + c) * L + l) * N + s) : 0;
        y0[bb][c] = (u32)v & M26;
        y1[bb][c] = (u32)(v >> 26);
      }
    }
#pragma unroll
    for (int a = 0; a < kMacTI; ++a)
#pragma unroll
      for (int bb = 0; bb < kMacTB; ++bb)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          acc[a][bb][c][0] += (u64)x0[a] * y0[bb][c];
          acc[a][bb][c][1] += (u64)x0[a] * y1[bb][c];
          acc[a][bb][c][1] += (u64)x1[a] * y0[bb][c];
          acc[a][bb][c][2] += (u64)x1[a] * y1[bb][c];
        }
  }

#pragma unroll
  for (int a = 0; a < kMacTI; ++a)
#pragma unroll
    for (int bb = 0; bb < kMacTB; ++bb) {
      u32 I = I0 + a, Lb = B0 + bb;
      if (I >= nI || Lb >= nLb) continue;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        u64 r0 = reduce_word(acc[a][bb][c][0], P);
        u64 r1 = csub(mul_shoup(acc[a][bb][c][1], P.r26, P.r26_sh, P.q), P.q);
        u64 r2 = csub(mul_shoup(acc[a][bb][c][2], P.r52, P.r52_sh, P.q), P.q);
        out[((((u64)Lb * nI + I) * 2 + c) * L + l) * N + s] = add_mod(add_mod(r0, r1, P.q), r2, P.q);
      }
    }
}

// One block per output polynomial (o, c, l): inverse NTT; for c = 0 subtract
// round(q s_i / t) where s_i is the mask of output o (Algorithm 1, step 3).
__global__ void __launch_bounds__(kNttThreads) k_intt_mask(u64* out, u64 seed, const __grid_constant__ Consts C) {
  extern __shared__ u64 sm[];
  const u64 poly = blockIdx.x;
  const u32 l = poly % C.L;
  const u32 c = (poly / C.L) % 2;
  const u32 o = (u32)(poly / (2 * C.L));
  const PrimeConsts& P = C.p[l];
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
  set((const void*)k_ntt_inverse, one);
  set((const void*)k_poly_mul, two);
  set((const void*)k_keygen, one);
  set((const void*)k_encrypt, one);
  set((const void*)k_decrypt, all);
  set((const void*)k_encode_weights, one);
  set((const void*)k_intt_mask, one);
  return e;
}

cudaError_t launch_ntt_forward(const Consts& C, const u64* src, u64* dst, u64 npolys, cudaStream_t st) {
  if (npolys) k_ntt_forward<<<(unsigned)npolys, kNttThreads, poly_smem(C), st>>>(src, dst, C);
  return cudaGetLastError();
}

cudaError_t launch_ntt_inverse(const Consts& C, const u64* src, u64* dst, u64 npolys, cudaStream_t st) {
  if (npolys) k_ntt_inverse<<<(unsigned)npolys, kNttThreads, poly_smem(C), st>>>(src, dst, C);
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

cudaError_t launch_unmask(const Consts& C, u64 seed, u32 m, u32 n, Blk b, u32 nI, u64* share, cudaStream_t st) {
  u64 total = (u64)m * n;
  if (total) k_unmask<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(seed, m, n, b, nI, share, C);
  return cudaGetLastError();
}

cudaError_t launch_encode_weights(const Consts& C, const u64* W, u32 k, u32 n, Blk b, u32 nI, u32 nJ, u64* pt,
                                  cudaStream_t st) {
  u64 polys = (u64)nI * nJ * C.L;
  if (polys) k_encode_weights<<<(unsigned)polys, kNttThreads, poly_smem(C), st>>>(W, k, n, b, nJ, pt, C);
  return cudaGetLastError();
}

cudaError_t launch_mac(const Consts& C, const u64* ctN, const u64* pt, u64* out, u32 nI, u32 nJ, u32 nLb,
                       cudaStream_t st) {
  u32 tilesI = (nI + kMacTI - 1) / kMacTI, tilesB = (nLb + kMacTB - 1) / kMacTB;
  if ((u64)tilesI * tilesB == 0) return cudaGetLastError();
  u64 chunks = (C.N + kMacThreads - 1) / kMacThreads;
  dim3 grid((unsigned)(chunks * tilesI * tilesB), C.L);
  k_mac<<<grid, kMacThreads, 0, st>>>(ctN, pt, out, nI, nJ, nLb, tilesI, C);
  return cudaGetLastError();
}

cudaError_t launch_intt_mask(const Consts& C, u64* out, u64 out_cts, u64 seed, cudaStream_t st) {
  u64 polys = out_cts * 2 * C.L;
  if (polys) k_intt_mask<<<(unsigned)polys, kNttThreads, poly_smem(C), st>>>(out, seed, C);
  return cudaGetLastError();
}

}  // namespace he
