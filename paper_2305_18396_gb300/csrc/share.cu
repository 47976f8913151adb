// share.cu -- the server-local side of the linear layers (Sec. 3.1.1): the products of
// the server's own plaintext shares, W<x>_1 + b for a fully connected layer and
// <X>_1 <Y>_1 for an attention product, mod t = 2^log2_t; and the accumulation of the
// server's mask shares pi_C^{-1}(s) of the Pi_MatMul calls into them.
//
// Arithmetic: residues mod 2^log2_t with 2^log2_t dividing 2^64, so every sum and product
// may wrap mod 2^64 and is reduced once at the end.  With a = a0 + 2^32 a1 and
// b = b0 + 2^32 b1 (32-bit halves), a b = a0 b0 + 2^32 (a0 b1 + a1 b0) (mod 2^64): one
// mad.wide.u32 into a 64-bit sum and two 32-bit multiply-adds into a 32-bit sum per term.
//
// Packed cross term (log2_t <= 37): only (a0 b1 + a1 b0) mod 32 reaches the result, and
// it equals (a0' b1 + a1 b0') mod 32 with a0' = a0 mod 32, b0' = b0 mod 32 and a1, b1 taken
// mod 32.  Packing A' = a0' + 2^16 a1 and B' = b0' + 2^16 b1 gives, mod 2^32,
// A' B' = a0' b0' + 2^16 (a0' b1 + a1 b0') + (a multiple of 2^32): one 32-bit multiply-add
// per term.  Over 16 terms the low field stays below 16 * 31^2 < 2^16 and the cross field
// below 16 * 2 * 31^2 < 2^16, so after each 16-term k-step the cross sum is read from
// bits 16..31 and the packed accumulator restarts.
#include "kernels.h"

namespace he {

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kTM = 4, kTN = 4, kShareThreads = 256;

__device__ __forceinline__ void mac_wrap(u64& lo, u32& mid, u64 a, u64 b) {
  const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
  asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(lo) : "r"(a0), "r"(b0));
  mid += a0 * b1 + a1 * b0;
}

// One 64 x 64 output tile over the k-range [kbeg, kend) of batch item blockIdx.z / splits.
// 16 x 16 threads; thread (tx, ty) owns rows ty + 16 i and columns tx + 16 j (i, j < 4), so
// the shared-memory reads of a k-step are a broadcast (A) and one contiguous 128-byte row
// per half-warp (B).  The next k-step's tiles are fetched into registers while the
// current one is multiplied.  Shared memory holds each word as (low half, packed
// cross-term word) when PACKED, else as it is.
// atomic = 0: out = (acc + bias + X W) mod t.  atomic = 1: out += X W (wrapping, a partial
// sum of a split k range; a finishing pass reduces mod t).
template <bool PACKED>
__global__ void __launch_bounds__(kShareThreads, 2) k_share_matmul(const u64* __restrict__ X, const u64* __restrict__ W,
                                                                u32 m, u32 k, u32 n, u32 kchunk, u32 splits,
                                                                u64 tmask, const u64* __restrict__ bias,
                                                                const u64* acc, u64* out, int atomic) {
  __shared__ u64 As[kBK][kBM + 1];  // k-major
  __shared__ u64 Bs[kBK][kBN];
  const u32 tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const u32 row0 = blockIdx.y * kBM, col0 = blockIdx.x * kBN;
  const u32 split = blockIdx.z % splits;
  const u64 item = blockIdx.z / splits;
  X += item * m * k;
  W += item * k * n;
  out += item * m * n;
  if (acc) acc += item * m * n;
  if (bias) bias += item * n;
  const u32 kbeg = split * kchunk, kend = min(k, kbeg + kchunk);

  u64 lo[kTM][kTN];
  u32 mid[kTM][kTN], mp[kTM][kTN];
#pragma unroll
  for (int i = 0; i < kTM; ++i)
#pragma unroll
    for (int j = 0; j < kTN; ++j) lo[i][j] = 0, mid[i][j] = 0, mp[i][j] = 0;

  u64 ra[4], rb[4];  // (64 x 16) and (16 x 64) tiles: 4 words per thread each
  auto fetch = [&](u32 k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const u32 idx = tid + kShareThreads * q;
      const u32 r = idx / kBK, c = idx % kBK, gr = row0 + r, gk = k0 + c;
      ra[q] = (gr < m && gk < kend) ? X[(u64)gr * k + gk] : 0;
      const u32 rr = idx / kBN, cc = idx % kBN, gk2 = k0 + rr, gc = col0 + cc;
      rb[q] = (gk2 < kend && gc < n) ? W[(u64)gk2 * n + gc] : 0;
    }
  };
  auto pack = [](u64 v) -> u64 {  // (low half, (v0 mod 32) + 2^16 (v1 mod 32))
    if (!PACKED) return v;
    const u64 c = (v & 31) | (((v >> 32) & 31) << 16);
    return (v & 0xffffffffull) | (c << 32);
  };
  auto stash = [&] {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const u32 idx = tid + kShareThreads * q;
      As[idx % kBK][idx / kBK] = pack(ra[q]);
      Bs[idx / kBN][idx % kBN] = pack(rb[q]);
    }
  };

  if (kbeg < kend) fetch(kbeg);
  for (u32 k0 = kbeg; k0 < kend; k0 += kBK) {
    __syncthreads();
    stash();
    __syncthreads();
    if (k0 + kBK < kend) fetch(k0 + kBK);
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      u64 a[kTM], b[kTN];
#pragma unroll
      for (int i = 0; i < kTM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < kTN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < kTM; ++i)
#pragma unroll
        for (int j = 0; j < kTN; ++j) {
          if (PACKED) {
            asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(lo[i][j]) : "r"((u32)a[i]), "r"((u32)b[j]));
            mp[i][j] += (u32)(a[i] >> 32) * (u32)(b[j] >> 32);
          } else {
            mac_wrap(lo[i][j], mid[i][j], a[i], b[j]);
          }
        }
    }
    if (PACKED) {
#pragma unroll
      for (int i = 0; i < kTM; ++i)
#pragma unroll
        for (int j = 0; j < kTN; ++j) mid[i][j] += mp[i][j] >> 16, mp[i][j] = 0;
    }
  }

#pragma unroll
  for (int i = 0; i < kTM; ++i) {
    const u32 r = row0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < kTN; ++j) {
      const u32 c = col0 + tx + 16 * j;
      if (r < m && c < n) {
        u64 v = lo[i][j] + ((u64)mid[i][j] << 32);
        u64* dst = out + (u64)r * n + c;
        if (atomic) {
          atomicAdd((unsigned long long*)dst, (unsigned long long)v);
        } else {
          if (bias) v += bias[c];
          if (acc) v += acc[(u64)r * n + c];
          *dst = v & tmask;
        }
      }
    }
  }
}

// Split-k set-up: out = acc + bias (wrapping; not yet reduced), over batch items of m x n.
__global__ void k_share_init(u64 total, u64 mn, u32 n, const u64* __restrict__ bias, const u64* acc, u64* out) {
  const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  u64 v = bias ? bias[(e / mn) * n + (e % mn) % n] : 0;
  if (acc) v += acc[e];
  out[e] = v;
}

__global__ void k_share_finish(u64 total, u64 tmask, u64* out) {
  const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < total) out[e] &= tmask;
}

// out (+)= pi_C^{-1}(s) of the masks of one Pi_MatMul (m x n product), or its transpose.
__global__ void k_unmask_acc(u64 seed, u32 m, u32 n, Blk b, u32 nI, int accumulate, int transpose, u64* out,
                             const __grid_constant__ Consts C) {
  const u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (u64)m * n) return;
  const u32 row = (u32)(e / n), col = (u32)(e % n);
  const u32 Lb = row / b.m_b, l = row % b.m_b, I = col / b.n_b, i = col % b.n_b;
  const u32 coef = l * b.n_b * b.k_b + i * b.k_b + b.k_b - 1;
  const u64 s = lo64(draw(seed, coef, Lb * nI + I, kDomainMask, 0)) & C.tmask;
  u64* dst = transpose ? out + (u64)col * m + row : out + e;
  *dst = ((accumulate ? *dst : 0) + s) & C.tmask;
}

}  // namespace

u32 share_matmul_splits(u32 m, u32 k, u32 n, u32 batch, int sms) {
  const u64 tiles = (u64)((n + kBN - 1) / kBN) * ((m + kBM - 1) / kBM) * batch;
  const u32 ksteps = (k + kBK - 1) / kBK;
  u64 want = tiles ? (2ull * (u64)sms + tiles - 1) / tiles : 1;
  want = want < 1 ? 1 : want;
  u64 cap = ksteps / 4 > 1 ? ksteps / 4 : 1;  // at least 4 k-steps per split
  const u64 zcap = 65535 / (batch ? batch : 1);  // grid z = splits x batch
  cap = cap < zcap ? cap : zcap;
  return (u32)(want < cap ? want : cap);
}

cudaError_t launch_share_matmul(const Consts& C, const u64* X, const u64* W, const u64* bias, const u64* acc, u32 m,
                                u32 k, u32 n, u32 batch, u32 splits, u64* out, cudaStream_t st) {
  const u64 total = (u64)m * n * batch;
  if (!total) return cudaGetLastError();
  splits = splits ? splits : 1;
  const u32 kchunk = ((((k + splits - 1) / splits) + kBK - 1) / kBK) * kBK;
  const dim3 grid((n + kBN - 1) / kBN, (m + kBM - 1) / kBM, splits * batch);
  const bool packed = C.log2t <= 37;  // the packed cross term covers bits 32..36 only
  auto mm = packed ? k_share_matmul<true> : k_share_matmul<false>;
  if (splits <= 1) {
    mm<<<grid, kShareThreads, 0, st>>>(X, W, m, k, n, k ? kchunk : 0, 1, C.tmask, bias, acc, out, 0);
    return cudaGetLastError();
  }
  const unsigned eb = (unsigned)((total + 255) / 256);
  k_share_init<<<eb, 256, 0, st>>>(total, (u64)m * n, n, bias, acc, out);
  mm<<<grid, kShareThreads, 0, st>>>(X, W, m, k, n, kchunk, splits, C.tmask, nullptr, nullptr, out, 1);
  k_share_finish<<<eb, 256, 0, st>>>(total, C.tmask, out);
  return cudaGetLastError();
}

cudaError_t launch_unmask_acc(const Consts& C, u64 seed, u32 m, u32 n, Blk b, u32 nI, int accumulate, int transpose,
                              u64* out, cudaStream_t st) {
  const u64 total = (u64)m * n;
  if (total)
    k_unmask_acc<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(seed, m, n, b, nI, accumulate, transpose, out, C);
  return cudaGetLastError();
}

}  // namespace he
