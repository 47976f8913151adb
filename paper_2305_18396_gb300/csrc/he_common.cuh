// he_common.cuh -- shared device definitions of the GB300 HE library:
// parameter structs passed to kernels by value, 64-bit modular arithmetic on
// the 32-bit integer pipes, Philox4x32-10 and the error sampler.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace he {

typedef uint64_t u64;
typedef unsigned int u32;

constexpr int kMaxPrimes = 3;
constexpr int kGaussBound = 19;

// Philox counter "domain" word (third counter word) for each kind of draw.
constexpr u32 kDomainSecret = 1;
constexpr u32 kDomainUniform = 2;
constexpr u32 kDomainError = 3;
constexpr u32 kDomainMask = 4;
constexpr u32 kDomainFill = 7;  // timing data of the autotuner (never a key, error or mask)

// Per-prime constants.  "_sh" fields are Shoup companions w' = floor(w 2^64 / q).
struct PrimeConsts {
  u64 q;
  u64 two_q;
  u64 mu;          // floor(2^64 / q): Shoup companion of 1 (Barrett-style reduction of a word)
  u64 ninv, ninv_sh;   // N^{-1} mod q
  u64 tinv, tinv_sh;   // t^{-1} mod q
  u64 r25, r25_sh;     // 2^25 mod q
  u64 r32, r32_sh;     // 2^32 (below q)
  u64 r50, r50_sh;     // 2^50 mod q
  u64 r64, r64_sh;     // 2^64 mod q
  u64 crt, crt_sh;     // ((Q / q)^{-1} mod q), for decryption
  u64 theta_hi, theta_lo;  // floor(t 2^128 / q) as two words (decryption)
  u32 pw256_lo[13], pw256_hi[13];  // 256^d mod q (d < 13) as 32-bit halves (tensor-core MAC epilogue)
  u64 pw256_bias;                  // 2^24 sum_d 256^d mod q
  const u64* psi;      // psi^{brev(k)}, k < N       (forward twiddles)
  const u64* psi_sh;
  const u64* ipsi;     // psi^{-brev(k)}, k < N      (inverse twiddles)
  const u64* ipsi_sh;
  // coset products (coset.cuh): for k < N/2 the four words (1 + psi^{brev(k)} w) / (2N),
  // its Shoup companion, (1 - psi^{brev(k)} w) / (2N), its companion; w = psi^{-N/2}
  const u64* fold;
};

struct Consts {
  u32 N, logN, L, log2t;
  u32 logR;     // log2 of the values per thread of the register-blocked transforms (N >= 512)
  u64 tmask;    // t - 1
  u64 q_mod_t;  // (q_0 ... q_{L-1}) mod t
  PrimeConsts p[kMaxPrimes];
};

// ---------------------------------------------------------------- arithmetic

// x w - qh q mod 2^64 for the library's primes q = q1 2^32 + 1 (he_params_init accepts only
// q = 1 mod 2^32): the low 64 bits of qh q are qh + 2^32 ((qh mod 2^32) q1 mod 2^32), one
// 32-bit multiply instead of the three of a 64-bit product.
__device__ __forceinline__ u64 sub_qh_q(u64 xw, u64 qh, u64 q) {
  return xw - qh - ((u64)((u32)qh * (u32)(q >> 32)) << 32);
}

// x * w mod q up to one extra q: result in [0, 2q) for any x < 2^64, w < q < 2^63.
__device__ __forceinline__ u64 mul_shoup(u64 x, u64 w, u64 w_sh, u64 q) {
  return sub_qh_q(x * w, __umul64hi(x, w_sh), q);
}

// Shoup product with an estimated quotient, for the lazily reduced forward transforms:
// x < 2^56, w < q < 2^50, w_sh = floor(w 2^64 / q).  With x = x1 2^32 + x0 and
// w_sh = s1 2^32 + s0, the quotient floor(x w_sh / 2^64) is x1 s1 + floor(x1 s0 / 2^32)
// + floor(x0 s1 / 2^32) + (at most 2: the three dropped fractions, x0 s0 / 2^64 among
// them, sum to less than 3).  Taking the estimate leaves the result x w - qh q in
// [0, 4q) instead of Shoup's [0, 2q).
__device__ __forceinline__ u64 mul_shoup_lazy(u64 x, u64 w, u64 w_sh, u64 q) {
  const u32 x0 = (u32)x, x1 = (u32)(x >> 32), s0 = (u32)w_sh, s1 = (u32)(w_sh >> 32);
  const u64 qh = (u64)x1 * s1 + __umulhi(x1, s0) + __umulhi(x0, s1);
  return sub_qh_q(x * w, qh, q);
}

__device__ __forceinline__ u64 csub(u64 x, u64 b) { return x >= b ? x - b : x; }

// x mod q for any 64-bit x.
__device__ __forceinline__ u64 reduce_word(u64 x, const PrimeConsts& P) {
  return csub(mul_shoup(x, 1, P.mu, P.q), P.q);
}

__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) { return csub(a + b, q); }
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// round(q m / t) mod q_l for m in [0, t): with R = (q m) mod t,
// round(q m / t) = (q m - R) / t + [2R >= t]  and  (q m - R) / t = -R t^{-1} (mod q_l).
__device__ __forceinline__ u64 delta_residue(u64 m, const Consts& C, const PrimeConsts& P) {
  u64 R = (C.q_mod_t * m) & C.tmask;  // low log2t bits survive the 64-bit wrap
  u64 v = csub(mul_shoup(R, P.tinv, P.tinv_sh, P.q), P.q);
  v = v ? P.q - v : 0;
  u64 up = (2 * R > C.tmask) ? 1 : 0;  // 2R >= t
  return add_mod(v, up, P.q);
}

// ---------------------------------------------------------------- Philox4x32-10

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    u32 lo0 = 0xD2511F53u * x.x, hi0 = __umulhi(0xD2511F53u, x.x);
    u32 lo1 = 0xCD9E8D57u * x.z, hi1 = __umulhi(0xCD9E8D57u, x.z);
    x = make_uint4(hi1 ^ x.y ^ k.x, lo1, hi0 ^ x.w ^ k.y, lo0);
  }
  return x;
}

__device__ __forceinline__ uint4 draw(u64 seed, u32 coef, u32 obj, u32 domain, u32 lane) {
  return philox4x32_10(make_uint4(coef, obj, domain, lane), make_uint2((u32)seed, (u32)(seed >> 32)));
}

__device__ __forceinline__ u64 lo64(uint4 w) { return (u64)w.x | ((u64)w.y << 32); }
__device__ __forceinline__ u64 hi64(uint4 w) { return (u64)w.z | ((u64)w.w << 32); }

}  // namespace he
