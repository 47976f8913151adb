// ntt.cuh -- block-level negacyclic NTT over one residue polynomial held in
// shared memory (the polynomial product of the footnote in Sec. 3.1.3 is
// NTT, slot-wise product, inverse NTT).
//
// Forward: Cooley-Tukey with the psi powers merged into the twiddles
// (psi^{brev(k)}), natural-order input, bit-reversed slot order out.
// Inverse: Gentleman-Sande with psi^{-brev(k)}, bit-reversed in, natural out,
// followed by the N^{-1} scaling.
//
// Lazy reduction: forward butterflies keep values in [0, q + 2 q s) after
// stage s (no conditional subtraction; q < 2^50 keeps 13 stages below 2^55);
// the inverse keeps [0, 2q).  Both return fully reduced values in [0, q).
#pragma once

#include "he_common.cuh"

namespace he {

// All threads of the block must call these (they synchronize internally).
// Input: a[0..N) in [0, q).  Output: a[0..N) in [0, q), slot j = a(psi^{2 brev(j) + 1}).
__device__ __forceinline__ void ntt_forward_smem(u64* a, u32 logN, const PrimeConsts& P) {
  const u32 half = 1u << (logN - 1);
  const u64 two_q = P.two_q, q = P.q;
  for (u32 s = 0; s < logN; ++s) {
    const u32 tlog = logN - 1 - s;  // butterfly span t = 2^tlog, groups m = 2^s
    const u32 t = 1u << tlog;
    for (u32 b = threadIdx.x; b < half; b += blockDim.x) {
      u32 g = b >> tlog;
      u32 j = (g << (tlog + 1)) + (b & (t - 1));
      u32 widx = (1u << s) + g;
      u64 w = __ldg(P.psi + widx), wsh = __ldg(P.psi_sh + widx);
      u64 U = a[j];
      u64 V = mul_shoup(a[j + t], w, wsh, q);
      a[j] = U + V;
      a[j + t] = U - V + two_q;
    }
    __syncthreads();
  }
  const u32 N = 1u << logN;
  for (u32 i = threadIdx.x; i < N; i += blockDim.x) a[i] = reduce_word(a[i], P);
  __syncthreads();
}

// Input: a[0..N) in [0, 2q), slot order of ntt_forward_smem.  Output: coefficients in [0, q).
__device__ __forceinline__ void ntt_inverse_smem(u64* a, u32 logN, const PrimeConsts& P) {
  const u32 half = 1u << (logN - 1);
  const u64 two_q = P.two_q, q = P.q;
  for (u32 s = 0; s < logN; ++s) {
    const u32 tlog = s;  // span t = 2^s, groups h = N / 2t
    const u32 t = 1u << tlog;
    const u32 h = half >> s;
    for (u32 b = threadIdx.x; b < half; b += blockDim.x) {
      u32 g = b >> tlog;
      u32 j = (g << (tlog + 1)) + (b & (t - 1));
      u32 widx = h + g;
      u64 w = __ldg(P.ipsi + widx), wsh = __ldg(P.ipsi_sh + widx);
      u64 U = a[j], V = a[j + t];
      a[j] = csub(U + V, two_q);
      a[j + t] = mul_shoup(U - V + two_q, w, wsh, q);
    }
    __syncthreads();
  }
  const u32 N = 1u << logN;
  for (u32 i = threadIdx.x; i < N; i += blockDim.x) a[i] = csub(mul_shoup(a[i], P.ninv, P.ninv_sh, q), q);
  __syncthreads();
}

}  // namespace he
