// coset.cuh -- the negacyclic polynomial product of Algorithm 1 step 3 (a_{I,J} times a
// ciphertext component, mod x^N + 1 and q_l) through the ring's cosets, for weight
// polynomials of small support.
//
// The footnote of Sec. 3.1.3 multiplies polynomials by NTT, slot-wise product, inverse NTT.
// A weight block of pi_A fills only its lowest n_b k_b coefficients, yet its NTT has N slots:
// the resident weights then cost N residues for n_b k_b values.  This file computes the same
// product with weights of 2D residues, D = max(8, n_b k_b rounded up to a power of two):
//
//  * x^N + 1 is the product of the G = N / D factors x^D - zeta_g, zeta_g the roots of
//    y^G = -1.  The first log2 G stages of the forward negacyclic NTT (Cooley-Tukey, twiddles
//    psi^{brev(2^s + g)}) reduce a ciphertext component b to its G residues
//    b_g = b mod (x^D - zeta_g), block g of length D, with zeta_g = psi^{brev(G/2 + g/2)} for
//    even g and its negative for odd g.
//  * a has degree < D, so a mod (x^D - zeta_g) = a for every g.  The product a b_g (degree
//    < 2D - 1) is unchanged by reduction mod x^{2D} + 1, so it is the slot-wise product of the
//    zero-padded length-2D negacyclic NTTs of a and b_g -- a transform that does not depend
//    on g.  Its twiddles psi_{4D}^{brev_{2D}(k)} equal the length-N table's psi^{brev(k)},
//    k < 2D.  The weights are stored as these 2D values; each ciphertext component becomes G
//    blocks of 2D values (2N in all).
//  * Summed over the k-blocks J in that domain (the multiply-accumulate), the inverse
//    length-2D transform gives the linear product c_g = lo + x^D hi, folded to
//    lo + zeta_g hi = c_g mod (x^D - zeta_g); the inverse of the first log2 G stages then
//    returns the N coefficients of the product mod x^N + 1.  The fold and the scale
//    (2N)^{-1} of the whole inverse are one step: with U, V the two inputs of the last
//    inverse butterfly (span D, twiddle w = psi^{-N/2}),
//        lo + zeta_g hi = (1 + zeta_g w) U + (1 - zeta_g w) V,
//    the per-coset factors (1 +- psi^{brev(k)} w) (2N)^{-1} read from a table (PrimeConsts
//    fold), swapped for odd g.
//
// The slot order of the length-2D transform is its natural Cooley-Tukey output order
// (slot s = h D + position in half h); the weights, the ciphertexts and the inverse use the
// same order, so no permutation is needed.  All functions here run on one residue
// polynomial (or one block of polynomials) per thread block, in shared memory, and are
// called by every thread of the block.
#pragma once

#include "he_common.cuh"
#include "ntt.cuh"

namespace he {

// log2 D of a product: D = max(8, next power of two of n_b k_b).
__host__ __device__ inline u32 coset_logD(u32 nbkb) {
  u32 d = 3;
  while ((1u << d) < nbkb) ++d;
  return d;
}

// Forward, first log2 G stages: a[0, N) in [0, q) (natural order) becomes the G residues
// b_g in blocks of D, values in [0, (1 + 2 log2 G) q).
__device__ __forceinline__ void coset_head_fwd(u64* a, u32 logN, u32 logG, const PrimeConsts& P) {
  const u32 half = 1u << (logN - 1);
  for (u32 s = 0; s < logG; ++s) {
    const u32 tlog = logN - 1 - s, t = 1u << tlog;
    for (u32 b = threadIdx.x; b < half; b += blockDim.x) {
      const u32 g = b >> tlog, j = (g << (tlog + 1)) + (b & (t - 1));
      const u32 widx = (1u << s) + g;
      const u64 w = __ldg(P.psi + widx), wsh = __ldg(P.psi_sh + widx);
      const u64 U = a[j], V = mul_shoup(a[j + t], w, wsh, P.q);
      a[j] = U + V;
      a[j + t] = U - V + P.two_q;
    }
    __syncthreads();
  }
}

// Zero-padded length-2D negacyclic NTT of each of the G blocks of A (block g = A[g D, g D + D),
// values below 2^60): store(g, s, v) receives slot s < 2D of block g, v in [0, q).  B is a
// work buffer of N words.  The first stage of the transform pairs each value with a zero
// and only copies it (both halves start as the block); the log2 D stages after it run on
// each half.  Synchronizes internally; A is unchanged.
template <class Store>
__device__ __forceinline__ void coset_tail_fwd(const u64* A, u64* B, u32 logN, u32 logD, const PrimeConsts& P,
                                               Store store) {
  const u32 N = 1u << logN, D = 1u << logD, half = N >> 1;
  for (u32 h = 0; h < 2; ++h) {
    for (u32 e = threadIdx.x; e < N; e += blockDim.x) B[e] = A[e];
    __syncthreads();
    for (u32 s = 1; s <= logD; ++s) {
      const u32 tlog = logD - s, t = 1u << tlog;
      for (u32 b = threadIdx.x; b < half; b += blockDim.x) {
        const u32 g = b >> (logD - 1), bl = b & ((D >> 1) - 1);
        const u32 lg = bl >> tlog, j = g * D + (lg << (tlog + 1)) + (bl & (t - 1));
        const u32 widx = (1u << s) + (h << (s - 1)) + lg;
        const u64 w = __ldg(P.psi + widx), wsh = __ldg(P.psi_sh + widx);
        const u64 U = B[j], V = mul_shoup(B[j + t], w, wsh, P.q);
        B[j] = U + V;
        B[j + t] = U - V + P.two_q;
      }
      __syncthreads();
    }
    for (u32 e = threadIdx.x; e < N; e += blockDim.x) store(e >> logD, (h << logD) + (e & (D - 1)), reduce_word(B[e], P));
    __syncthreads();
  }
}

// Inverse: A holds the slots [0, D) and B the slots [D, 2D) of every block g (A[g D + j] =
// slot j, B[g D + j] = slot D + j), values in [0, 2q).  Leaves in A the N coefficients of the
// polynomial whose forward transform those slots are (natural order), in [0, 2q).
__device__ __forceinline__ void coset_inverse(u64* A, u64* B, u32 logN, u32 logD, const PrimeConsts& P) {
  const u32 N = 1u << logN, D = 1u << logD, half = N >> 1, logG = logN - logD, G = 1u << logG;
  const u64 q = P.q, two_q = P.two_q;
  for (u32 s = logD; s >= 1; --s) {  // inverse of the length-2D transform, each half
    const u32 tlog = logD - s, t = 1u << tlog;
    for (u32 b = threadIdx.x; b < N; b += blockDim.x) {
      const u32 h = b >= half ? 1u : 0u, bb = b - h * half;
      const u32 g = bb >> (logD - 1), bl = bb & ((D >> 1) - 1);
      const u32 lg = bl >> tlog, j = g * D + (lg << (tlog + 1)) + (bl & (t - 1));
      const u32 widx = (1u << s) + (h << (s - 1)) + lg;
      u64* X = h ? B : A;
      const u64 w = __ldg(P.ipsi + widx), wsh = __ldg(P.ipsi_sh + widx);
      const u64 U = X[j], V = X[j + t];
      X[j] = csub(U + V, two_q);
      X[j + t] = mul_shoup(U - V + two_q, w, wsh, q);
    }
    __syncthreads();
  }
  for (u32 e = threadIdx.x; e < N; e += blockDim.x) {  // last butterfly + fold + (2N)^{-1}
    const u32 g = e >> logD;
    const u64* f = P.fold + 4 * ((G >> 1) + (g >> 1));
    const u32 o = (g & 1) ? 2 : 0;  // odd g: zeta_g = -psi^{brev(k)}, the factors swap
    A[e] = csub(mul_shoup(A[e], __ldg(f + o), __ldg(f + o + 1), q) + mul_shoup(B[e], __ldg(f + 2 - o), __ldg(f + 3 - o), q),
                two_q);
  }
  __syncthreads();
  for (u32 s = logG; s-- > 0;) {  // inverse of the first log2 G forward stages
    const u32 tlog = logN - 1 - s, t = 1u << tlog;
    for (u32 b = threadIdx.x; b < half; b += blockDim.x) {
      const u32 g = b >> tlog, j = (g << (tlog + 1)) + (b & (t - 1));
      const u32 widx = (1u << s) + g;
      const u64 w = __ldg(P.ipsi + widx), wsh = __ldg(P.ipsi_sh + widx);
      const u64 U = A[j], V = A[j + t];
      A[j] = csub(U + V, two_q);
      A[j + t] = mul_shoup(U - V + two_q, w, wsh, q);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- register-blocked forms
//
// For D <= 32 (the geometry of products of many rows per ciphertext) the transforms run
// like the library's register-blocked NTT (ntt.cuh, S = NttShape<log2 N, 4>, N / 16
// threads): the first log2 G stages are the forward NTT's register passes stopped after
// stage log2 G - 1; then each thread takes whole cosets (one half of a length-2D
// transform, D values) from shared memory into registers.  The inverse takes each
// coset's 2D slots into registers for the inverse length-2D transform and the fold, and
// runs the inverse NTT's register passes over the stages of span D .. N/2.  Same
// arithmetic as the functions above (lazy forward ranges below 2^56, inverse in [0, 2q)).

constexpr int kCosetFastMaxLogD = 5;

// Forward stages [S0, LOGG) as register passes of at most LOGR stages; values in sm
// (padded, natural order) before and after.
template <class S, int S0, int LOGG>
__device__ __forceinline__ void coset_head_passes(u64 (&x)[S::R], u64* sm, const PrimeConsts& P) {
  if constexpr (S0 < LOGG) {
    constexpr int RS = (LOGG - S0) < S::LOGR ? (LOGG - S0) : S::LOGR;
    fwd_load_smem<S, S0, RS>(x, sm);
    fwd_pass_regs<S, S0, RS>(x, P);
    fwd_store_smem<S, S0, RS>(x, sm);
    __syncthreads();
    coset_head_passes<S, S0 + RS, LOGG>(x, sm, P);
  }
}

// The zero-padded length-2D transforms of the G = N / D blocks in sm (padded layout): work
// item (h, g) -- half h of coset g -- per thread, consecutive threads on consecutive
// cosets.  store(g, slot, v), v in [0, q).
template <class S, int LOGD, class Store>
__device__ __forceinline__ void coset_tail_regs(const u64* sm, const PrimeConsts& P, Store&& store) {
  constexpr int D = 1 << LOGD;
  constexpr u32 G = S::N >> LOGD;
  const u64 q = P.q, four_q = 2 * P.two_q;
  for (u32 it = threadIdx.x; it < 2 * G; it += S::T) {
    const u32 h = it / G, g = it % G;
    u64 v[D];
#pragma unroll
    for (int j = 0; j < D; ++j) v[j] = sm[S::pad(g * D + j)];
#pragma unroll
    for (int s = 1; s <= LOGD; ++s) {
      const int t = D >> s;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        if (j & t) continue;
        const u32 widx = (1u << s) + (h << (s - 1)) + (u32)(j / (2 * t));
        const u64 w = __ldg(P.psi + widx), wsh = __ldg(P.psi_sh + widx);
        const u64 U = v[j], V = mul_shoup_lazy(v[j + t], w, wsh, q);
        v[j] = U + V;
        v[j + t] = U - V + four_q;
      }
    }
#pragma unroll
    for (int j = 0; j < D; ++j) store(g, (h << LOGD) + j, reduce_word(v[j], P));
  }
}

// Forward coset transform of one polynomial: load(e) -> coefficient e in [0, q) (coalesced),
// store(g, slot, v) as above.  sm: S::kSmemWords words.  blockDim.x == S::T.
template <class S, int LOGD, class Load, class Store>
__device__ __forceinline__ void coset_forward_fast(u64* sm, const PrimeConsts& P, Load&& load, Store&& store) {
#pragma unroll
  for (int i = 0; i < S::R; ++i) {
    const u32 e = threadIdx.x + S::T * i;
    sm[S::pad(e)] = load(e);
  }
  __syncthreads();
  u64 x[S::R];
  coset_head_passes<S, 0, S::kLogN - LOGD>(x, sm, P);
  coset_tail_regs<S, LOGD>(sm, P, store);
}

// Inverse stages of span 2^S0 .. N/2 as register passes (sm padded); the last pass leaves
// its values in x (inv_elem<S, S0, RS> layout) and returns that pass's first stage.
template <class S, int S0>
__device__ __forceinline__ void coset_inv_head_passes(u64 (&x)[S::R], u64* sm, const PrimeConsts& P) {
  constexpr int RS = (S::kLogN - S0) < S::LOGR ? (S::kLogN - S0) : S::LOGR;
  inv_load_smem<S, S0, RS>(x, sm);
  inv_pass_regs<S, S0, RS>(x, P);
  if constexpr (S0 + RS < S::kLogN) {
    inv_store_smem<S, S0, RS>(x, sm);
    __syncthreads();
    coset_inv_head_passes<S, S0 + RS>(x, sm, P);
  }
}
template <class S, int S0>
__host__ __device__ constexpr int coset_inv_last_s0() {
  constexpr int RS = (S::kLogN - S0) < S::LOGR ? (S::kLogN - S0) : S::LOGR;
  if constexpr (S0 + RS < S::kLogN) return coset_inv_last_s0<S, S0 + RS>();
  else return S0;
}

// Inverse coset transform of one output component: src[g 2D + slot] is the sum at slot
// `slot` of coset g, in [0, q) (src 16-byte aligned); store(e, v) <- coefficient e in
// [0, q) (each e once).  sm: S::kSmemWords words.  blockDim.x == S::T.
template <class S, int LOGD, class Store>
__device__ __forceinline__ void coset_inverse_fast(u64* sm, const PrimeConsts& P, const u64* __restrict__ src,
                                                   Store&& store) {
  constexpr int D = 1 << LOGD;
  constexpr u32 G = S::N >> LOGD;
  const u64 q = P.q, two_q = P.two_q;
  for (u32 g = threadIdx.x; g < G; g += S::T) {
    const u64* f = P.fold + 4 * ((G >> 1) + (g >> 1));
    const u32 o = (g & 1) ? 2 : 0;  // odd g: zeta_g = -psi^{brev(k)}, the factors swap
    const u64 fa = __ldg(f + o), fa_sh = __ldg(f + o + 1), fb = __ldg(f + 2 - o), fb_sh = __ldg(f + 3 - o);
#pragma unroll
    for (u32 h = 0; h < 2; ++h) {
      u64 v[D];
      const ulonglong2* sv = reinterpret_cast<const ulonglong2*>(src + ((u64)g << (LOGD + 1)) + (h << LOGD));
#pragma unroll
      for (int j = 0; j < D; j += 2) {
        const ulonglong2 t = sv[j >> 1];
        v[j] = t.x;
        v[j + 1] = t.y;
      }
#pragma unroll
      for (int s = LOGD; s >= 1; --s) {
        const int t = D >> s;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          if (j & t) continue;
          const u32 widx = (1u << s) + (h << (s - 1)) + (u32)(j / (2 * t));
          const u64 w = __ldg(P.ipsi + widx), wsh = __ldg(P.ipsi_sh + widx);
          const u64 U = v[j], V = v[j + t];
          v[j] = csub(U + V, two_q);
          v[j + t] = mul_shoup(U - V + two_q, w, wsh, q);
        }
      }
      if (h == 0) {  // parked in this thread's own words of sm until the second half is done
#pragma unroll
        for (int j = 0; j < D; ++j) sm[S::pad(g * D + j)] = v[j];
      } else {  // last butterfly of the length-2D inverse, fold by zeta_g, (2N)^{-1}
#pragma unroll
        for (int j = 0; j < D; ++j) {
          u64& y = sm[S::pad(g * D + j)];
          y = csub(mul_shoup(y, fa, fa_sh, q) + mul_shoup(v[j], fb, fb_sh, q), two_q);
        }
      }
    }
  }
  __syncthreads();
  u64 x[S::R];
  coset_inv_head_passes<S, LOGD>(x, sm, P);
  constexpr int S0L = coset_inv_last_s0<S, LOGD>();
  constexpr int RSL = S::kLogN - S0L;
#pragma unroll
  for (int hh = 0; hh < (S::R >> RSL); ++hh)
#pragma unroll
    for (int j = 0; j < (1 << RSL); ++j) store(inv_elem<S, S0L, RSL>(hh, j), csub(x[hh * (1 << RSL) + j], q));
}

// ---------------------------------------------------------------- register passes, D = 64, 128
//
// For cosets too long to hold in one thread, each half's length-D transform is a batched
// transform over all G cosets: the full NTT's register passes over the stages log2 G ..
// log2 N - 1 with the tail's twiddle indices (fwd_pass_regs / inv_pass_regs, TAILG / TAILD).
// Each half works on its own padded copy of the polynomial: 2 S::kSmemWords words.

constexpr int kCosetPassMinLogD = 6, kCosetPassMaxLogD = 7;

template <class S, int S0, int LOGG, class Store>
__device__ __forceinline__ void coset_tail_passes(u64 (&x)[S::R], u64* sm, const PrimeConsts& P, u32 h,
                                                  Store&& store) {
  constexpr int RS = (S::kLogN - S0) < S::LOGR ? (S::kLogN - S0) : S::LOGR;
  fwd_load_smem<S, S0, RS>(x, sm);
  fwd_pass_regs<S, S0, RS, LOGG>(x, P, h);
  if constexpr (S0 + RS < S::kLogN) {
    fwd_store_smem<S, S0, RS>(x, sm);
    __syncthreads();
    coset_tail_passes<S, S0 + RS, LOGG>(x, sm, P, h, store);
  } else {
    constexpr int LOGD = S::kLogN - LOGG;
#pragma unroll
    for (int hh = 0; hh < (S::R >> RS); ++hh)
#pragma unroll
      for (int j = 0; j < (1 << RS); ++j) {
        const u32 e = fwd_elem<S, S0, RS>(hh, j);
        store(e >> LOGD, (h << LOGD) + (e & ((1u << LOGD) - 1)), reduce_word(x[hh * (1 << RS) + j], P));
      }
  }
}

// Both halves of the zero-padded length-2D transforms of the G blocks in sm (padded, values
// below 2^56 after at most log2 G lazy stages); sm2: a second S::kSmemWords words.  sm is
// overwritten by the second half.
template <class S, int LOGD, class Store>
__device__ __forceinline__ void coset_tail_both(u64* sm, u64* sm2, const PrimeConsts& P, Store&& store) {
  constexpr int LOGG = S::kLogN - LOGD;
  for (u32 i = threadIdx.x; i < (u32)S::kSmemWords; i += S::T) sm2[i] = sm[i];
  __syncthreads();
  u64 x[S::R];
  coset_tail_passes<S, LOGG, LOGG>(x, sm2, P, 0u, store);
  coset_tail_passes<S, LOGG, LOGG>(x, sm, P, 1u, store);
}

template <class S, int LOGD, class Load, class Store>
__device__ __forceinline__ void coset_forward_passes(u64* sm, u64* sm2, const PrimeConsts& P, Load&& load,
                                                     Store&& store) {
#pragma unroll
  for (int i = 0; i < S::R; ++i) {
    const u32 e = threadIdx.x + S::T * i;
    sm[S::pad(e)] = load(e);
  }
  __syncthreads();
  u64 x[S::R];
  coset_head_passes<S, 0, S::kLogN - LOGD>(x, sm, P);
  coset_tail_both<S, LOGD>(sm, sm2, P, store);
}

template <class S, int S0, int LOGD>
__device__ __forceinline__ void coset_inv_tail_passes(u64 (&x)[S::R], u64* sm, const PrimeConsts& P, u32 h) {
  if constexpr (S0 < LOGD) {
    constexpr int RS = (LOGD - S0) < S::LOGR ? (LOGD - S0) : S::LOGR;
    inv_load_smem<S, S0, RS>(x, sm);
    inv_pass_regs<S, S0, RS, LOGD>(x, P, h);
    inv_store_smem<S, S0, RS>(x, sm);
    __syncthreads();
    coset_inv_tail_passes<S, S0 + RS, LOGD>(x, sm, P, h);
  }
}

// As coset_inverse_fast, for D = 2^LOGD too long for one thread: smA, smB: S::kSmemWords
// words each (the two halves), src 16-byte aligned.
template <class S, int LOGD, class Store>
__device__ __forceinline__ void coset_inverse_passes(u64* smA, u64* smB, const PrimeConsts& P,
                                                     const u64* __restrict__ src, Store&& store) {
  constexpr u32 D = 1u << LOGD, G = S::N >> LOGD;
  const u64 q = P.q, two_q = P.two_q;
  for (u32 e = 2 * threadIdx.x; e < 2 * (u32)S::N; e += 2 * S::T) {  // pairs of slots, coalesced
    const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(src + e);
    const u32 g = e >> (LOGD + 1), pos = e & (2 * D - 1);
    u64* half = pos < D ? smA : smB;
    half[S::pad(g * D + (pos & (D - 1)))] = t.x;
    half[S::pad(g * D + (pos & (D - 1)) + 1)] = t.y;
  }
  __syncthreads();
  u64 x[S::R];
  coset_inv_tail_passes<S, 0, LOGD>(x, smA, P, 0u);
  coset_inv_tail_passes<S, 0, LOGD>(x, smB, P, 1u);
  for (u32 e = threadIdx.x; e < (u32)S::N; e += S::T) {  // last butterfly + fold + (2N)^{-1}
    const u32 g = e >> LOGD;
    const u64* f = P.fold + 4 * ((G >> 1) + (g >> 1));
    const u32 o = (g & 1) ? 2 : 0;  // odd g: zeta_g = -psi^{brev(k)}, the factors swap
    u64& y = smA[S::pad(e)];
    y = csub(mul_shoup(y, __ldg(f + o), __ldg(f + o + 1), q) + mul_shoup(smB[S::pad(e)], __ldg(f + 2 - o), __ldg(f + 3 - o), q),
             two_q);
  }
  __syncthreads();
  coset_inv_head_passes<S, LOGD>(x, smA, P);
  constexpr int S0L = coset_inv_last_s0<S, LOGD>();
  constexpr int RSL = S::kLogN - S0L;
#pragma unroll
  for (int hh = 0; hh < (S::R >> RSL); ++hh)
#pragma unroll
    for (int j = 0; j < (1 << RSL); ++j) store(inv_elem<S, S0L, RSL>(hh, j), csub(x[hh * (1 << RSL) + j], q));
}

}  // namespace he

