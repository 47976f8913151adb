// ntt.cuh -- block-level negacyclic NTT over one residue polynomial (the polynomial
// product of the footnote in Sec. 3.1.3 is NTT, slot-wise product, inverse NTT).
//
// Forward: Cooley-Tukey with the psi powers merged into the twiddles (psi^{brev(k)}),
// natural-order input, bit-reversed slot order out: slot j holds a(psi^{2 brev(j) + 1}).
// Inverse: Gentleman-Sande with psi^{-brev(k)}, bit-reversed in, natural out, times N^{-1}.
//
// Register-blocked form (N >= 512): a block of T = N / R threads, R = 2^LOGR values per
// thread.  The log2(N) butterfly stages are cut into passes of at most LOGR stages; in a
// pass every thread holds whole radix-2^RS groups in registers, runs the RS stages there and
// exchanges through shared memory only between passes (3 round trips for N = 4096 / 8192
// instead of one per stage).  Shared memory is padded (one word every 2^LOGR) so the
// contiguous groups of the innermost pass are free of bank conflicts.
//
// Lazy reduction: forward butterflies use a Shoup product with an estimated quotient
// (mul_shoup_lazy, result in [0, 4q)) and keep values in [0, q + 4 q s) after stage s (no
// conditional subtraction; q < 2^50 keeps 13 stages below 2^56); the inverse keeps
// [0, 2q).  Both produce fully reduced values in [0, q).
#pragma once

#include "he_common.cuh"

namespace he {

// ------------------------------------------------------------------ simple form (N < 512)

// All threads of the block call these.  Input a[0..N) in [0, q); output in [0, q).
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

// Input a[0..N) in [0, 2q), slot order of the forward transform.  Output in [0, q).
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

// ------------------------------------------------------------------ register-blocked form


// The radices built: 2^LOGR values per thread.  16 (LOGR = 4) everywhere; 8 and 32 as well
// at N = 4096 and 8192, where a context may select them (he_set_ntt_radix) or have them
// measured (he_autotune_ntt_radix).  Measured on GB300 (whole BERT layers, before the
// register caps below): 16 beats 8 and 32 at N = 4096 (3.28 ms vs 3.47 / 3.65 ms per
// layer) and 32 at N = 8192 (40.3 vs 45.0 ms per BERT-large layer: 128 instead of 242
// registers, twice the resident warps).
constexpr int kNttLogRDefault = 4;
__host__ __device__ constexpr bool ntt_radix_built(u32 logN, u32 logR) {
  return logN >= 9 && logN <= 13 && (logR == 4 || ((logN == 12 || logN == 13) && (logR == 3 || logR == 5)));
}
// X(LOGN, LOGR, ...) for every built pair (instantiation and dispatch lists).
#define HE_NTT_SHAPES(X, ...)                                                                          \
  X(9, 4, __VA_ARGS__) X(10, 4, __VA_ARGS__) X(11, 4, __VA_ARGS__) X(12, 3, __VA_ARGS__)             \
  X(12, 4, __VA_ARGS__) X(12, 5, __VA_ARGS__) X(13, 3, __VA_ARGS__) X(13, 4, __VA_ARGS__)           \
  X(13, 5, __VA_ARGS__)
// Dispatch key of a (log N, LOGR) pair.
#define HE_NTT_KEY(LOGN, LOGR) ((LOGN) * 8 + (LOGR))

template <int LOGN, int LOGR_ = kNttLogRDefault>
struct NttShape {
  static constexpr int kLogN = LOGN;
  static constexpr int N = 1 << LOGN;
  static constexpr int LOGR = LOGR_;
  static constexpr int R = 1 << LOGR;
  static constexpr int T = N / R;                   // threads per block
  // Minimum resident blocks per SM asked of the compiler, which caps registers per thread.
  // Measured on the BERT-base layer (N = 4096, 256 threads): with no cap the whole-layer
  // transforms take up to 170 registers and run one block per SM; three blocks (80
  // registers) make the step 3.178 ms against 3.555 with none and 3.217 with four (64
  // registers, where the transforms spill); with the estimated-quotient forward product
  // three blocks also beat four for the forward transforms alone (3.069 vs 3.091 ms).
  // At 512 threads (N = 8192) 128 registers already allow one block of 16 warps; 32 values
  // per thread need their registers (no cap).
  static constexpr int kMinBlocks = (LOGR <= 4 && T <= 256) ? 3 : 1;
  static constexpr int P = (LOGN + LOGR - 1) / LOGR;  // passes
  static constexpr int RS0 = LOGN - LOGR * (P - 1);   // stages of the outermost pass
  static constexpr int kSmemWords = N + (N >> LOGR);  // padded
  __device__ __forceinline__ static u32 pad(u32 e) { return e + (e >> LOGR); }
};

// One forward (Cooley-Tukey) pass over stages [S0, S0 + RS) on the R values in x:
// x[h * 2^RS + j] is element e = blk * 2^(LOGN - S0) + off + j * t_last of group
// g = tid + T * h, with t_last = 2^(LOGN - S0 - RS), blk = g / t_last, off = g % t_last.
// TAILG >= 0: the stages are those of the zero-padded length-2D transforms of G = 2^TAILG
// cosets of length D (coset.cuh), half th: stage S0 + u is the transform's stage
// sp = S0 + u - TAILG + 1, whose twiddle index is 2^sp + th 2^(sp - 1) + (the group's
// index within its coset half) instead of the full transform's 2^(S0 + u) + (group index).
template <class S, int S0, int RS, int TAILG = -1>
__device__ __forceinline__ void fwd_pass_regs(u64 (&x)[S::R], const PrimeConsts& P, u32 th = 0) {
  constexpr int G = S::R >> RS;
  constexpr int TLAST_LOG = S::kLogN - S0 - RS;
  const u64 four_q = 2 * P.two_q, q = P.q;
#pragma unroll
  for (int h = 0; h < G; ++h) {
    const u32 g = threadIdx.x + S::T * h;
    const u32 blk = g >> TLAST_LOG;
#pragma unroll
    for (int u = 0; u < RS; ++u) {
      const int span = 1 << (RS - 1 - u);
#pragma unroll
      for (int j = 0; j < (1 << RS); ++j) {
        if (j & span) continue;
        u32 widx = (1u << (S0 + u)) + (blk << u) + (j >> (RS - u));
        if constexpr (TAILG >= 0) {
          const int sp = S0 + u - TAILG + 1;
          widx = (1u << sp) + (th << (sp - 1)) + (widx & ((1u << (sp - 1)) - 1));
        }
        const u64 w = __ldg(P.psi + widx), wsh = __ldg(P.psi_sh + widx);
        u64& A = x[h * (1 << RS) + j];
        u64& Bv = x[h * (1 << RS) + j + span];
        const u64 U = A;
        const u64 V = mul_shoup_lazy(Bv, w, wsh, q);  // [0, 4q)
        A = U + V;
        Bv = U - V + four_q;
      }
    }
  }
}

template <class S, int S0, int RS>
__device__ __forceinline__ u32 fwd_elem(int h, int j) {
  constexpr int TLAST_LOG = S::kLogN - S0 - RS;
  const u32 g = threadIdx.x + S::T * h;
  return ((g >> TLAST_LOG) << (S::kLogN - S0)) + (g & ((1u << TLAST_LOG) - 1)) + ((u32)j << TLAST_LOG);
}

template <class S, int S0, int RS>
__device__ __forceinline__ void fwd_load_smem(u64 (&x)[S::R], const u64* sm) {
#pragma unroll
  for (int h = 0; h < (S::R >> RS); ++h)
#pragma unroll
    for (int j = 0; j < (1 << RS); ++j) x[h * (1 << RS) + j] = sm[S::pad(fwd_elem<S, S0, RS>(h, j))];
}

template <class S, int S0, int RS>
__device__ __forceinline__ void fwd_store_smem(const u64 (&x)[S::R], u64* sm) {
#pragma unroll
  for (int h = 0; h < (S::R >> RS); ++h)
#pragma unroll
    for (int j = 0; j < (1 << RS); ++j) sm[S::pad(fwd_elem<S, S0, RS>(h, j))] = x[h * (1 << RS) + j];
}

// Remaining forward passes, recursively (S0 = first stage of the pass).
// Passes that start below `start` are skipped (their stages already ran, or were copies,
// with the values left in shared memory in natural order); the last pass always leaves
// its values in x.  `start` is the same for every thread of the block.
template <class S, int S0>
__device__ __forceinline__ void fwd_rest(u64 (&x)[S::R], u64* sm, const PrimeConsts& P, u32 start = 0) {
  if constexpr (S0 < S::kLogN) {
    const bool run = (u32)S0 >= start;
    if (run || S0 + S::LOGR == S::kLogN) fwd_load_smem<S, S0, S::LOGR>(x, sm);
    if (run) fwd_pass_regs<S, S0, S::LOGR>(x, P);
    if constexpr (S0 + S::LOGR < S::kLogN) {
      if (run) {
        fwd_store_smem<S, S0, S::LOGR>(x, sm);
        __syncthreads();
      }
      fwd_rest<S, S0 + S::LOGR>(x, sm, P, start);
    }
  }
}

// Forward NTT of one polynomial by the whole block (blockDim.x == S::T).
//   load(e)      -> coefficient e in [0, q) (called for every e, first pass pattern,
//                   coalesced across the warp);
//   store(e, v)  <- slot e, fully reduced (called for every e in increasing-e order per
//                   thread stride, coalesced);
//   prefix       -- the coefficients at and above `prefix` are zero (default: none);
//   sm: S::kSmemWords words of shared memory.  Synchronizes internally.
// Sparse input (a weight block of Algorithm 1's encoding pi_A fills only its lowest
// n_b k_b = N / m_b coefficients).  Stage s pairs e with e + N / 2^(s+1).  With
// prefix <= N / 2^s0 every butterfly of stages 0 .. s0 - 1 has V = 0 and passes U through,
// so after them element e holds coefficient e mod N / 2^s0: those stages are copies (the
// skipped "+ 4q" offsets change nothing mod q, and the final reduction is exact).
//   s0 == RS0: the first pass is replaced by copying each group's one nonzero element in
//              registers;
//   s0 >  RS0: the replicated input is written to shared memory, the stages from s0 up to
//              the next pass boundary run there one by one, and the register passes resume
//              at that boundary (fwd_rest's `start`): log2 N - s0 stages instead of log2 N.
template <class S>
__device__ __forceinline__ void fwd_stage_smem(u64* sm, u32 s, const PrimeConsts& P) {
  const u32 tlog = S::kLogN - 1 - s, span = 1u << tlog;
  const u64 four_q = 2 * P.two_q;
  for (u32 b = threadIdx.x; b < (u32)(S::N / 2); b += S::T) {
    const u32 g = b >> tlog;
    const u32 j = (g << (tlog + 1)) + (b & (span - 1));
    const u32 widx = (1u << s) + g;
    const u64 w = __ldg(P.psi + widx), wsh = __ldg(P.psi_sh + widx);
    const u64 U = sm[S::pad(j)];
    const u64 V = mul_shoup_lazy(sm[S::pad(j + span)], w, wsh, P.q);
    sm[S::pad(j)] = U + V;
    sm[S::pad(j + span)] = U - V + four_q;
  }
}

template <class S, class Load, class Store>
__device__ __forceinline__ void ntt_forward_block(u64* sm, const PrimeConsts& P, Load&& load, Store&& store,
                                                  u32 prefix = S::N) {
  u64 x[S::R];
  const u32 s0 = prefix <= 1 ? (u32)S::kLogN : (u32)S::kLogN - (32 - __clz(prefix - 1));  // prefix <= N >> s0
  u32 start = 0;  // first register pass to run
  if (s0 > (u32)S::RS0) {
    const u32 mask = (S::N >> s0) - 1;
    if ((S::N >> s0) <= S::T) {  // every element of this thread maps to the same coefficient
      const u64 v = load(threadIdx.x & mask);
#pragma unroll
      for (int i = 0; i < S::R; ++i) sm[S::pad(threadIdx.x + S::T * i)] = v;
    } else {
#pragma unroll
      for (int i = 0; i < S::R; ++i) {
        const u32 e = threadIdx.x + S::T * i;
        sm[S::pad(e)] = load(e & mask);
      }
    }
    __syncthreads();
    start = min((u32)S::RS0 + ((s0 - S::RS0 + S::LOGR - 1) / S::LOGR) * S::LOGR, (u32)S::kLogN);
    for (u32 s = s0; s < start; ++s) {
      fwd_stage_smem<S>(sm, s, P);
      __syncthreads();
    }
  } else {
    if (s0 == (u32)S::RS0) {
#pragma unroll
      for (int h = 0; h < (S::R >> S::RS0); ++h) {
        const u64 v = load(fwd_elem<S, 0, S::RS0>(h, 0));
#pragma unroll
        for (int j = 0; j < (1 << S::RS0); ++j) x[h * (1 << S::RS0) + j] = v;
      }
    } else {
#pragma unroll
      for (int h = 0; h < (S::R >> S::RS0); ++h)
#pragma unroll
        for (int j = 0; j < (1 << S::RS0); ++j) x[h * (1 << S::RS0) + j] = load(fwd_elem<S, 0, S::RS0>(h, j));
      fwd_pass_regs<S, 0, S::RS0>(x, P);
    }
    fwd_store_smem<S, 0, S::RS0>(x, sm);
    __syncthreads();
  }
  fwd_rest<S, S::RS0>(x, sm, P, start);
  // last pass ended with contiguous groups in registers: reduce, stage, copy out coalesced
  constexpr int S0L = S::kLogN - S::LOGR;
#pragma unroll
  for (int j = 0; j < S::R; ++j) x[j] = reduce_word(x[j], P);
  __syncthreads();
  fwd_store_smem<S, S0L, S::LOGR>(x, sm);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < S::R; ++i) {
    const u32 e = threadIdx.x + S::T * i;
    store(e, sm[S::pad(e)]);
  }
}

// ---- inverse (Gentleman-Sande).  Pass over stages [S0, S0 + RS): group g has elements
// e = blk * 2^(S0 + RS) + off + j * 2^S0, blk = g >> S0, off = g & (2^S0 - 1).

template <class S, int S0, int RS>
__device__ __forceinline__ u32 inv_elem(int h, int j) {
  const u32 g = threadIdx.x + S::T * h;
  return ((g >> S0) << (S0 + RS)) + (g & ((1u << S0) - 1)) + ((u32)j << S0);
}

// TAILD >= 0: inverse stages (span 2^(S0 + u) < 2^TAILD) of the zero-padded length-2D
// transforms of cosets of length D = 2^TAILD, half th: the transform's stage
// sp = TAILD - (S0 + u), twiddle index 2^sp + th 2^(sp - 1) + (the group's index within its
// coset half) instead of N / 2^(S0 + u + 1) + (group index).
template <class S, int S0, int RS, int TAILD = -1>
__device__ __forceinline__ void inv_pass_regs(u64 (&x)[S::R], const PrimeConsts& P, u32 th = 0) {
  constexpr int G = S::R >> RS;
  const u64 two_q = P.two_q, q = P.q;
#pragma unroll
  for (int h = 0; h < G; ++h) {
    const u32 g = threadIdx.x + S::T * h;
    const u32 blk = g >> S0;
#pragma unroll
    for (int u = 0; u < RS; ++u) {
      const int span = 1 << u;
#pragma unroll
      for (int j = 0; j < (1 << RS); ++j) {
        if (j & span) continue;
        u32 widx = (u32)(S::N >> (S0 + u + 1)) + (blk << (RS - u - 1)) + (j >> (u + 1));
        if constexpr (TAILD >= 0) {
          const int sp = TAILD - (S0 + u);
          const u32 gi = (blk << (RS - u - 1)) + (j >> (u + 1));
          widx = (1u << sp) + (th << (sp - 1)) + (gi & ((1u << (sp - 1)) - 1));
        }
        const u64 w = __ldg(P.ipsi + widx), wsh = __ldg(P.ipsi_sh + widx);
        u64& A = x[h * (1 << RS) + j];
        u64& Bv = x[h * (1 << RS) + j + span];
        const u64 U = A, V = Bv;
        A = csub(U + V, two_q);
        Bv = mul_shoup(U - V + two_q, w, wsh, q);
      }
    }
  }
}

template <class S, int S0, int RS>
__device__ __forceinline__ void inv_load_smem(u64 (&x)[S::R], const u64* sm) {
#pragma unroll
  for (int h = 0; h < (S::R >> RS); ++h)
#pragma unroll
    for (int j = 0; j < (1 << RS); ++j) x[h * (1 << RS) + j] = sm[S::pad(inv_elem<S, S0, RS>(h, j))];
}

template <class S, int S0, int RS>
__device__ __forceinline__ void inv_store_smem(const u64 (&x)[S::R], u64* sm) {
#pragma unroll
  for (int h = 0; h < (S::R >> RS); ++h)
#pragma unroll
    for (int j = 0; j < (1 << RS); ++j) sm[S::pad(inv_elem<S, S0, RS>(h, j))] = x[h * (1 << RS) + j];
}

template <class S, int S0>
__device__ __forceinline__ void inv_middle(u64 (&x)[S::R], u64* sm, const PrimeConsts& P) {
  // passes of LOGR stages starting at S0, up to the last (outermost) pass of RS0 stages
  if constexpr (S0 + S::RS0 < S::kLogN) {
    inv_load_smem<S, S0, S::LOGR>(x, sm);
    inv_pass_regs<S, S0, S::LOGR>(x, P);
    inv_store_smem<S, S0, S::LOGR>(x, sm);
    __syncthreads();
    inv_middle<S, S0 + S::LOGR>(x, sm, P);
  }
}

// Inverse NTT of one polynomial by the whole block (blockDim.x == S::T).
//   load(e)     -> slot e in [0, 2q) (called in coalesced order);
//   store(e, v) <- coefficient e in [0, q) (outermost-pass pattern, coalesced).
template <class S, class Load, class Store>
__device__ __forceinline__ void ntt_inverse_block(u64* sm, const PrimeConsts& P, Load&& load, Store&& store) {
#pragma unroll
  for (int i = 0; i < S::R; ++i) {
    const u32 e = threadIdx.x + S::T * i;
    sm[S::pad(e)] = load(e);
  }
  __syncthreads();
  u64 x[S::R];
  inv_middle<S, 0>(x, sm, P);
  constexpr int S0L = S::kLogN - S::RS0;
  inv_load_smem<S, S0L, S::RS0>(x, sm);
  inv_pass_regs<S, S0L, S::RS0>(x, P);
#pragma unroll
  for (int h = 0; h < (S::R >> S::RS0); ++h)
#pragma unroll
    for (int j = 0; j < (1 << S::RS0); ++j) {
      const u64 v = csub(mul_shoup(x[h * (1 << S::RS0) + j], P.ninv, P.ninv_sh, P.q), P.q);
      store(inv_elem<S, S0L, S::RS0>(h, j), v);
    }
}

// Compact-output mode, one c0 polynomial (prime l) of output ciphertext o: inverse NTT kept
// only at the coefficients e = g k_b + k_b - 1, then c0_e - round(q s_e / t) for the mask
// s of output o under `seed`.  src: N NTT-domain words in [0, q); dst: N / k_b words.
// sm: c0_smem_words(N, log2 k_b) words of shared memory.  All threads of the block call it.
//
// The first log2 k_b Gentleman-Sande stages pair elements inside aligned groups of k_b
// consecutive slots, and the kept position of group g (its last element) depends on that
// group alone: for k_b <= 16 each thread loads whole groups (16-byte loads), runs the
// pruned stages in registers (k_b - 1 Shoup products: stage s keeps the positions whose
// low s + 1 bits are all ones) and writes one value to a compact array.  The remaining
// log2(N / k_b) stages are an inverse transform of length N / k_b on that array: the
// index of stage s's twiddle, N / 2^(s+1) + group, falls below N / k_b, where the table
// entries are exactly the twiddles of that shorter transform (psi^{k_b} as its root).
__host__ __device__ constexpr u32 c0_smem_words(u32 N, u32 logkb) {
  return logkb <= 4 ? (N >> logkb) : N + (N >> logkb);
}

template <int LOGKB>
__device__ __forceinline__ u64 c0_pruned_group(const u64* __restrict__ src, u32 g, u32 N, bool vec,
                                               const PrimeConsts& P) {
  constexpr int KB = 1 << LOGKB;
  u64 v[KB];
  const u64* p = src + (u64)g * KB;
  if (vec) {  // 16-byte aligned group start (KB even, src 16-byte aligned)
#pragma unroll
    for (int i = 0; i < KB; i += 2) {
      const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(p + i);
      v[i] = t.x;
      v[i + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < KB; ++i) v[i] = p[i];
  }
#pragma unroll
  for (int s = 0; s < LOGKB; ++s) {
    const int span = 1 << s;
#pragma unroll
    for (int i = (2 << s) - 1; i < KB; i += (2 << s)) {
      const u32 widx = (N >> (s + 1)) + ((g * KB + i) >> (s + 1));
      v[i] = mul_shoup(v[i - span] - v[i] + P.two_q, __ldg(P.ipsi + widx), __ldg(P.ipsi_sh + widx), P.q);
    }
  }
  return v[KB - 1];
}

__device__ __forceinline__ void ntt_inverse_c0_targets(const u64* src, u64* dst, u32 logkb, u64 seed, u32 o, u32 l,
                                                       const Consts& C, u64* sm) {
  const PrimeConsts P = C.p[l];
  const u32 N = C.N, logN = C.logN, Nc = N >> logkb;
  const u64 q = P.q, two_q = P.two_q;
  u64* z;  // compact values
  if (logkb <= 4) {
    z = sm;
    const bool vec = logkb >= 1 && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
    for (u32 g = threadIdx.x; g < Nc; g += blockDim.x) {
      u64 zv;
      switch (logkb) {
        case 0: zv = src[g]; break;
        case 1: zv = c0_pruned_group<1>(src, g, N, vec, P); break;
        case 2: zv = c0_pruned_group<2>(src, g, N, vec, P); break;
        case 3: zv = c0_pruned_group<3>(src, g, N, vec, P); break;
        default: zv = c0_pruned_group<4>(src, g, N, vec, P); break;
      }
      z[g] = zv;
    }
  } else {  // long groups: stage the whole polynomial in shared memory
    z = sm + N;
    for (u32 i = threadIdx.x; i < N; i += blockDim.x) sm[i] = src[i];
    __syncthreads();
    for (u32 s = 0; s < logkb; ++s) {
      const u32 span = 1u << s, ones = (2u << s) - 1;
      for (u32 t = threadIdx.x; t < (N >> (s + 1)); t += blockDim.x) {
        const u32 p = (t << (s + 1)) | ones;
        const u32 widx = (N >> (s + 1)) + (p >> (s + 1));
        const u64 U = sm[p - span], V = sm[p];
        sm[p] = mul_shoup(U - V + two_q, __ldg(P.ipsi + widx), __ldg(P.ipsi_sh + widx), q);
      }
      __syncthreads();
    }
    const u32 kb = 1u << logkb;
    for (u32 g = threadIdx.x; g < Nc; g += blockDim.x) z[g] = sm[g * kb + kb - 1];
  }
  __syncthreads();
  // remaining stages on the compact array (span 2^(s - log2 k_b) there)
  for (u32 s = logkb; s < logN; ++s) {
    const u32 cs = s - logkb, span = 1u << cs;
    for (u32 b = threadIdx.x; b < (Nc >> 1); b += blockDim.x) {
      const u32 grp = b >> cs;
      const u32 j = (grp << (cs + 1)) + (b & (span - 1));
      const u32 widx = (N >> (s + 1)) + grp;
      const u64 U = z[j], V = z[j + span];
      z[j] = csub(U + V, two_q);
      z[j + span] = mul_shoup(U - V + two_q, __ldg(P.ipsi + widx), __ldg(P.ipsi_sh + widx), q);
    }
    __syncthreads();
  }
  const u32 kb = 1u << logkb;
  for (u32 g = threadIdx.x; g < Nc; g += blockDim.x) {
    u64 v = csub(mul_shoup(z[g], P.ninv, P.ninv_sh, q), q);
    const u32 e = g * kb + kb - 1;
    const u64 sv = lo64(draw(seed, e, o, kDomainMask, 0)) & C.tmask;
    dst[g] = sub_mod(v, delta_residue(sv, C, P), q);
  }
}

}  // namespace he
