/*
 * he_oracle.c -- plain, slow CPU reference ("oracle") for the server-side
 * homomorphic matrix product of Algorithm 1 (Sec. 3.1.1, "Linear Operators")
 * over the RNS variant of BFV described in Sec. 2.2 ("Homomorphic
 * Encryption").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA library.
 *
 * Every modular operation here is the definition written out with 128-bit
 * integers and the `%` operator: no Montgomery/Barrett/Shoup tricks, no lazy
 * reduction, no blocking or fusion.  The NTT is the textbook iterative
 * radix-2 transform of the negacyclic evaluation map; the element-wise
 * product plus inverse transform is the polynomial product of the footnote
 * in Sec. 3.1.3 ("Hardware parallelization of HE operations").
 *
 * Pins (see tests/test_oracle_pins.py): Miller-Rabin vs sympy, the NTT vs
 * its O(N^2) definition and vs schoolbook negacyclic products, Philox
 * known-answer vectors, the Gaussian CDT vs an independent high-precision
 * evaluation, round(q*m/t) residues vs Python big integers, Dec(Enc(m)) = m,
 * and decrypted matrix products vs brute-force integer matrix products.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#include "gauss_cdt.h" /* OR_GAUSS_BOUND, OR_GAUSS_CDT[]: written by gen_gauss_cdt.py */

typedef uint64_t u64;
typedef uint32_t u32;
typedef int64_t i64;
typedef unsigned __int128 u128;

#define OR_MAX_PRIMES 8

/* Philox counter "domain" word (third counter word) for each kind of draw. */
#define OR_DOMAIN_SECRET 1u
#define OR_DOMAIN_UNIFORM 2u
#define OR_DOMAIN_ERROR 3u
#define OR_DOMAIN_MASK 4u

/* ------------------------------------------------------------------ */
/* Modular arithmetic: definitions with 128-bit intermediates.         */
/* ------------------------------------------------------------------ */

static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static u64 submod(u64 a, u64 b, u64 q) { return addmod(a % q, q - (b % q), q); }

static u64 powmod(u64 b, u64 e, u64 q) {
  u64 r = 1 % q;
  b %= q;
  while (e) {
    if (e & 1) r = mulmod(r, b, q);
    b = mulmod(b, b, q);
    e >>= 1;
  }
  return r;
}

/* Inverse modulo a prime by Fermat's little theorem. */
static u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }

/* Signed integer -> residue in [0, q). */
static u64 reduce_signed(i64 v, u64 q) {
  if (v >= 0) return (u64)v % q;
  u64 mag = ((u64)(-(v + 1))) + 1; /* |v| without overflow */
  mag %= q;
  return mag == 0 ? 0 : q - mag;
}

/* Deterministic Miller-Rabin for 64-bit n (the first 12 prime bases suffice). */
int or_is_prime(u64 n) {
  static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return 0;
  for (int i = 0; i < 12; i++) {
    if (n % bases[i] == 0) return n == bases[i];
  }
  u64 d = n - 1;
  int r = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    r++;
  }
  for (int i = 0; i < 12; i++) {
    u64 x = powmod(bases[i], d, n);
    if (x == 1 || x == n - 1) continue;
    int witness = 1;
    for (int j = 1; j < r; j++) {
      x = mulmod(x, x, n);
      if (x == n - 1) {
        witness = 0;
        break;
      }
    }
    if (witness) return 0;
  }
  return 1;
}

/* A primitive 2N-th root of unity mod prime q: psi with psi^N = -1.
 * Returns 0 when 2N does not divide q - 1. */
u64 or_primitive_2n_root(u64 q, u32 N) {
  u64 twoN = 2 * (u64)N;
  if ((q - 1) % twoN != 0) return 0;
  for (u64 g = 2; g < q; g++) {
    u64 c = powmod(g, (q - 1) / twoN, q);
    if (powmod(c, N, q) == q - 1) return c;
  }
  return 0;
}

/* ------------------------------------------------------------------ */
/* Negacyclic NTT (footnote of Sec. 3.1.3): evaluation of a(x) at the    */
/* odd powers of psi,  A_k = sum_i a_i psi^{(2k+1) i}  (k = 0..N-1),      */
/* i.e. a cyclic DFT with omega = psi^2 of (a_i psi^i).                  */
/* ------------------------------------------------------------------ */

static void bit_reverse_permute(u64* a, u32 N) {
  for (u32 i = 1, j = 0; i < N; i++) {
    u32 bit = N >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      u64 tmp = a[i];
      a[i] = a[j];
      a[j] = tmp;
    }
  }
}

/* Textbook iterative radix-2 cyclic DFT over Z_q with root omega (natural order in and out). */
static void cyclic_dft(u64* a, u32 N, u64 q, u64 omega) {
  bit_reverse_permute(a, N);
  for (u32 len = 2; len <= N; len <<= 1) {
    u64 wlen = powmod(omega, N / len, q);
    for (u32 i = 0; i < N; i += len) {
      u64 w = 1;
      for (u32 j = 0; j < len / 2; j++) {
        u64 u = a[i + j];
        u64 v = mulmod(a[i + j + len / 2], w, q);
        a[i + j] = addmod(u, v, q);
        a[i + j + len / 2] = submod(u, v, q);
        w = mulmod(w, wlen, q);
      }
    }
  }
}

static void ntt_forward_one(u64* a, u32 N, u64 q, u64 psi) {
  u64 p = 1;
  for (u32 i = 0; i < N; i++) {
    a[i] = mulmod(a[i], p, q);
    p = mulmod(p, psi, q);
  }
  cyclic_dft(a, N, q, mulmod(psi, psi, q));
}

static void ntt_inverse_one(u64* a, u32 N, u64 q, u64 psi) {
  u64 psi_inv = invmod(psi, q);
  cyclic_dft(a, N, q, mulmod(psi_inv, psi_inv, q));
  u64 n_inv = invmod(N % q, q);
  u64 p = n_inv;
  for (u32 i = 0; i < N; i++) {
    a[i] = mulmod(a[i], p, q);
    p = mulmod(p, psi_inv, q);
  }
}

void or_ntt_forward(u64* a, u32 N, u64 q, u64 psi, size_t count) {
#pragma omp parallel for schedule(dynamic)
  for (long p = 0; p < (long)count; p++) ntt_forward_one(a + (size_t)p * N, N, q, psi);
}

void or_ntt_inverse(u64* a, u32 N, u64 q, u64 psi, size_t count) {
#pragma omp parallel for schedule(dynamic)
  for (long p = 0; p < (long)count; p++) ntt_inverse_one(a + (size_t)p * N, N, q, psi);
}

/* c = a * b in Z_q[x]/(x^N + 1), straight from the definition (x^N = -1). */
void or_negacyclic_mul_schoolbook(const u64* a, const u64* b, u64* c, u32 N, u64 q) {
  for (u32 k = 0; k < N; k++) c[k] = 0;
  for (u32 i = 0; i < N; i++) {
    for (u32 j = 0; j < N; j++) {
      u64 prod = mulmod(a[i] % q, b[j] % q, q);
      u32 k = i + j;
      if (k < N)
        c[k] = addmod(c[k], prod, q);
      else
        c[k - N] = submod(c[k - N], prod, q);
    }
  }
}

/* Negacyclic product through the NTT (used by encryption/decryption). */
static void negacyclic_mul_ntt(const u64* a, const u64* b, u64* c, u32 N, u64 q, u64 psi) {
  u64* fa = (u64*)malloc(sizeof(u64) * N);
  u64* fb = (u64*)malloc(sizeof(u64) * N);
  for (u32 i = 0; i < N; i++) {
    fa[i] = a[i] % q;
    fb[i] = b[i] % q;
  }
  ntt_forward_one(fa, N, q, psi);
  ntt_forward_one(fb, N, q, psi);
  for (u32 i = 0; i < N; i++) c[i] = mulmod(fa[i], fb[i], q);
  ntt_inverse_one(c, N, q, psi);
  free(fa);
  free(fb);
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers:  */
/* as easy as 1, 2, 3", SC'11): 10 rounds of the 4x32 S-P network with    */
/* multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments            */
/* 0x9E3779B9 / 0xBB67AE85.                                              */
/* ------------------------------------------------------------------ */

void or_philox4x32_10(const u32 ctr[4], const u32 key[2], u32 out[4]) {
  u32 x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  u32 k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; round++) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    u64 p0 = (u64)0xD2511F53u * x0;
    u64 p1 = (u64)0xCD9E8D57u * x2;
    u32 y0 = (u32)(p1 >> 32) ^ x1 ^ k0;
    u32 y1 = (u32)p1;
    u32 y2 = (u32)(p0 >> 32) ^ x3 ^ k1;
    u32 y3 = (u32)p0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

/* One Philox block for counter (coef, obj, domain, lane) under key = seed. */
static void draw_block(u64 seed, u32 coef, u32 obj, u32 domain, u32 lane, u32 out[4]) {
  u32 ctr[4] = {coef, obj, domain, lane};
  u32 key[2] = {(u32)seed, (u32)(seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

static u64 draw64(u64 seed, u32 coef, u32 obj, u32 domain, u32 lane) {
  u32 w[4];
  draw_block(seed, coef, obj, domain, lane, w);
  return (u64)w[0] | ((u64)w[1] << 32);
}

/* Secret key: ternary coefficients (draw mod 3) - 1. */
void or_sample_ternary(u64 seed, u32 N, i64* s) {
  for (u32 i = 0; i < N; i++) s[i] = (i64)(draw64(seed, i, 0, OR_DOMAIN_SECRET, 0) % 3) - 1;
}

/* Uniform residue mod q: a 128-bit draw reduced mod q (lane = prime index). */
void or_sample_uniform(u64 seed, u32 obj, u32 prime_index, u64 q, u32 N, u64* a) {
  for (u32 i = 0; i < N; i++) {
    u32 w[4];
    draw_block(seed, i, obj, OR_DOMAIN_UNIFORM, prime_index, w);
    u128 v = (u128)w[0] | ((u128)w[1] << 32) | ((u128)w[2] << 64) | ((u128)w[3] << 96);
    a[i] = (u64)(v % q);
  }
}

/* Discrete Gaussian (sigma = 3.2, |e| <= 19) by inversion of its CDT: the value of
 * one 64-bit draw u is e = -B + #{ j : u >= T_j }. */
i64 or_gauss_from_draw(u64 u) {
  i64 v = -(i64)OR_GAUSS_BOUND;
  for (u32 j = 0; j < 2 * OR_GAUSS_BOUND; j++)
    if (u >= OR_GAUSS_CDT[j]) v++;
  return v;
}

void or_sample_gauss(u64 seed, u32 obj, u32 N, i64* e) {
  for (u32 i = 0; i < N; i++) e[i] = or_gauss_from_draw(draw64(seed, i, obj, OR_DOMAIN_ERROR, 0));
}

/* Server mask coefficients: uniform in Z_t, t = 2^log2t (low bits of a 64-bit draw). */
void or_sample_mask(u64 seed, u32 obj, u32 N, u32 log2t, u64* s) {
  u64 tmask = (log2t >= 64) ? ~(u64)0 : (((u64)1 << log2t) - 1);
  for (u32 i = 0; i < N; i++) s[i] = draw64(seed, i, obj, OR_DOMAIN_MASK, 0) & tmask;
}

void or_gauss_cdt(u64* out) {
  for (u32 j = 0; j < 2 * OR_GAUSS_BOUND; j++) out[j] = OR_GAUSS_CDT[j];
}

u32 or_gauss_bound(void) { return OR_GAUSS_BOUND; }

/* ------------------------------------------------------------------ */
/* BFV scaling: Delta(m) = round(q * m / t), q = prod q_l, t = 2^log2t.  */
/* With R = (q * m) mod t:  round(q m / t) = (q m - R)/t + [2R >= t],    */
/* and (q m - R)/t = -R * t^{-1}  (mod q_l)  because q m = 0 (mod q_l).   */
/* ------------------------------------------------------------------ */

void or_delta_residues(const u64* q, u32 L, u32 log2t, u64 m, u64* out) {
  u64 tmask = ((u64)1 << log2t) - 1;
  u64 q_mod_t = 1;
  for (u32 l = 0; l < L; l++) q_mod_t = (u64)(((u128)q_mod_t * (q[l] & tmask)) & tmask);
  u64 R = (u64)(((u128)q_mod_t * (m & tmask)) & tmask);
  u64 round_up = (2 * (u128)R >= ((u128)1 << log2t)) ? 1 : 0;
  for (u32 l = 0; l < L; l++) {
    u64 tinv = invmod(((u64)1 << log2t) % q[l], q[l]);
    u64 v = submod(0, mulmod(R % q[l], tinv, q[l]), q[l]);
    out[l] = addmod(v, round_up, q[l]);
  }
}

/* ------------------------------------------------------------------ */
/* Symmetric-key BFV (Sec. 2.2): c1 = a, c0 = -a*s + e + Delta(m).        */
/* Ciphertexts are [cnt][2][L][N] u64, coefficient form.                 */
/* ------------------------------------------------------------------ */

void or_encrypt(u32 N, u32 L, const u64* q, const u64* psi, u32 log2t, const i64* s,
                const u64* m, u32 cnt, u32 obj0, u64 seed, u64* ct) {
#pragma omp parallel for schedule(dynamic)
  for (long j = 0; j < (long)cnt; j++) {
    i64* e = (i64*)malloc(sizeof(i64) * N);
    u64* a = (u64*)malloc(sizeof(u64) * N);
    u64* sl = (u64*)malloc(sizeof(u64) * N);
    u64* as = (u64*)malloc(sizeof(u64) * N);
    u64 delta[OR_MAX_PRIMES];
    const u32 obj = obj0 + (u32)j; /* ciphertext index: the object word of every draw */
    or_sample_gauss(seed, obj, N, e);
    for (u32 l = 0; l < L; l++) {
      u64* c0 = ct + (((size_t)j * 2 + 0) * L + l) * N;
      u64* c1 = ct + (((size_t)j * 2 + 1) * L + l) * N;
      or_sample_uniform(seed, obj, l, q[l], N, a);
      for (u32 i = 0; i < N; i++) sl[i] = reduce_signed(s[i], q[l]);
      negacyclic_mul_ntt(a, sl, as, N, q[l], psi[l]);
      for (u32 i = 0; i < N; i++) {
        or_delta_residues(q, L, log2t, m[(size_t)j * N + i], delta);
        u64 v = submod(0, as[i], q[l]);
        v = addmod(v, reduce_signed(e[i], q[l]), q[l]);
        v = addmod(v, delta[l], q[l]);
        c0[i] = v;
        c1[i] = a[i];
      }
    }
    free(e);
    free(a);
    free(sl);
    free(as);
  }
}

/* Decryption core (Sec. 3.1.3, "Reducing the communication cost"):
 * x = c0 + c1 * s  mod each q_l.  The CRT and the rounding by t/q are done
 * with exact big integers by the Python layer. */
void or_decrypt_residues(u32 N, u32 L, const u64* q, const u64* psi, const i64* s, const u64* ct,
                         u32 cnt, u64* x) {
#pragma omp parallel for schedule(dynamic)
  for (long j = 0; j < (long)cnt; j++) {
    u64* sl = (u64*)malloc(sizeof(u64) * N);
    u64* prod = (u64*)malloc(sizeof(u64) * N);
    for (u32 l = 0; l < L; l++) {
      const u64* c0 = ct + (((size_t)j * 2 + 0) * L + l) * N;
      const u64* c1 = ct + (((size_t)j * 2 + 1) * L + l) * N;
      for (u32 i = 0; i < N; i++) sl[i] = reduce_signed(s[i], q[l]);
      negacyclic_mul_ntt(c1, sl, prod, N, q[l], psi[l]);
      for (u32 i = 0; i < N; i++) x[((size_t)j * L + l) * N + i] = addmod(c0[i], prod[i], q[l]);
    }
    free(sl);
    free(prod);
  }
}

/* ------------------------------------------------------------------ */
/* Step 3 of Algorithm 1 with the block split of Sec. 3.1.1:             */
/*   [[c_{Lb,I}]] = sum_J a_{I,J} * [[b_{Lb,J}]],                        */
/* computed slot-wise in the NTT domain (footnote of Sec. 3.1.3).        */
/*   pt_ntt : [nI][nJ][L][N]      (NTT of the centred-lifted a_{I,J})    */
/*   ct_ntt : [nLb][nJ][2][L][N]  (NTT of each input ciphertext poly)    */
/*   out    : [nsel][2][L][N]     (NTT domain), output o = Lb*nI + I     */
/* ------------------------------------------------------------------ */

void or_ctpt_accumulate(u32 N, u32 L, const u64* q, const u64* pt_ntt, const u64* ct_ntt, u32 nI,
                        u32 nJ, u32 nLb, const u32* sel, u32 nsel, u64* out) {
  (void)nLb;
#pragma omp parallel for schedule(dynamic)
  for (long s = 0; s < (long)nsel; s++) {
    u32 o = sel[s];
    u32 Lb = o / nI, I = o % nI;
    for (u32 c = 0; c < 2; c++) {
      for (u32 l = 0; l < L; l++) {
        u64* dst = out + (((size_t)s * 2 + c) * L + l) * N;
        for (u32 i = 0; i < N; i++) {
          u64 acc = 0;
          for (u32 J = 0; J < nJ; J++) {
            u64 a = pt_ntt[(((size_t)I * nJ + J) * L + l) * N + i];
            u64 b = ct_ntt[((((size_t)Lb * nJ + J) * 2 + c) * L + l) * N + i];
            acc = addmod(acc, mulmod(a, b, q[l]), q[l]);
          }
          dst[i] = acc;
        }
      }
    }
  }
}

/* Step 3 of Algorithm 1, the re-mask: c0 <- c0 - Delta(s) for the server's
 * uniform share s of output ciphertext `obj[j]`.  ct: [cnt][2][L][N]. */
void or_apply_mask(u32 N, u32 L, const u64* q, u32 log2t, u64 seed, const u32* obj, u32 cnt,
                   u64* ct) {
#pragma omp parallel for schedule(dynamic)
  for (long j = 0; j < (long)cnt; j++) {
    u64* s = (u64*)malloc(sizeof(u64) * N);
    u64 delta[OR_MAX_PRIMES];
    or_sample_mask(seed, obj[j], N, log2t, s);
    for (u32 i = 0; i < N; i++) {
      or_delta_residues(q, L, log2t, s[i], delta);
      for (u32 l = 0; l < L; l++) {
        u64* c0 = ct + (((size_t)j * 2 + 0) * L + l) * N;
        c0[i] = submod(c0[i], delta[l], q[l]);
      }
    }
    free(s);
  }
}

int or_max_primes(void) { return OR_MAX_PRIMES; }

/* Server-local share product of a linear layer (Sec. 3.1.1, "Fully connected" and
 * "Attention"): out = (acc + X W + bias) mod 2^log2t, row-major, bias [n] and acc [m][n]
 * optional (NULL).  The definition as a triple loop in 64-bit unsigned arithmetic: it
 * wraps mod 2^64, and 2^log2t divides 2^64, so the final mask is the exact residue. */
void or_share_matmul(u32 m, u32 k, u32 n, const u64* X, const u64* W, const u64* bias, const u64* acc,
                     u32 log2t, u64* out) {
  const u64 tmask = (log2t >= 64) ? ~(u64)0 : (((u64)1 << log2t) - 1);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < (long)m; i++) {
    for (u32 j = 0; j < n; j++) {
      u64 s = 0;
      for (u32 l = 0; l < k; l++) s += X[(size_t)i * k + l] * W[(size_t)l * n + j];
      if (bias) s += bias[j];
      if (acc) s += acc[(size_t)i * n + j];
      out[(size_t)i * n + j] = s & tmask;
    }
  }
}
