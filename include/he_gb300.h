/*
 * he_gb300.h -- C ABI of the GB300 library for the server-side homomorphic
 * matrix product of Algorithm 1 (Sec. 3.1.1, "Linear Operators") over RNS
 * BFV (Sec. 2.2, "Homomorphic Encryption").
 *
 * Roles (footnote of Sec. 3.1.1, "Attention"): the client holds X (m x k, an
 * additive share in Z_t) and encrypts it; the server holds W (k x n, weights
 * or its own share).  In Algorithm 1's notation A = W^T and B = X^T, so the
 * protocol produces additive shares of C = (X W)^T; both parties transpose at
 * decode and every share returned here is laid out as X W (m x n).
 *
 * Block split (Sec. 3.1.1: larger matrices "split into smaller blocks"): a
 * blocking {m_b, k_b, n_b} with m_b * k_b * n_b <= N plays the role of
 * Algorithm 1's (n, r, m).  Block counts: nI = ceil(n/n_b), nJ = ceil(k/k_b),
 * nLb = ceil(m/m_b).  The blocking is part of the wire format: the same one
 * must be passed to pack, encode, matmul, unmask and unpack.
 *
 * Memory: every data pointer is caller-owned DEVICE memory (e.g. a torch
 * tensor on the context's device) unless a function says otherwise; the
 * library owns only the context and its tables.  All u64 values are
 * little-endian machine words.  Nothing here throws; every function returns
 * an int status and he_last_error() describes the last failure of the
 * calling thread.  A context may be used by one host thread at a time.
 * `stream` is a cudaStream_t (NULL = legacy default stream); all GPU work is
 * enqueued asynchronously on it unless stated otherwise.
 *
 * Layouts (row-major, u64 words):
 *   plaintext polys  [cnt][N]            coefficients in Z_t
 *   ciphertexts      [cnt][2][L][N]      (c0, c1), residues in [0, q_l), coefficient form
 *   input ciphertext  index Lb * nJ + J   (encrypts pi_B of block (J, Lb) of X^T)
 *   output ciphertext index Lb * nI + I   (share of block (Lb, I) of X W)
 *   encoded weights  opaque, he_sizes().pt_words words (transform form, resident: the
 *                    2D-slot coset transforms of the blocks under the default engine,
 *                    N-slot NTTs under HE_MAC_TENSOR / HE_MAC_INTEGER)
 *   secret key       opaque, L * N words (NTT form)
 *   X, W, shares     [rows][cols] values in Z_t (only the low log2_t bits are read)
 */
#ifndef HE_GB300_H
#define HE_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HE_API __attribute__((visibility("default")))
#else
#define HE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define HE_OK 0       /* success                                              */
#define HE_EINVAL 1   /* bad argument: shape, parameters, blocking, NULL ptr  */
#define HE_ENOMEM 2   /* device allocation failed, or workspace too small     */
#define HE_ECUDA 3    /* a CUDA runtime call or kernel launch failed          */
#define HE_ETIMEOUT 4 /* a bounded device wait expired                         */
#define HE_ENOISE 5   /* decryption found the noise budget exhausted           */

/* ---- flags for he_matmul ------------------------------------------------ */
#define HE_FLAGS_NONE 0u
/* Compact output (Sec. 3.1.3, "Reducing the communication cost"): decrypting
 * coefficient e needs only (c0)_e and all of c1, and pi_C^{-1} reads only the
 * coefficients e = i k_b + k_b - 1.  With this flag each output ciphertext is
 * [c0 at those e: L x (N / k_b)][c1: L x N] (he_sizes().out_words_compact words in
 * all) and c0 is computed only there.  Needs a power-of-two k_b.  The kept words
 * equal the corresponding words of the full output bit for bit. */
#define HE_DROP_C0 1u
/* he_matmul_host only: return once the copies and kernels are enqueued on `stream`
 * instead of waiting for ct_out_host; the caller synchronizes the stream before
 * reading ct_out_host (and must keep both host buffers and the workspace alive until
 * then).  With pinned host buffers this lets calls on different streams overlap their
 * transfers with each other's kernels. */
#define HE_ASYNC 2u

typedef struct he_ctx he_ctx;

typedef struct {
  uint32_t m_b, k_b, n_b;
} he_blocking;

typedef struct {
  uint32_t nI, nJ, nLb;     /* block counts                                  */
  uint64_t in_cts;          /* nLb * nJ input ciphertexts                    */
  uint64_t out_cts;         /* nLb * nI output ciphertexts                   */
  uint64_t pts;             /* nI * nJ encoded weight plaintexts             */
  uint64_t in_words;        /* in_cts * 2 * L * N                            */
  uint64_t out_words;       /* out_cts * 2 * L * N                           */
  uint64_t pt_words;        /* words of the opaque encoded-weight buffer (its layout
                               depends on the engine and, for coset products, on D)   */
  uint64_t packed_words;    /* in_cts * N: he_pack_input output              */
  uint64_t workspace_bytes; /* device workspace he_matmul needs              */
  uint64_t out_words_compact;       /* output words with HE_DROP_C0 (0 if k_b is not a power of two) */
  uint64_t workspace_bytes_compact; /* workspace with HE_DROP_C0                                    */
} he_size_info;

/* Most recent error message of the calling thread ("" if none). */
HE_API const char* he_last_error(void);

/* Parameters {N, t, q} of Sec. 2.2 with q = q_0 ... q_{L-1} (RNS), t = 2^log2_t.
 * N: power of two in [32, 8192].  L in [1, 3] (L * N <= 3 * 8192).
 * q: L distinct primes, each = 1 mod 2N and = 1 mod 2^32 (q_l = c 2^32 + 1, whose products
 *    the kernels reduce with one 32-bit multiply), 2^log2_t < q_l < 2^50 (host array).
 * log2_t in [2, 48].  device: CUDA ordinal the context (and all buffers passed
 * with it) lives on.  Allocates the NTT twiddle tables on that device.
 * Returns HE_EINVAL on any invalid parameter (no GPU call made), HE_ECUDA or
 * HE_ENOMEM on device failures; *ctx is NULL on error. */
HE_API int he_params_init(he_ctx** ctx, uint32_t N, uint32_t L, const uint64_t* q, uint32_t log2_t, int device);

/* Frees the context and its device tables (NULL is a no-op). */
HE_API int he_ctx_free(he_ctx* ctx);

/* Host-side query: N, L, log2_t, the primes and the 2N-th roots psi_l the
 * library chose (psi_l^N = -1 mod q_l).  Arrays hold L entries; any pointer
 * may be NULL. */
HE_API int he_get_params(const he_ctx* ctx, uint32_t* N, uint32_t* L, uint32_t* log2_t, uint64_t* q, uint64_t* psi);

/* Host-side: buffer sizes for an (m x k) . (k x n) product under `blk`.
 * m, k or n == 0 is valid (an empty product: zero-size buffers). */
HE_API int he_sizes(const he_ctx* ctx, uint32_t m, uint32_t k, uint32_t n, const he_blocking* blk, he_size_info* out);

/* Host-side: the blocking this library picks for a shape: powers of two with
 * m_b k_b n_b <= N (at most 4096 k-blocks) minimising a GB300 cost model of he_matmul:
 * transform work (NTT of the input polynomials, inverse NTT of the outputs and, if
 * weights_per_call is non-zero -- weights encoded on every call, e.g. the server's
 * share in an attention product -- the NTT of the weights), multiply-accumulate
 * work divided by its tile fill on the engine the context's setting (he_set_mac_engine)
 * gives a blocking, and algorithmic HBM bytes (the tensor-core engine's weights in their
 * 14-byte digit form).  Ties go to the larger m_b, then k_b. */
HE_API int he_default_blocking(const he_ctx* ctx, uint32_t m, uint32_t k, uint32_t n, uint32_t weights_per_call,
                               he_blocking* out);

/* The same choice without a context (no GPU needed), for the default engine
 * (HE_MAC_AUTO): N a power of two, L >= 1. */
HE_API int he_choose_blocking(uint32_t N, uint32_t L, uint32_t m, uint32_t k, uint32_t n, uint32_t weights_per_call,
                              he_blocking* out);

/* Measured choice of the blocking (an autotuner; the paper has no counterpart).  Takes
 * the `candidates` cheapest blockings under he_choose_blocking's cost model (0 means 6,
 * at most 16; with HE_DROP_C0 only power-of-two k_b), times each on pseudo-random inputs
 * of this shape -- weight encoding (inside the timed region when weights_per_call),
 * then the product of `batch` (0 means 1) same-shape items with `flags` -- and returns
 * the fastest in *out and its time per call (ms, best of three after a warm-up) in
 * *best_ms.  scratch: caller-owned device memory of scratch_bytes; with scratch == NULL
 * nothing runs and *scratch_needed receives the bytes the largest candidate needs
 * (scratch_needed may be NULL otherwise).  Synchronizes `stream`.  m, k or n = 0 returns
 * the model's choice untimed.  The blocking is the wire format: the client must pack
 * with the one returned.  Errors: HE_EINVAL (bad flags, batch * L > 65535), HE_ENOMEM
 * (scratch too small), HE_ECUDA, HE_ETIMEOUT. */
HE_API int he_autotune_blocking(he_ctx* ctx, uint32_t m, uint32_t k, uint32_t n, uint32_t weights_per_call,
                                uint32_t flags, uint32_t batch, uint32_t candidates, void* scratch,
                                size_t scratch_bytes, size_t* scratch_needed, he_blocking* out, float* best_ms,
                                void* stream);

/* Radix of the number-theoretic transforms (the polynomial products of Sec. 3.1.3's
 * footnote, done as NTT, slot-wise product, inverse NTT): each thread of a transform
 * holds 2^log2_values coefficients and runs log2_values butterfly stages in registers
 * per pass.  Built: 4 (16 values, the default) for 512 <= N <= 8192, and 3 and 5 as well
 * for N = 4096 and 8192.  Outputs are bit-identical for every radix (transforms end fully
 * reduced); only speed differs.  The setting applies to launches enqueued afterwards (a
 * CUDA graph keeps the radix it captured) and must not change while another thread
 * uses the context.  N < 512 accepts only 4.  Errors: HE_EINVAL (not built for N). */
HE_API int he_set_ntt_radix(he_ctx* ctx, uint32_t log2_values);
HE_API int he_get_ntt_radix(const he_ctx* ctx, uint32_t* log2_values);

/* Measured choice of that radix (an autotuner; the paper has no counterpart): for every
 * radix built for N, times forward and inverse transforms of cnt ciphertext components
 * (cnt * L polynomials of pseudo-random residues, in place; cnt = 0 means enough for 256
 * MB, larger than L2), one warm-up and three timed round trips, and selects the fastest
 * for the context -- another radix than the default 4 only when it is at least 5% faster
 * (the transforms timed alone are not the layer).  ms (may be NULL): 3 floats, the best round trip in milliseconds for
 * log2_values 3, 4, 5, -1 where not built.  *chosen (may be NULL) receives the selected
 * log2_values.  scratch: caller-owned device memory; with scratch == NULL nothing runs
 * and *scratch_needed (may be NULL) receives cnt * L * N * 8.  Synchronizes `stream`.
 * N < 512: nothing runs, *chosen = 4, *scratch_needed = 0.  Errors: HE_ENOMEM (scratch too small), HE_ECUDA;
 * on an error the radix in force before the call is kept. */
HE_API int he_autotune_ntt_radix(he_ctx* ctx, uint32_t cnt, void* scratch, size_t scratch_bytes,
                                 size_t* scratch_needed, float* ms, uint32_t* chosen, void* stream);

/* Which multiply-accumulate evaluates step 3 of Algorithm 1 in the NTT domain (the
 * slot-wise sum over the k-blocks of ciphertext x plaintext products; footnote of Sec.
 * 3.1.3).  Both are exact and give bit-identical outputs; they differ in speed and in the
 * memory layout of the encoded weights and of the workspace.
 *   HE_MAC_INTEGER: 64-bit residues split into 25-bit halves, three 32 x 32 -> 64-bit
 *     integer multiply-adds per slot product (Karatsuba) on the CUDA cores.
 *   HE_MAC_TENSOR: residues split into seven balanced 8-bit digits, exact in bf16; the
 *     digit products summed on the tcgen05 tensor cores with f32 accumulation (every sum
 *     stays an exact integer below 2^24) and recombined mod q_l.  Needs N >= 512.
 *   HE_MAC_COSET: the tensor-core multiply-accumulate through the ring's cosets where
 *     n_b k_b <= N/2 (else as HE_MAC_TENSOR).  A weight block of pi_A has at most n_b k_b
 *     nonzero coefficients; with D = max(8, n_b k_b rounded up to a power of two) and
 *     G = N / D, x^N + 1 splits into the G factors x^D - zeta_g.  The inputs get the first
 *     log2 G NTT stages (their residues mod each factor) and then a zero-padded length-2D
 *     transform per coset; the weights get only that length-2D transform, which is the
 *     same for every coset.  The weights then cost 2D residues per block instead of N, the
 *     workspace twice the inputs' and outputs' NTT size, and the multiply-accumulate twice
 *     the slot products; an inverse per coset, a fold by zeta_g and the inverse of the first
 *     stages give the same output ciphertexts bit for bit.
 *   HE_MAC_AUTO (the default): the coset form wherever it applies (N >= 512); else the
 *     tensor cores for products of at least 32 k-blocks (k / k_b), the integer path
 *     otherwise.
 * The choice fixes the layout of he_encode_weights' output and of the workspace (he_sizes
 * reports both for the engine in force), so set it before encoding weights and keep it
 * while those weights are in use.  Must not change while another thread uses the
 * context.  Errors: HE_EINVAL (unknown engine). */
#define HE_MAC_AUTO 0u
#define HE_MAC_INTEGER 1u
#define HE_MAC_TENSOR 2u
#define HE_MAC_COSET 3u
HE_API int he_set_mac_engine(he_ctx* ctx, uint32_t engine);
HE_API int he_get_mac_engine(const he_ctx* ctx, uint32_t* engine);
/* Host-side: *yes = 1 if products of inner dimension k under blk use the tensor cores on
 * this context (engine and N as above), else 0. */
HE_API int he_mac_uses_tensor_cores(const he_ctx* ctx, uint32_t k, const he_blocking* blk, uint32_t* yes);
/* Host-side: *yes = 1 if products under blk take the coset form on this context
 * (HE_MAC_COSET above: HE_MAC_AUTO or HE_MAC_COSET, N >= 512, n_b k_b <= N/2), else 0.
 * Errors: HE_EINVAL (NULL argument, invalid blocking). */
HE_API int he_mac_uses_cosets(const he_ctx* ctx, const he_blocking* blk, uint32_t* yes);

/* ---- test client (Sec. 2.2 BFV; encrypt/decrypt are the client's side) -- */

/* Secret key s with ternary coefficients, coefficient i = (u mod 3) - 1 for the
 * 64-bit Philox4x32-10 draw u at counter (i, 0, 1, 0), key = seed.
 * sk: device, L * N words (written in the library's NTT form). */
HE_API int he_keygen(he_ctx* ctx, uint64_t seed, uint64_t* sk, void* stream);

/* Symmetric BFV encryption of cnt plaintext polys: c1 = a, c0 = -a s + e +
 * round(q m / t) mod q_l.  a_l uniform (128-bit Philox draw at counter
 * (i, j, 2, l) reduced mod q_l); e discrete Gaussian sigma 3.2, |e| <= 19
 * (CDT inversion of the 64-bit draw at counter (i, j, 3, 0)); j = index of
 * the plaintext in the batch; key = seed.  Use a fresh seed per batch.
 * plain: device [cnt][N]; ct: device [cnt][2][L][N]. */
HE_API int he_encrypt(he_ctx* ctx, const uint64_t* sk, const uint64_t* plain, uint32_t cnt, uint64_t seed, uint64_t* ct,
               void* stream);

/* Decryption m = round(t [c0 + c1 s]_q / q) mod t (Sec. 3.1.3, "Reducing the
 * communication cost": decryption is c0 + c1 s).  plain: device [cnt][N].
 * noise_budget: optional device int32[cnt], per ciphertext
 * floor(log2(q/2) - log2 max_i |t x_i - q round(t x_i / q)|) (capped at 63).
 * min_budget_host: optional host int32; if given, the call synchronizes the
 * stream, stores the minimum budget there and returns HE_ENOISE if it is <= 0. */
HE_API int he_decrypt(he_ctx* ctx, const uint64_t* sk, const uint64_t* ct, uint32_t cnt, uint64_t* plain,
               int32_t* noise_budget, int32_t* min_budget_host, void* stream);

/* Client packing pi_B of Algorithm 1 on B = X^T, per block (J, Lb):
 * b = sum_{j<k_b, l<m_b} X[Lb m_b + l][J k_b + j] x^{l n_b k_b + j}.
 * X: device [m][k]; polys: device [nLb * nJ][N] (he_sizes().packed_words). */
HE_API int he_pack_input(he_ctx* ctx, const uint64_t* X, uint32_t m, uint32_t k, const he_blocking* blk, uint64_t* polys,
                  void* stream);

/* Client decoding pi_C^{-1} of Algorithm 1 (transposed): its share of X W,
 * share[Lb m_b + l][I n_b + i] = dec[Lb nI + I][l n_b k_b + i k_b + k_b - 1].
 * dec: device [nLb * nI][N] decrypted outputs; client_share: device [m][n]. */
HE_API int he_unpack_output(he_ctx* ctx, const uint64_t* dec, uint32_t m, uint32_t n, const he_blocking* blk,
                     uint64_t* client_share, void* stream);

/* ---- server (the hot path) ---------------------------------------------- */

/* Server encoding pi_A of Algorithm 1 on A = W^T, per block (I, J):
 * a = sum_{i<n_b, j<k_b} W[J k_b + j][I n_b + i] x^{i k_b + k_b - 1 - j},
 * coefficients lifted to the centred range [-t/2, t/2), reduced mod each q_l
 * and transformed to the NTT domain (footnote of Sec. 3.1.3).
 * W: device [k][n]; pt: device, he_sizes().pt_words words (opaque). */
HE_API int he_encode_weights(he_ctx* ctx, const uint64_t* W, uint32_t k, uint32_t n, const he_blocking* blk, uint64_t* pt,
                      void* stream);

/* he_encode_weights for `batch` matrices W + b * k * n into pt + b * pt_words. */
HE_API int he_encode_weights_batch(he_ctx* ctx, const uint64_t* W, uint32_t k, uint32_t n, const he_blocking* blk,
                                   uint32_t batch, uint64_t* pt, void* stream);

/* Step 3 of Algorithm 1 for every output block: [[c_{Lb,I}]] = sum_J
 * a_{I,J} * [[b_{Lb,J}]] (NTT, slot-wise multiply-accumulate, inverse NTT),
 * then the re-mask c0 <- c0 - round(q s / t) with the server's share s of
 * output o = Lb nI + I: s_i = low log2_t bits of the 64-bit Philox draw at
 * counter (i, o, 4, 0), key = mask_seed.  Use a fresh mask_seed per call.
 * ct_in: device [in_cts][2][L][N]; pt: from he_encode_weights with the same
 * k, n and blk; ct_out: device [out_cts][2][L][N]; workspace: device,
 * >= he_sizes().workspace_bytes (HE_ENOMEM if smaller).
 * ct_out must not overlap ct_in, pt or workspace.  flags: HE_FLAGS_NONE or HE_DROP_C0
 * (then ct_out holds he_sizes().out_words_compact words and the workspace must be
 * >= he_sizes().workspace_bytes_compact). */
HE_API int he_matmul(he_ctx* ctx, const uint64_t* ct_in, const uint64_t* pt, uint32_t m, uint32_t k, uint32_t n,
              const he_blocking* blk, uint64_t mask_seed, uint32_t flags, uint64_t* ct_out, void* workspace,
              size_t workspace_bytes, void* stream);

/* The same product with the ciphertexts in HOST memory (pinned memory gives
 * asynchronous copies): ct_in_host is copied to the device workspace, the
 * product is computed as by he_matmul, and the output is copied back to
 * ct_out_host; the call returns once ct_out_host holds the result (or, with HE_ASYNC,
 * once everything is enqueued on `stream`).
 * workspace: device, >= he_sizes().workspace_bytes + 8 * (in_words + out_words). */
HE_API int he_matmul_host(he_ctx* ctx, const uint64_t* ct_in_host, const uint64_t* pt, uint32_t m, uint32_t k, uint32_t n,
                   const he_blocking* blk, uint64_t mask_seed, uint32_t flags, uint64_t* ct_out_host, void* workspace,
                   size_t workspace_bytes, void* stream);

/* he_matmul_batch with the ciphertexts in HOST memory (layouts as he_matmul_batch):
 * copies in, computes, copies out, as he_matmul_host does for one product.
 * workspace: device, >= batch times what he_matmul_host needs for one product. */
HE_API int he_matmul_batch_host(he_ctx* ctx, const uint64_t* ct_in_host, const uint64_t* pt, uint32_t m, uint32_t k,
                                uint32_t n, const he_blocking* blk, uint32_t batch, uint64_t mask_seed,
                                uint32_t flags, uint64_t* ct_out_host, void* workspace, size_t workspace_bytes,
                                void* stream);

/* `batch` independent products of one shape and blocking in one set of launches (e.g.
 * the per-head attention cross terms of a layer).  Item b reads ct_in + b * in_words and
 * pt + b * pt_words, writes ct_out + b * out_words, and is re-masked with seed
 * mask_seed + b: the result is bit-identical to `batch` he_matmul calls with those
 * seeds.  workspace >= batch * he_sizes().workspace_bytes.  batch * L <= 65535. */
HE_API int he_matmul_batch(he_ctx* ctx, const uint64_t* ct_in, const uint64_t* pt, uint32_t m, uint32_t k, uint32_t n,
                           const he_blocking* blk, uint32_t batch, uint64_t mask_seed, uint32_t flags,
                           uint64_t* ct_out, void* workspace, size_t workspace_bytes, void* stream);

/* he_matmul_multi only (a product's flags): the product's mask_seed field holds the
 * address of a device uint64_t, and the kernels read the seed from there when they run.
 * A CUDA graph that captured the launch then re-masks with whatever seed the word holds
 * at each replay (write it on the replay's stream before the replay).  The word must
 * stay valid until the launch completes. */
#define HE_SEED_DEVICE 16u

/* One product of a multi-product launch. */
typedef struct {
  const uint64_t* ct_in; /* device, in_words                                   */
  const uint64_t* pt;    /* device, from he_encode_weights with this k, n, blk  */
  uint64_t* ct_out;      /* device, out_words (out_words_compact with DROP_C0)  */
  uint32_t m, k, n;
  he_blocking blk;
  uint32_t flags;        /* HE_FLAGS_NONE, HE_DROP_C0, HE_SEED_DEVICE (or'ed)   */
  uint64_t mask_seed;    /* the seed, or with HE_SEED_DEVICE its device address */
} he_product;

/* Up to 64 products of any shapes, blockings and output modes (e.g. the requests a
 * serving loop has admitted) in one set of launches: one forward-NTT grid, one
 * multiply-accumulate grid and one or two inverse-NTT grids over the union of the
 * products' work.  Each product's output is bit-identical to its own he_matmul call.
 * workspace: device, >= he_multi_workspace_bytes(ctx, count, items).  The call only
 * enqueues kernels (no allocation, copy or synchronization), so it can be captured in
 * a CUDA graph; with HE_SEED_DEVICE products the graph takes fresh seeds per replay. */
HE_API int he_matmul_multi(he_ctx* ctx, uint32_t count, const he_product* items, void* workspace,
                           size_t workspace_bytes, void* stream);
HE_API int he_multi_workspace_bytes(const he_ctx* ctx, uint32_t count, const he_product* items, size_t* bytes);

/* he_matmul_multi from HOST buffers: each product's ct_in and ct_out are host pointers
 * (pinned memory lets the copies overlap other streams' work).  Enqueues on `stream` one
 * host-to-device copy per input, the multi-product launch and one device-to-host copy
 * per output, staging them in the workspace, then waits for the stream unless flags has
 * HE_ASYNC (the caller then synchronizes before reading ct_out and keeps the host
 * buffers and the workspace alive until then).  Calls on two streams with their own
 * workspaces overlap one call's transfers with the other's kernels.
 * workspace: device, >= he_multi_host_workspace_bytes(ctx, count, items). */
HE_API int he_matmul_multi_host(he_ctx* ctx, uint32_t count, const he_product* items, uint32_t flags, void* workspace,
                                size_t workspace_bytes, void* stream);
HE_API int he_multi_host_workspace_bytes(const he_ctx* ctx, uint32_t count, const he_product* items, size_t* bytes);

/* Overlapped host-buffer execution of multi-product launches: a server's transfer
 * pipeline (the paper has no counterpart; it moves the ciphertexts of Algorithm 1 steps 2
 * and 4 between host and device).  A pipe owns three CUDA streams -- uploads, compute,
 * downloads -- and cycles through `depth` staging slots of the caller's workspace.  Each
 * he_pipe_submit enqueues
 *   - on the upload stream, one host-to-device copy per product input into the next slot,
 *     after the launch that last used that slot has finished reading it;
 *   - on the compute stream, the multi-product launch (as he_matmul_multi), after those
 *     copies and after the downloads that last read the slot's outputs;
 *   - on the download stream, one device-to-host copy per product output, after the launch.
 * Each queue runs in submission order, so consecutive submits overlap one's uploads with
 * another's kernels and a third's downloads (an upload of a later submit never competes
 * with the one the next launch waits for).  Nothing blocks but he_pipe_wait.
 * The pipe's streams do not wait for other streams: what the launches read (encoded
 * weights, seeds in device memory) must be complete, or enqueued on the compute stream,
 * before the submit.
 * Ownership: the pipe owns its streams and events (he_pipe_free); the caller owns the
 * workspace and the host buffers and keeps them alive and unchanged (inputs) or unread
 * (outputs) until he_pipe_wait returns.  Host buffers should be pinned (pageable copies
 * are synchronous and serialize the pipeline).  Errors: HE_EINVAL for a NULL argument,
 * depth 0 or > 16; HE_ENOMEM for a workspace below he_pipe_workspace_bytes(); HE_ECUDA for a
 * failed enqueue; kernels' expired waits are reported by he_device_status. */
typedef struct he_pipe he_pipe;
HE_API int he_pipe_create(he_ctx* ctx, uint32_t depth, he_pipe** pipe);
HE_API int he_pipe_free(he_pipe* pipe);
/* The pipe's compute stream: work the caller enqueues there (e.g. encoding the server's
 * per-request shares for the next submit) is ordered with the pipe's launches. */
HE_API int he_pipe_compute_stream(he_pipe* pipe, void** stream);
/* Device workspace for submits of these products: depth slots, each the largest
 * multi-product workspace of the launches (64 products each) plus every staged input and
 * output. */
HE_API int he_pipe_workspace_bytes(const he_pipe* pipe, uint32_t count, const he_product* items, size_t* bytes);
/* items: any number of products with HOST ct_in / ct_out (device pt; flags and mask seeds
 * as in he_matmul_multi), run as consecutive multi-product launches of up to 64 products.
 * workspace: device, the same on every submit of this pipe; slot i is
 * [i * slot, (i + 1) * slot) with slot = workspace_bytes / depth rounded down to 256 bytes,
 * and depth * slot must be >= he_pipe_workspace_bytes(pipe, count, items). */
HE_API int he_pipe_submit(he_pipe* pipe, uint32_t count, const he_product* items, void* workspace,
                          size_t workspace_bytes);
/* Blocks until every submitted product's outputs are in host memory. */
HE_API int he_pipe_wait(he_pipe* pipe);

/* he_matmul for callers that cannot allocate device memory.  Some callers have no
 * way to obtain a workspace: a serving process whose device memory is already
 * reserved by another allocator (where cudaMalloc would fail, or would stall the
 * device while requests are in flight), or a host program that is not permitted to
 * manage device memory.  This entry point computes exactly what he_matmul computes
 * with the same flags (HE_FLAGS_NONE or HE_DROP_C0; ct_out then holds out_words or
 * out_words_compact words) and allocates nothing: its scratch (the NTT of the input
 * ciphertexts, and with HE_DROP_C0 the NTT-domain c0 of the outputs) is a fixed
 * device array of HE_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that
 * loads the library keeps until the process exits.
 * - Products whose he_sizes().workspace_bytes (workspace_bytes_compact with
 *   HE_DROP_C0) exceeds HE_NOALLOC_SCRATCH_BYTES are rejected with HE_EINVAL before
 *   any GPU work; so is HE_ASYNC or any other flag.
 * - The first call on a device looks up the array's device address (with that
 *   device current); make that first call before any stream capture.
 * - All calls share the one array and it keeps the last call's contents (every word
 *   a call reads is first written by the same call, so nothing is cleared).  Calls
 *   that overlap on the GPU -- on different streams or host threads -- race on it:
 *   serialize them, e.g. on one stream.
 * The paper has no counterpart to this entry point; it exists for deployment. */
#define HE_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
HE_API int he_matmul_noalloc(he_ctx* ctx, const uint64_t* ct_in, const uint64_t* pt, uint32_t m, uint32_t k,
                             uint32_t n, const he_blocking* blk, uint64_t mask_seed, uint32_t flags, uint64_t* ct_out,
                             void* stream);

/* Client side of HE_DROP_C0: expand cnt compact ciphertexts (k_b of the product's
 * blocking) to full [cnt][2][L][N] ciphertexts, c0 zero outside the kept
 * coefficients, for he_decrypt (whose other coefficients are then meaningless). */
HE_API int he_expand_compact(he_ctx* ctx, const uint64_t* ct_compact, uint32_t cnt, uint32_t k_b, uint64_t* ct_full,
                             void* stream);

/* Ciphertexts on the wire between client and server (Algorithm 1: the client sends its
 * encrypted share, the server returns the re-masked product; Sec. 3.1.3, "Reducing the
 * communication cost": only c1 and the decoded c0 coefficients need to travel).  The
 * wire format is the library's ciphertext layout in coefficient form, little-endian u64
 * words: with k_b = 0, full ciphertexts [cnt][2][L][N]; with a power-of-two k_b (at most
 * N), compact ciphertexts as written by HE_DROP_C0 for a product of that k_b, each
 * [c0 at the decoded coefficients: L x N / k_b][c1: L x N].
 *
 * he_ct_export copies cnt ciphertexts from device memory `ct` (caller-owned) to
 * host_buf (caller-owned, cnt x words per ciphertext) and returns once host_buf holds
 * them (synchronizes `stream`).
 *
 * he_ct_import copies host_buf to device memory `ct` (caller-owned) and checks on the
 * GPU that every word is a residue of its prime (below q_l); it synchronizes `stream`
 * and returns HE_EINVAL naming the count and the first offending word (ciphertext,
 * component, prime) if not -- `ct` then holds the rejected words and must not be used.
 *
 * Errors: HE_EINVAL (NULL ctx or buffer with cnt > 0, k_b neither 0 nor a power of two
 * <= N, residue out of range), HE_ECUDA.  cnt = 0 does nothing. */
HE_API int he_ct_export(he_ctx* ctx, const uint64_t* ct, uint32_t cnt, uint32_t k_b, uint64_t* host_buf,
                        void* stream);
HE_API int he_ct_import(he_ctx* ctx, const uint64_t* host_buf, uint32_t cnt, uint32_t k_b, uint64_t* ct,
                        void* stream);

/* Server's share pi_C^{-1}(s) of X W for the masks of he_matmul(mask_seed):
 * share[Lb m_b + l][I n_b + i] = s_{Lb nI + I}[l n_b k_b + i k_b + k_b - 1].
 * server_share: device [m][n] (requires k only through blk->k_b). */
HE_API int he_unmask(he_ctx* ctx, uint64_t mask_seed, uint32_t m, uint32_t n, const he_blocking* blk, uint64_t* server_share,
              void* stream);

/* ---- server-local share products (Sec. 3.1.1) -------------------------- */

/* The server's own plaintext side of a linear layer.  A fully connected layer gives the
 * server the share W<x>_0's mask share plus W<x>_1 + b; an attention product gives it
 * its cross-term mask shares plus <X>_1 <Y>_1 (Sec. 3.1.1, "Fully connected" and
 * "Attention").  This computes
 *     out = (acc + X W + bias) mod t
 * X: device [m][k], W: device [k][n], bias: device [n] or NULL, acc: device [m][n] or
 * NULL (may be the same buffer as out), out: device [m][n]; every value in Z_t (only
 * the low log2_t bits of X, W, bias and acc matter: t divides 2^64 and the arithmetic
 * wraps mod 2^64 before the final reduction).  k = 0 gives acc + bias.  Errors:
 * HE_EINVAL for a NULL ctx, X (k > 0), W (k > 0) or out; HE_ECUDA on a launch failure. */
HE_API int he_share_matmul(he_ctx* ctx, const uint64_t* X, const uint64_t* W, const uint64_t* bias,
                           const uint64_t* acc, uint32_t m, uint32_t k, uint32_t n, uint64_t* out, void* stream);

/* he_share_matmul over `batch` same-shape items in one launch (e.g. the per-head
 * <X>_1 <Y>_1 products of an attention layer): item b reads X + b m k, W + b k n,
 * bias + b n, acc + b m n and writes out + b m n.  batch <= 65535; batch = 0 does
 * nothing.  Errors as for he_share_matmul. */
HE_API int he_share_matmul_batch(he_ctx* ctx, const uint64_t* X, const uint64_t* W, const uint64_t* bias,
                                 const uint64_t* acc, uint32_t m, uint32_t k, uint32_t n, uint32_t batch,
                                 uint64_t* out, void* stream);

/* he_unmask into an existing share: with HE_UNMASK_ACCUMULATE the mask share of the
 * Pi_MatMul of an (m x k) . (k x n) product (blocking blk, mask_seed) is added mod t to
 * out instead of overwriting it; with HE_UNMASK_TRANSPOSE it goes to out as its
 * transpose, out being [n][m] (the cross term of an attention product that runs in the
 * transposed form of the Sec. 3.1.1 footnote).  out: device memory, caller-owned. */
#define HE_UNMASK_ACCUMULATE 4u
#define HE_UNMASK_TRANSPOSE 8u
HE_API int he_unmask_acc(he_ctx* ctx, uint64_t mask_seed, uint32_t m, uint32_t n, const he_blocking* blk,
                         uint32_t flags, uint64_t* out, void* stream);

/* ---- test hooks --------------------------------------------------------- */

/* In-place negacyclic NTT of cnt polys laid out [cnt][L][N] (prime l for row l),
 * residues in [0, q_l).  Forward output is in the library's slot order:
 * slot j holds a(psi_l^{2 brev(j) + 1}) (brev = log2(N)-bit reversal). */
HE_API int he_ntt_forward(he_ctx* ctx, uint64_t* polys, uint32_t cnt, void* stream);
HE_API int he_ntt_inverse(he_ctx* ctx, uint64_t* polys, uint32_t cnt, void* stream);

/* c = a * b in Z_{q_l}[x]/(x^N + 1) for cnt polys laid out [cnt][L][N]
 * (NTT, slot-wise product, inverse NTT; footnote of Sec. 3.1.3).  c may alias a. */
HE_API int he_poly_mul(he_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t* c, uint32_t cnt, void* stream);

/* Failure-detection check: launches one kernel whose bounded wait (the same one the
 * multiply-accumulate uses for its data copies) waits on a barrier nothing completes,
 * gives up after limit_ms (1..2000) and records the error; he_device_status then
 * returns HE_ETIMEOUT.  The context stays usable. */
HE_API int he_test_wait_timeout(he_ctx* ctx, uint32_t limit_ms, void* stream);

/* Host-side copy of the library's Gaussian inversion table (2 * 19 words). */
HE_API int he_gauss_cdt(uint64_t* out, uint32_t cap);

/* ---- profiling (CUDA events recorded on the launching stream) ----------- */

typedef struct {
  char name[32];     /* kernel family                          */
  uint64_t launches; /* launches timed since the last reset    */
  double total_ms;   /* sum of event-measured durations        */
} he_kernel_stat;

/* Enable (1) / disable (0) per-launch event timing; enabling resets stats. */
HE_API int he_profile_enable(he_ctx* ctx, int on);
/* Synchronizes the recorded events and returns up to cap stats in *n. */
HE_API int he_profile_read(he_ctx* ctx, he_kernel_stat* out, uint32_t cap, uint32_t* n);
/* Synchronizes `stream` and reports whether any kernel of this context gave up a
 * bounded wait (a data copy that never completed) since the last call:
 * HE_ETIMEOUT if so (the flag is then cleared; the affected outputs are invalid),
 * HE_OK otherwise. */
HE_API int he_device_status(he_ctx* ctx, void* stream);

/* Integer roofline probe: times dependency-free chains of mad.wide.u32 (the
 * instruction the multiply-accumulate kernel is built on) over every SM and returns
 * the achieved rate (operations/s) and, optionally, per SM per (maximum) clock.
 * scratch: device, >= (number of SMs) x 2048 words.  Synchronizes the stream.  Not
 * part of the protocol: it supplies the peak for roofline reporting. */
HE_API int he_probe_mad_wide(he_ctx* ctx, uint64_t* scratch, size_t scratch_words, double* ops_per_s,
                             double* per_sm_per_clock, void* stream);

/* Tensor-core rate probe for roofline reporting (the paper has no counterpart).  kind 0:
 * dense tcgen05 MMAs with bf16 operands and f32 accumulation (kind::f16; M = 128, N = 256,
 * K = 16, operands in shared memory, one issuing thread per block, two blocks per SM on
 * every SM).  kind 1: warp-level mma.sync m16n8k32 with signed 8-bit operands and s32
 * accumulation -- the only 8-bit integer tensor instruction sm_103a offers (tcgen05.mma
 * kind::i8 is not supported for this target).  These are the two exact routes for
 * splitting the slot-wise multiply-accumulate (Algorithm 1 step 3) into small integer
 * limbs.  Returns the achieved rate in operations (2 per multiply-add) per second.
 * scratch: device, >= 4 x (number of SMs) words.  Synchronizes the stream.  A bounded wait
 * that expires is reported by he_device_status. */
HE_API int he_probe_tensor(he_ctx* ctx, uint32_t kind, double* ops_per_s, uint32_t* scratch, size_t scratch_words,
                           void* stream);

/* Test hook: D = A B^T on the tcgen05 tensor cores through the library's shared-memory and
 * instruction descriptor encodings.  A: device, 128 x k bf16; B: device, n x k bf16
 * (row-major); D: device, 128 x n f32.  n a multiple of 16 in [16, 256]; k a positive
 * multiple of 16 with (128 + n) x k x 2 <= 200 KB.  Errors: HE_EINVAL, HE_ECUDA. */
HE_API int he_test_tc_gemm(he_ctx* ctx, uint32_t n, uint32_t k, const void* A, const void* B, void* D, void* stream);

/* Number of kernels this context has launched since creation. */
HE_API int he_launch_count(const he_ctx* ctx, uint64_t* out);

#ifdef __cplusplus
}
#endif

#endif /* HE_GB300_H */
