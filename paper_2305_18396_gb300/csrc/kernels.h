// kernels.h -- host-side launchers of the library's CUDA kernels (internal).
#pragma once

#include "he_common.cuh"

namespace he {

struct Blk {
  u32 m_b, k_b, n_b;
};

// Each launcher enqueues one kernel on `st` and returns cudaGetLastError().
// Shared-memory attributes are set once per device by configure_kernels().
cudaError_t configure_kernels(const Consts& C);

cudaError_t launch_ntt_forward(const Consts& C, const u64* src, u64* dst, u64 npolys, cudaStream_t st);
cudaError_t launch_ntt_inverse(const Consts& C, const u64* src, u64* dst, u64 npolys, cudaStream_t st);
cudaError_t launch_poly_mul(const Consts& C, const u64* a, const u64* b, u64* c, u64 npolys, cudaStream_t st);

cudaError_t launch_keygen(const Consts& C, u64 seed, u64* sk, cudaStream_t st);
cudaError_t launch_encrypt(const Consts& C, const u64* sk, const u64* plain, u32 cnt, u64 seed, u64* ct,
                           cudaStream_t st);
cudaError_t launch_decrypt(const Consts& C, const u64* sk, const u64* ct, u32 cnt, u64* plain, int* budget,
                           cudaStream_t st);
cudaError_t launch_pack(const Consts& C, const u64* X, u32 m, u32 k, Blk b, u32 nJ, u32 nLb, u64* polys,
                        cudaStream_t st);
cudaError_t launch_unpack(const Consts& C, const u64* dec, u32 m, u32 n, Blk b, u32 nI, u64* share,
                          cudaStream_t st);
cudaError_t launch_unmask(const Consts& C, u64 seed, u32 m, u32 n, Blk b, u32 nI, u64* share, cudaStream_t st);
cudaError_t launch_fill_random(const Consts& C, u64* dst, u64 words, u64 seed, int mode, cudaStream_t st);
// share.cu: server-local share products and mask-share accumulation
u32 share_matmul_splits(u32 m, u32 k, u32 n, u32 batch, int sms);
cudaError_t launch_share_matmul(const Consts& C, const u64* X, const u64* W, const u64* bias, const u64* acc, u32 m,
                                u32 k, u32 n, u32 batch, u32 splits, u64* out, cudaStream_t st);
cudaError_t launch_unmask_acc(const Consts& C, u64 seed, u32 m, u32 n, Blk b, u32 nI, int accumulate, int transpose,
                              u64* out, cudaStream_t st);

// Products come in batches of identical shape laid out back to back (batch = 1 for one).
// tc: write the digit tiles of the tensor-core multiply-accumulate (mac_tc.cuh) instead of the
// slot-chunked layout (per product tc_weight_words(nI, nJ, L, N) words instead of nI nJ L N;
// the buffer is cleared first).
cudaError_t launch_encode_weights(const Consts& C, const u64* W, u32 k, u32 n, Blk b, u32 nI, u32 nJ, u32 batch,
                                  u32 tc, u64* pt, cudaStream_t st);
// Slot-wise sum_J pt[I][J] * ctN[Lb][J] for every output (Lb, I), both components, all primes.
// Forward NTT of a product's input ciphertexts (wire format) into the slot-chunked
// operand layout the multiply-accumulate kernel streams.
cudaError_t launch_ntt_forward_mm(const Consts& C, const u64* ct_in, u64* ctN, u32 nJ, u32 nLb, u32 batch, u32 tc,
                                  cudaStream_t st);
// err: device int set to 1 if a bounded wait inside the kernel expired.  Component c of
// global output ciphertext g (item * out_cts + Lb * nI + I), prime l, is written at
// out_c + g * stride_c + l * N (NTT domain).
cudaError_t launch_mac(const Consts& C, const u64* ctN, const u64* pt, u64* out0, u64 stride0, u64* out1, u64 stride1,
                       u32 nI, u32 nJ, u32 nLb, u32 batch, int* err, cudaStream_t st);
// The same on the tensor cores, operands in the stage-tiled layout (mac_tc.cuh); N >= 512.
cudaError_t launch_mac_tc(const Consts& C, const u64* ctN, const u64* pt, u64* out0, u64 stride0, u64* out1,
                          u64 stride1, u32 nI, u32 nJ, u32 nLb, u32 batch, int* err, cudaStream_t st);
// Compact-output mode: in-place inverse NTT of the c1 polynomials (c1 of ciphertext g at
// base + g * ct_stride), and the pruned inverse NTT + mask of c0 at the coefficients
// e = i k_b + k_b - 1 only (NTT-domain c0 of ciphertext g at src + g L N).
cudaError_t launch_intt_c1(const Consts& C, u64* base, u64 ct_stride, u64 cts, cudaStream_t st);
// Counts the words of cnt wire-format ciphertexts (c0 with N >> logkb words per prime, then
// c1) not below their prime into bad[0] and the first such index into bad[1] (the caller
// sets bad[0] = 0 and bad[1] = ~0 first).
cudaError_t launch_check_residues(const Consts& C, const u64* ct, u64 cnt, u32 logkb, u64* bad, cudaStream_t st);
// Compact ciphertexts -> full ciphertexts with zero c0 outside the kept coefficients.
cudaError_t launch_expand_compact(const Consts& C, const u64* src, u64 cnt, u32 logkb, u64* dst, cudaStream_t st);
cudaError_t launch_intt_c0_targets(const Consts& C, const u64* src, u64* dst, u64 ct_stride, u64 out_cts, u32 batch,
                                   u32 logkb, u64 seed, cudaStream_t st);
// Inverse NTT of every output polynomial, then c0 -= round(q s / t) for the mask of output o
// (batch item b uses seed + b).
cudaError_t launch_intt_mask(const Consts& C, u64* out, u64 out_cts, u32 batch, u64 seed, cudaStream_t st);

// Integer roofline probe: times sms * 8 blocks of 256 threads, each 2048 x 64 mad.wide.u32
// (`out`: sms * 8 * 256 words of scratch).
cudaError_t probe_mad_wide(int sms, u64* out, float* ms, cudaStream_t st);

// Tensor-core rate probes (tc_probe.cu), timed with events (*ms): kind 0, 2 x sms blocks each
// issuing *iters_used tcgen05 MMAs of M = 128, N = 256, K = 16 (bf16 -> f32); kind 1,
// 4 x sms blocks of 256 threads issuing 8 x *iters_used warp-level mma.sync m16n8k32
// (s8 -> s32) per warp.  *err set if a bounded wait expired; sink: 4 x sms words.
cudaError_t probe_tensor(int kind, int sms, int* err, uint32_t* sink, float* ms, int* iters_used, cudaStream_t st);
// D (128 x n f32 words) = A (128 x k bf16) . B (n x k bf16)^T through tcgen05; A, B
// row-major; n in [16, 256] a multiple of 16; k a multiple of 16 with (128 + n) k 2 <= 200 KB.
cudaError_t launch_tc_check(const void* A, const void* B, void* D, uint32_t n, uint32_t k, int* err, cudaStream_t st);

// Runs one bounded wait on an mbarrier nothing completes (limit_ns), setting *err on expiry.
cudaError_t launch_wait_timeout_check(uint64_t limit_ns, int* err, cudaStream_t st);

// Streaming multiprocessors of the current device (cached per device).
int device_sms();

// Fixed device scratch of he_matmul_noalloc (no allocation at call time).
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
constexpr int kMaxDevices = 64;
// Device address of that scratch on `device`, which must be the current device.  The first
// call per device looks the address up with cudaGetSymbolAddress; later calls reuse it.
cudaError_t noalloc_scratch_address(int device, void** ptr);

}  // namespace he
