// tcgen05.cuh -- the sm_100-family tensor-core primitives the library uses, as inline PTX:
// tensor-memory (TMEM) allocation, the shared-memory matrix descriptor and the instruction
// descriptor of tcgen05.mma, the MMA itself (one thread issues it), its completion on an
// mbarrier (tcgen05.commit) and the warp-wide TMEM -> register load of the epilogue.
//
// Operand layout used throughout: K-major, no swizzle ("interleaved" canonical layout).  A
// tile of R rows x K elements of 16 bytes per row-chunk is stored as core matrices of 8 rows
// x 16 bytes (128 contiguous bytes, row i at +16 i); the core matrix of row group g and K
// chunk c sits at g * SBO + c * LBO.  With LBO = 128 and SBO = 128 * (K bytes / 16) the tile
// is [g][c][row in group][16 bytes], and the MMA of K step k (32 bytes of K per row) starts
// at the tile base + k * 256 bytes.
#pragma once

#include <cstdint>

#include "async.cuh"

namespace he {
namespace tc {

// Shared-memory matrix descriptor (64 bits): start address >> 4 in bits 0-13, leading
// (K-direction) core-matrix byte offset >> 4 in bits 16-29, stride (M/N-direction 8-row
// group) byte offset >> 4 in bits 32-45, descriptor version 1 in bits 46-47, base offset 0,
// relative LBO mode, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(const void* tile, uint32_t lbo_bytes, uint32_t sbo_bytes) {
  const uint32_t a = smem_addr(tile);
  return (uint64_t)((a >> 4) & 0x3FFFu) | ((uint64_t)((lbo_bytes >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo_bytes >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor (32 bits): D format in bits 4-5, A format in bits 7-9, B format in
// bits 10-12, both operands K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits
// 24-28.  Dense, no negation, no saturation.
//   kind::f16: D 1 = f32; A/B 1 = bf16.
__host__ __device__ constexpr uint32_t idesc(uint32_t dfmt, uint32_t afmt, uint32_t bfmt, uint32_t M, uint32_t N) {
  return (dfmt << 4) | (afmt << 7) | (bfmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_bf16_f32(uint32_t M, uint32_t N) { return idesc(1, 1, 1, M, N); }

// TMEM columns: a power of two >= 32.  Executed by one whole warp; the base address is
// written to *slot (shared memory).  The warp then gives up its permit to allocate again.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// By the warp that allocated, after every use of the columns has completed.
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] . B[smem]^T for one K step; `accumulate` = 0 overwrites D.  One thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t id,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(id), "r"(accumulate)
      : "memory");
}

// The mbarrier receives one arrival when every MMA this thread issued before has completed.
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// Warp-wide load of 8 consecutive 32-bit TMEM columns of the warp's 32 lanes (lane = thread):
// taddr = base + (first lane << 16) + first column; the warp may only touch lanes
// 32 (warp % 4) .. 32 (warp % 4) + 31.  Values are valid after wait_ld().
__device__ __forceinline__ void ld_32x32b_x8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr)
               : "memory");
}

__device__ __forceinline__ void ld_32x32b_x4(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr)
               : "memory");
}

__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Generic-proxy shared-memory writes (operand tiles built by threads) made visible to the
// tensor core (async proxy) before the MMA that reads them.
__device__ __forceinline__ void fence_smem_to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Byte offset of element (row, k) of a K-major no-swizzle tile with `kbytes` bytes of K per
// row and `esize` bytes per element (the layout described at the top of this file).
__host__ __device__ constexpr uint32_t tile_offset(uint32_t row, uint32_t k, uint32_t kbytes, uint32_t esize) {
  return (row >> 3) * (kbytes * 8) + ((k * esize) >> 4) * 128 + (row & 7) * 16 + ((k * esize) & 15);
}

}  // namespace tc
}  // namespace he
