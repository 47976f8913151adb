// multi.h -- descriptor table and launchers of the multi-product launch (multi.cu).
#pragma once

#include "he_common.cuh"
#include "kernels.h"

namespace he {

constexpr int kMaxMulti = 64;  // products per multi-product launch

// One request of a merged launch item (below): its own inputs, outputs and mask seed, and
// the first row-block it occupies in the item.
struct MultiSeg {
  const u64* ct_in;     // input ciphertexts, wire format
  u64* out;             // compact output ciphertexts
  u64 mask_seed;
  const u64* seed_dev;  // HE_SEED_DEVICE: the seed is read from here when the kernels run
  u32 lb0, pad;
};

// One item of a multi-product launch: a product, or (nseg > 0) several products that share
// their encoded weights, shape and blocking, merged into one whose row-blocks are the
// requests' row-blocks back to back -- every weight stage then serves all their rows.  A
// merged item's multiply-accumulate writes both components to the workspace (c0_ntt,
// c1_ntt); the inverse transforms write each request's compact output with its own seed.
// *_begin: first block of this item in each kernel's grid (prefix sums in item order).
struct MultiItem {
  const u64* ct_in;  // input ciphertexts, wire format
  const u64* pt;     // encoded weights (slot-chunked)
  u64* out;          // output ciphertexts (full or compact)
  u64* ctN;          // workspace: NTT of the inputs (slot-chunked)
  u64* c0_ntt;       // workspace (compact output only): NTT-domain c0 of every output
  u64 mask_seed;
  const u64* seed_dev;  // HE_SEED_DEVICE: the seed is read from here when the kernels run
  u64 fwd_begin, mac_begin, inv_begin, c0_begin, tc_begin;
  u32 nI, nJ, nLb, logkb;
  u32 compact, tilesR, tilesC, tc;  // tc: operands in the stage-tiled layout, tensor-core MAC
  u64* c1_ntt;                       // workspace (merged items): NTT-domain c1 of every output
  u32 seg0, nseg;                    // merged items: segments seg0 .. seg0 + nseg - 1
  // coset products (coset.cuh; tc is set too): the inputs' coset transforms in ctN (rows
  // (2 Lb + c) G + g, 2D slots per prime), the multiply-accumulate's sums in acc
  // ([out ct][2][L][2N]); cfwd_begin / cinv_begin: first block in the coset grids
  u64* acc;
  u64 cfwd_begin, cinv_begin;
  u32 coset, logD;
  // coset products of at most 64 k-blocks: the row-major tensor-core MAC (mac_tcr.cuh), weights
  // as row-major digit tiles; tcr_begin: first unit in its grid
  u64 tcr_begin;
  u32 tcr, pad2;
};

struct MultiTable {
  u32 count, nseg;
  MultiItem it[kMaxMulti];
  MultiSeg seg[kMaxMulti];
};

cudaError_t configure_multi_kernels();
cudaError_t configure_coset_kernels();  // coset.cu (called by configure_multi_kernels)
u32 mac_tile_rows();
u32 mac_tile_cols();
cudaError_t launch_fwd_multi(const Consts& C, const MultiTable& T, u64 blocks, cudaStream_t st);
cudaError_t launch_mac_multi(const Consts& C, const MultiTable& T, u64 blocks, int* err, cudaStream_t st);
// The tensor-core multiply-accumulate of the products flagged tc (units: their work units,
// spread over one block per SM).
cudaError_t launch_mac_tc_multi(const Consts& C, const MultiTable& T, u64 blocks, int* err, cudaStream_t st);
cudaError_t launch_inv_multi(const Consts& C, const MultiTable& T, u64 blocks, cudaStream_t st);
cudaError_t launch_c0_multi(const Consts& C, const MultiTable& T, u64 blocks, u32 c0_words, cudaStream_t st);
// Coset products: the forward transforms of their inputs (one block per input polynomial)
// and the inverse transforms, fold and mask of their outputs (one block per output
// component), each as one grid over the coset items of the table.
cudaError_t launch_coset_fwd_multi(const Consts& C, const MultiTable& T, u64 blocks, cudaStream_t st);
// The row-major tensor-core multiply-accumulate of the items flagged tcr (units: theirs).
cudaError_t launch_mac_tcr_multi(const Consts& C, const MultiTable& T, u64 units, int* err, cudaStream_t st);
cudaError_t launch_coset_inv_multi(const Consts& C, const MultiTable& T, u64 blocks, cudaStream_t st);
// Encoded weights of coset products: per weight block the zero-padded length-2D transform
// of its pi_A block, as bf16 digit tiles over 2D slots (row-major digit tiles when tcr);
// `batch` same-shape matrices.
cudaError_t launch_coset_encode_weights(const Consts& C, const u64* W, u32 k, u32 n, Blk b, u32 nI, u32 nJ, u32 batch,
                                        u32 tcr, u64* pt, cudaStream_t st);
// The inverse-NTT grid and the c0 grid as one launch where inv_c0_fused(C), else two.
bool inv_c0_fused(const Consts& C);
cudaError_t launch_inv_c0_multi(const Consts& C, const MultiTable& T, u64 inv_blocks, u64 c0_blocks, u32 c0_words,
                                cudaStream_t st);

}  // namespace he
