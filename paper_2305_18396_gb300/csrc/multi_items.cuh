// multi_items.cuh -- device-side lookups into the multi-product launch table (multi.h): the
// item a block belongs to, a merged item's segment, and mask seeds.
#pragma once

#include "multi.h"

namespace he {

// Largest i with begin(i) <= b (items sorted by their prefix sums).
template <class F>
__device__ __forceinline__ u32 find_item(const MultiTable& T, u64 b, F begin) {
  u32 lo = 0, hi = T.count - 1;
  while (lo < hi) {
    const u32 mid = (lo + hi + 1) >> 1;
    if (begin(T.it[mid]) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The item's mask seed: its value, or the word it points to (a seed that a replayed CUDA
// graph takes fresh on every replay).
__device__ __forceinline__ u64 item_seed(const MultiItem& it) { return it.seed_dev ? *it.seed_dev : it.mask_seed; }
__device__ __forceinline__ u64 seg_seed(const MultiSeg& sg) { return sg.seed_dev ? *sg.seed_dev : sg.mask_seed; }

// The segment of a merged item that holds row-block Lb (the last with lb0 <= Lb).
__device__ __forceinline__ const MultiSeg& find_seg(const MultiTable& T, const MultiItem& it, u32 Lb) {
  u32 s = it.seg0;
  for (u32 k = 1; k < it.nseg; ++k)
    if (T.seg[it.seg0 + k].lb0 <= Lb) s = it.seg0 + k;
  return T.seg[s];
}

}  // namespace he
