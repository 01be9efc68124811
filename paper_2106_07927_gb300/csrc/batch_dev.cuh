// Device-side structures of the batch engine shared by its kernels: stage counters, the header
// of the descriptor block, aggregation segments and the work-queue claims.
#pragma once
#include "common.cuh"

namespace r2t {

enum {
  kStCost = 0, kStRows = 1, kStShear = 2, kStWta = 3, kStMedian = 4,
  kNumCounters = 5
};

// Header of the device descriptor block. It is followed by Problem[cap], int prefix[3][cap + 1]
// (census + cost, wta, median items), then for the row and the sheared-column queue each
// AggSeg[cap] and int seg_prefix[cap + 1].
struct BatchHeader {
  int n;
  int total[kNumCounters];
  int pad;
  signed char dpl_by_d16[17];  // row-kernel disparities per lane, indexed by D / 16
};

struct AggSeg {
  int pair, begin, end, group;  // lines / chains [begin, end) of one pair, `group` per warp item
};

__device__ __forceinline__ int find_slot(const int* prefix, int n, int item) {
  int lo = 0, hi = n - 1;  // largest p with prefix[p] <= item
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int claim_block(unsigned* counter, int* s_item) {
  if (threadIdx.x == 0) *s_item = (int)atomicAdd(counter, 1u);
  __syncthreads();
  const int item = *s_item;
  __syncthreads();
  return item;
}

__device__ __forceinline__ int claim_warp(unsigned* counter) {
  int item = 0;
  if ((threadIdx.x & 31) == 0) item = (int)atomicAdd(counter, 1u);
  return __shfl_sync(0xffffffffu, item, 0);
}

}  // namespace r2t
