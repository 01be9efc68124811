// Device-side structures of the batch engine shared by its kernels: stage counters, the header
// of the descriptor block, aggregation segments and the work-queue claims.
#pragma once
#include "common.cuh"

namespace r2t {

enum {
  kStCost = 0, kStRows = 1, kStShear = 2, kStWta = 3, kStMedian = 4, kStCensus = 5,
  kNumCounters = 6
};

// Kernel settings of the batch for one bucket of pairs (see tune_bucket): disparities per lane of
// the row kernel (2, 4 or 8), disparities and chains per lane of the sheared kernel (16 with 1
// or 2 chains), pixels per WTA tile (64, 128 or 256, capped so the tile's sums take at most
// 64 KB). The persistent sheared kernel holds every setting it may meet inlined, so its settings
// are kept to the two that cost the most compile time to leave out.
struct BatchTune {
  signed char row_dpl, shear_dpl, shear_cpl, pad;
  short wta_px, pad2;
};
constexpr int kTuneBuckets = 34;
// Sheared-column settings a batch bucket may take: 16 disparities per lane, 1 or 2 chains.
__host__ __device__ inline bool batch_shear_ok(int dpl, int cpl) {
  return dpl == 16 && (cpl == 1 || cpl == 2);
}
// Bucket of a pair: its disparity count (D / 16) and its size class (W * H below or at least
// 2^18 pixels, about 512 x 512).
__host__ __device__ inline int tune_bucket(int W, int H, int D) {
  return 2 * (D / 16) + ((long long)W * H >= (1 << 18) ? 1 : 0);
}

// Header of the device descriptor block. It is followed by Problem[cap], int prefix[4][cap + 1]
// (cost, wta, median and census items), then for the row and the sheared-column queue each
// AggSeg[cap] and int seg_prefix[cap + 1].
struct BatchHeader {
  int n;
  int total[kNumCounters];
  int pad;
  BatchTune tune[kTuneBuckets];
};

struct AggSeg {
  int pair, begin, end, group;  // lines / chains [begin, end) of one pair, `group` per warp item
};

// One group of the batch: pairs [p0, p0 + np) of the descriptor arrays and, per stage, its items
// [lo, hi) in that stage's numbering (item prefixes are cumulative over the whole batch). Each
// group has its own kNumCounters queue counters.
struct GroupDesc {
  int p0, np;
  int lo[kNumCounters], hi[kNumCounters];
};
constexpr int kCountersPerGroup = 8;

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
