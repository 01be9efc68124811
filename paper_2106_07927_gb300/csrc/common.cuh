// Shared device helpers and the per-pair problem descriptor of the GB300 SGM kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace r2t {

constexpr uint16_t kInvalid = 0xFFFF;  // rejected disparity (Eq. LR_check "inv")
constexpr uint8_t kCostOutside = 255;  // cost where the matching pixel x - d lies left of the image
// Path-cost sentinel for disparities outside [0, D-1]. Any value v with v >= m + P2 - P1 for every
// reachable minimum m never wins the min of Eq. (sgm_path); 0xBFFF does so because m <= 255 + P2
// <= 16639 and P1, P2 <= 16384, and v + P1 still fits 16 bits.
constexpr uint32_t kSent = 0xBFFFu;

// Order of the D disparities inside one pixel's cost (uint8) and aggregated (uint16 / uint32)
// vectors. blocked == 0: disparity d sits at position d. blocked == 1: the disparities are owned
// by the lpl members of a lane group, dpl consecutive ones each, and are cut into chunks of
// `chunk` disparities; chunk c of member l sits at chunk slot c * lpl + l, so the members'
// accesses to chunk c are contiguous in memory (chunk = 16 for the cost, 4 for the sums).
// dpl and lpl are powers of two (their log2 in ldpl, llpl); chunk is 4 or 16 (log2 lc).
struct VolOrder {
  int blocked, ldpl, llpl;
};
__host__ __device__ inline int vol_pos(int d, VolOrder o, int lc) {
  if (!o.blocked) return d;
  const int l = d >> o.ldpl, w = d & ((1 << o.ldpl) - 1);
  return ((((w >> lc) << o.llpl) + l) << lc) + (w & ((1 << lc) - 1));
}
// Inverse of vol_pos: the disparity stored at position p.
__host__ __device__ inline int vol_index(int p, VolOrder o, int lc) {
  if (!o.blocked) return p;
  const int c = p >> lc, k = c >> o.llpl, l = c & ((1 << o.llpl) - 1);
  return (l << o.ldpl) + (k << lc) + (p & ((1 << lc) - 1));
}

__host__ __device__ inline int pow2ceil(int v) {
  int p = 1;
  while (p < v) p *= 2;
  return p;
}
__host__ __device__ inline int ilog2(int v) {
  int l = 0;
  while ((1 << (l + 1)) <= v) l++;
  return l;
}
// Disparities per lane of the short-line aggregation kernel, which fixes the volumes' order:
// blocked when the D / dpl lane members are a power of two, natural otherwise.
__host__ __device__ inline int bulk_dpl(int D) { return D % 32 == 0 ? 32 : 16; }
__host__ __device__ inline VolOrder vol_order_for(int D) {
  VolOrder o;
  const int dpl = bulk_dpl(D), lpl = D / dpl;
  o.blocked = (lpl & (lpl - 1)) == 0 ? 1 : 0;
  o.ldpl = ilog2(dpl);
  o.llpl = ilog2(lpl);
  return o;
}

// Everything a kernel needs to know about one stereo pair. Volumes are [y][x][d] with the D
// disparities of a pixel contiguous, in the order `ord`.
struct Problem {
  const uint8_t* left;
  const uint8_t* right;
  int64_t in_pitch;   // bytes
  uint16_t* disp;     // final map
  int64_t out_pitch;  // bytes
  int W, H, D;
  VolOrder ord;       // disparity order inside the cost and aggregated vectors
  uint64_t* ctl;      // census descriptors of the left / right image, [H][W]
  uint64_t* ctr;
  uint8_t* cost;      // [H][W][D]
  void* agg;          // [H][W][D], uint16 (or uint32 when wide)
  uint16_t* dl;       // [H][W] winner-takes-all map
  uint16_t* dr;       // [H][W] approximate right map
  uint32_t* kr;       // [H][W] right-disparity keys S << 8 | d, reduced with atomicMin
  uint8_t* mask;      // [H][W] 1 = kept by the left-right check
};

// Method parameters shared by every pair of a call.
struct Method {
  int cw, ch;       // census window
  int P1, P2;
  int num_paths;    // 4 or 8
  int flags;        // 1 = LR check, 2 = median
  int lr_threshold;
  int wide;         // aggregated sums kept in uint32 (needed when 8 (255 + P2) > 65535)
};

__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

// Lanes per line and disparities per lane of the aggregation for a disparity count D.
__host__ __device__ inline int agg_lanes_for(int D, int dpl) {
  int need = (D + dpl - 1) / dpl;
  int lpl = 8;
  while (lpl < need) lpl *= 2;
  return lpl;
}

}  // namespace r2t
