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

__host__ __device__ inline int pow2ceil(int v) {
  int p = 1;
  while (p < v) p *= 2;
  return p;
}

// Everything a kernel needs to know about one stereo pair. Volumes are [y][x][d] with the D
// disparities of a pixel contiguous and in natural order.
struct Problem {
  const uint8_t* left;
  const uint8_t* right;
  int64_t in_pitch;   // bytes
  uint16_t* disp;     // final map
  int64_t out_pitch;  // bytes
  int W, H, D;
  uint8_t* cost;      // [H][W][D]
  uint64_t* ct;       // [2][H][W] census descriptors of the left, then the right image
  void* agg;          // [H][W][D], uint16 (or uint32 when wide)
  uint16_t* dl;       // [H][W] winner-takes-all map
  uint16_t* dr;       // [H][W] approximate right map
  uint32_t* kr;       // [H][W] right-disparity keys S << 8 | d, reduced with atomicMin
  uint8_t* mask;      // [H][W] 1 = kept by the left-right check
  float* disp_f;      // sub-pixel final map (caller's, out_pitch bytes per row); NULL: uint16 map
  uint8_t* flip;      // [2][H][W] right and left image, each flipped horizontally (exact check)
  uint16_t* dp;       // [H][W] D^L of that swapped, flipped pair (exact check); NULL: approximate
  uint2* nst;         // [2][H][W] patch sum and factor of the reference / matching image (NCC)
  int32_t* nsv;       // [2][H][W] exact patch variance N sum a^2 - (sum a)^2 of both images (NCC)
  unsigned* fault;    // range-check record {site, 0, byte offset (int64)} (RES2TAC_CHECK_BOUNDS)
};

// Debug build with range checks (compiled with -DRES2TAC_CHECK_BOUNDS): the checked global
// accesses of the aggregation and WTA kernels first test that [p, p + bytes) lies inside their
// buffer [lo, lo + size); a failing test records its site and byte offset in pb.fault (the first
// failure wins) and the access is skipped. Nothing traps. In the normal build every test is the
// constant true and compiles away.
// Sites: 1 row-kernel cost load, 2 row-kernel add into S, 3 sheared-kernel cost copy, 4 / 5
// sheared-kernel bulk add (run before / after a wrap), 6 WTA staging copy of S, 7 WTA store of D^L.
// Site 8 is recorded in every build: a block of the tensor-core cost kernel whose MMAs did not
// complete within its poll limit (it stores no cost).
#ifdef RES2TAC_CHECK_BOUNDS
static __device__ __noinline__ bool check_range(unsigned* fault, const void* p, int64_t bytes,
                                                const void* lo, int64_t size, int site) {
  const int64_t off = static_cast<const char*>(p) - static_cast<const char*>(lo);
  const bool ok = off >= 0 && bytes >= 0 && off + bytes <= size;
  if (!ok && fault && atomicCAS(fault, 0u, (unsigned)site) == 0u)
    reinterpret_cast<long long*>(fault)[1] = off;
  return ok;
}
#define R2T_CHECKED(pb, p, bytes, lo, size, site) \
  r2t::check_range((pb).fault, (p), (bytes), (lo), (size), (site))
#else
#define R2T_CHECKED(pb, p, bytes, lo, size, site) true
#endif

// Method parameters shared by every pair of a call.
struct Method {
  int cw, ch;       // census window
  int P1, P2;
  int num_paths;    // 4 or 8
  int flags;        // 1 = LR check, 2 = median, 4 = exact D^R for the check, 8 = NCC cost
  //                   (cw = ch = n: the NCC patch)
  int lr_threshold;
  int wide;         // aggregated sums kept in uint32 (needed when 8 (255 + P2) > 65535)
};

__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

}  // namespace r2t
