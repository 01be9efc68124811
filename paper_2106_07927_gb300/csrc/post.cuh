// Disparity selection and post-processing, Sec. 2.1.2 - 2.1.3, as block-level routines.
//
// wta_dr_tile: one block reads the aggregated vectors S(x, .) of T consecutive pixels of a row
// (each element of S is read from memory once, with 16-byte loads) and computes
//   D^L(x) = smallest d with the least S(x, d)                                  Eq. (wta)
// for those pixels, and its share of
//   D^R(x) = smallest d <= min(D-1, W-1-x) with the least S(x + d, d)          Eq. (right_disparity)
// for every target x whose sources x + d fall into the tile. The paper gathers S for D^R with
// strided, uncoalesced reads (Sec. 2.2.3); here every source is read once and its keys are
// scattered to its targets: targets whose D sources all lie in the tile get a plain store, the
// others (at most D - 1 per tile side) an atomicMin. Keys are S << 8 | d, so the minimum key
// carries the least S and, among equal S, the smallest d.
//
// lr_median_tile: the left-right check of Eq. (LR_check) (App. B) for a tile and its 1-pixel
// frame, then the 3x3 median of the valid pixels (Sec. 2.1.3): element [4] of the nine sorted
// values, where pixels outside the image and invalid pixels read 0xFFFF; invalid pixels stay
// invalid. The selection network (sort the three rows, then the median of {max of minima, median
// of medians, min of maxima}) selects the same element as the paper's five bubble-sort passes
// with fewer comparators.
#pragma once
#include "common.cuh"

namespace r2t {

// Default pixels per block of the WTA / right-disparity stage (T * D * 2 B of shared memory).
__host__ __device__ inline int wta_tile_px(int D) { return D > 128 ? 128 : 256; }
__host__ __device__ inline size_t wta_smem_bytes(int D, int T) { return (size_t)T * D * 2; }
__host__ __device__ inline int wta_items(int W, int H, int T) { return H * ((W + T - 1) / T); }

template <bool WIDE>
__device__ __forceinline__ void wta_dr_tile(const Problem& pb, int item, uint16_t* sm, int T) {
  const int W = pb.W, D = pb.D;
  const int ntx = (W + T - 1) / T;
  const int y = item / ntx, x0 = (item % ntx) * T;
  const int n = min(T, W - x0);
  const int64_t rowbase = (int64_t)y * W;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  // stage S of pixels [x0, x0 + n) in natural disparity order
  const int vpp = D / 8;  // 8-element vectors per pixel
  // exact v / vpp for v < 2^16: multiply by ceil(2^32 / vpp), keep the high word
  const uint32_t inv = (uint32_t)((0xFFFFFFFFull + vpp) / vpp);
  for (int v = threadIdx.x; v < n * vpp; v += blockDim.x) {
    const int px = (int)__umulhi((uint32_t)v, inv);
    const int p8 = (v - px * vpp) * 8;  // first element position of the vector
    const int64_t e = (rowbase + x0 + px) * D + p8;
    uint32_t w[4];
    if (WIDE) {
      const uint4* src = reinterpret_cast<const uint4*>(reinterpret_cast<const uint32_t*>(pb.agg) + e);
      const uint4 a = src[0], b = src[1];
      const uint32_t s[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int j = 0; j < 4; j++) w[j] = min(s[2 * j], 65535u) | (min(s[2 * j + 1], 65535u) << 16);
    } else {
      const uint4 a = *reinterpret_cast<const uint4*>(reinterpret_cast<const uint16_t*>(pb.agg) + e);
      w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    }
    uint16_t* dst = sm + px * D;
    const int d0 = vol_index(p8, pb.ord, 2), d1 = vol_index(p8 + 4, pb.ord, 2);
    *reinterpret_cast<uint2*>(dst + d0) = make_uint2(w[0], w[1]);
    *reinterpret_cast<uint2*>(dst + d1) = make_uint2(w[2], w[3]);
  }
  __syncthreads();
  for (int px = warp; px < n; px += nwarps) {
    const uint16_t* s = sm + px * D;
    uint32_t k = 0xFFFFFFFFu;
    for (int d = lane; d < D; d += 32) k = min(k, ((uint32_t)s[d] << 8) | (uint32_t)d);
    k = __reduce_min_sync(0xffffffffu, k);
    if (lane == 0) pb.dl[rowbase + x0 + px] = (uint16_t)(k & 0xFF);
  }
  // targets x in [x0 - D + 1, x0 + n) intersected with the image
  const int tlo = max(0, x0 - D + 1);
  for (int x = tlo + warp; x < x0 + n; x += nwarps) {
    uint32_t k = 0xFFFFFFFFu;
    for (int d = lane; d < D; d += 32) {
      const int src = x + d - x0;
      if (src >= 0 && src < n) k = min(k, ((uint32_t)sm[src * D + d] << 8) | (uint32_t)d);
    }
    k = __reduce_min_sync(0xffffffffu, k);
    if (lane == 0) {
      // all sources of x inside this tile: x >= x0 and min(x + D - 1, W - 1) < x0 + n
      const bool whole = x >= x0 && min(x + D - 1, W - 1) < x0 + n;
      if (whole)
        pb.kr[rowbase + x] = k;
      else if (k != 0xFFFFFFFFu)
        atomicMin(&pb.kr[rowbase + x], k);
    }
  }
  __syncthreads();
}

constexpr int kMedTW = 64;  // median tile: 64 x 4 pixels, one per thread
constexpr int kMedTH = 4;
__host__ __device__ inline int median_items(int W, int H) {
  return ((W + kMedTW - 1) / kMedTW) * ((H + kMedTH - 1) / kMedTH);
}
struct MedianSmem {
  uint16_t t[kMedTH + 2][kMedTW + 2];
};

__device__ __forceinline__ void sort2(uint32_t& a, uint32_t& b) {
  const uint32_t lo = min(a, b), hi = max(a, b);
  a = lo;
  b = hi;
}
__device__ __forceinline__ void sort3(uint32_t& a, uint32_t& b, uint32_t& c) {
  sort2(a, b);
  sort2(b, c);
  sort2(a, b);
}
__device__ __forceinline__ uint32_t med3(uint32_t a, uint32_t b, uint32_t c) {
  return max(min(a, b), min(max(a, b), c));
}

// Disparity of pixel (x, y) after the left-right check (or D^L when the check is off).
__device__ __forceinline__ uint32_t checked_disp(const Problem& pb, const Method& mt, int x, int y) {
  const int64_t row = (int64_t)y * pb.W;
  const int dl = pb.dl[row + x];
  if (!(mt.flags & 1)) return (uint32_t)dl;
  if (x - dl < 0) return kInvalid;
  const int dr = (int)(pb.kr[row + x - dl] & 0xFFu);
  const int diff = dl - dr;
  return (diff < 0 ? -diff : diff) <= mt.lr_threshold ? (uint32_t)dl : kInvalid;
}

// Final map of one 64 x 4 tile: LR check (+ median when flags & 2), plus the debug maps D^R and
// the LR mask of the tile's own pixels.
__device__ __forceinline__ void lr_median_tile(const Problem& pb, const Method& mt, int item,
                                               MedianSmem& sm) {
  const int W = pb.W, H = pb.H;
  const int ntx = (W + kMedTW - 1) / kMedTW;
  const int x0 = (item % ntx) * kMedTW, y0 = (item / ntx) * kMedTH;
  const bool median = (mt.flags & 2) != 0;
  if (median) {
    for (int i = threadIdx.x; i < (kMedTH + 2) * (kMedTW + 2); i += blockDim.x) {
      const int ty = i / (kMedTW + 2), tx = i % (kMedTW + 2);
      const int gx = x0 + tx - 1, gy = y0 + ty - 1;
      sm.t[ty][tx] =
          (gx >= 0 && gx < W && gy >= 0 && gy < H) ? (uint16_t)checked_disp(pb, mt, gx, gy) : kInvalid;
    }
    __syncthreads();
  }
  const int lx = threadIdx.x % kMedTW, ly = threadIdx.x / kMedTW;
  const int x = x0 + lx, y = y0 + ly;
  if (ly < kMedTH && x < W && y < H) {
    const int64_t p = (int64_t)y * W + x;
    uint32_t out;
    if (median) {
      out = sm.t[ly + 1][lx + 1];
      if (out != kInvalid) {
        uint32_t a0 = sm.t[ly][lx], a1 = sm.t[ly][lx + 1], a2 = sm.t[ly][lx + 2];
        uint32_t b0 = sm.t[ly + 1][lx], b1 = out, b2 = sm.t[ly + 1][lx + 2];
        uint32_t c0 = sm.t[ly + 2][lx], c1 = sm.t[ly + 2][lx + 1], c2 = sm.t[ly + 2][lx + 2];
        sort3(a0, a1, a2);
        sort3(b0, b1, b2);
        sort3(c0, c1, c2);
        const uint32_t lo = max(max(a0, b0), c0);
        const uint32_t mid = med3(a1, b1, c1);
        const uint32_t hi = min(min(a2, b2), c2);
        out = med3(lo, mid, hi);
      }
      pb.mask[p] = sm.t[ly + 1][lx + 1] != kInvalid ? 1 : 0;
    } else {
      out = checked_disp(pb, mt, x, y);
      pb.mask[p] = out != kInvalid ? 1 : 0;
    }
    pb.dr[p] = (uint16_t)(pb.kr[p] & 0xFFu);
    *reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(pb.disp) + (int64_t)y * pb.out_pitch +
                                 2 * (int64_t)x) = (uint16_t)out;
  }
  if (median) __syncthreads();
}

}  // namespace r2t
