// Disparity selection and post-processing, Sec. 2.1.2 - 2.1.3, as block-level routines.
//
// wta_lr_row: for one image row,
//   D^L(x) = smallest d with the least S(x, d)                          Eq. (wta)
//   D^R(x) = smallest d <= min(D-1, W-1-x) with the least S(x + d, d)   Eq. (right_disparity)
//   D(x)   = D^L(x) if x - D^L(x) >= 0 and |D^L(x) - D^R(x - D^L(x))| <= threshold, else inv
//                                                                        Eq. (LR_check)
// The paper reads S for D^R with strided, uncoalesced loads (Sec. 2.2.3). Here a block walks the
// row left to right in chunks of T pixels and keeps a rolling window of the last T + D pixels of
// S in shared memory, so each element of S is read from memory exactly once, with 16-byte loads.
// Ties resolve to the smallest d through one integer key (S << 8 | d) and one redux.sync.
//
// median_tile: 3x3 median of the valid pixels (Sec. 2.1.3): element [4] of the nine sorted values,
// with pixels outside the image and invalid pixels read as 0xFFFF; invalid pixels stay invalid.
// The selection network (sort the three rows, then the median of {max of minima, median of
// medians, min of maxima}) selects the same element as the paper's five bubble-sort passes with
// fewer comparators.
#pragma once
#include "common.cuh"

namespace r2t {

// Pixels per chunk of the row walk for a disparity count D (the window holds T + D pixels).
__host__ __device__ inline int wta_default_chunk(int D) { return D > 128 ? 64 : 128; }
__host__ __device__ inline size_t wta_smem_bytes(int D, int T) {
  const int ns = T + D;
  return (size_t)ns * D * 2 + (size_t)ns * 2 + (size_t)T * 2;
}

template <bool WIDE>
__device__ __forceinline__ void wta_lr_row(const Problem& pb, const Method& mt, int y, int T,
                                           uint16_t* smem, uint16_t* out_row) {
  const int W = pb.W, D = pb.D;
  const int NS = T + D;
  uint16_t* win = smem;              // NS slots x D
  uint16_t* drr = smem + NS * D;     // D^R ring, NS entries
  uint16_t* dls = drr + NS;          // D^L of the current chunk
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int64_t rowbase = (int64_t)y * W;
  int loaded = 0;
  for (int x0 = 0; x0 < W; x0 += T) {
    const int need = min(W, x0 + T + D - 1);
    // stream pixels [loaded, need) of S into their slots, 8 disparities per thread
    const int nvec = (need - loaded) * (D / 8);
    for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
      const int px = loaded + v / (D / 8);
      const int d0 = (v % (D / 8)) * 8;
      const int64_t e = (rowbase + px) * D + d0;
      uint4 o;
      if (WIDE) {
        const uint4* src = reinterpret_cast<const uint4*>(reinterpret_cast<const uint32_t*>(pb.agg) + e);
        uint4 a = src[0], b = src[1];
        uint32_t s[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int j = 0; j < 8; j++) s[j] = min(s[j], 65535u);
        o.x = s[0] | (s[1] << 16); o.y = s[2] | (s[3] << 16);
        o.z = s[4] | (s[5] << 16); o.w = s[6] | (s[7] << 16);
      } else {
        o = *reinterpret_cast<const uint4*>(reinterpret_cast<const uint16_t*>(pb.agg) + e);
      }
      *reinterpret_cast<uint4*>(win + (px % NS) * D + d0) = o;
    }
    loaded = need;
    __syncthreads();
    const int nx = min(T, W - x0);
    for (int px = warp; px < nx; px += nwarps) {
      const int x = x0 + px;
      const uint16_t* sl = win + (x % NS) * D;
      uint32_t kl = 0xFFFFFFFFu, kr = 0xFFFFFFFFu;
      const int dmax_r = min(D - 1, W - 1 - x);
      for (int d = lane; d < D; d += 32) {
        kl = min(kl, ((uint32_t)sl[d] << 8) | (uint32_t)d);
        if (d <= dmax_r) kr = min(kr, ((uint32_t)win[((x + d) % NS) * D + d] << 8) | (uint32_t)d);
      }
      kl = __reduce_min_sync(0xffffffffu, kl);
      kr = __reduce_min_sync(0xffffffffu, kr);
      if (lane == 0) {
        const uint16_t dl = (uint16_t)(kl & 0xFF), dr = (uint16_t)(kr & 0xFF);
        dls[px] = dl;
        drr[x % NS] = dr;
        pb.dl[rowbase + x] = dl;
        pb.dr[rowbase + x] = dr;
      }
    }
    __syncthreads();
    for (int px = threadIdx.x; px < nx; px += blockDim.x) {
      const int x = x0 + px;
      const int dl = dls[px];
      bool keep = true;
      if (mt.flags & 1) {
        keep = false;
        if (x - dl >= 0) {
          const int diff = dl - (int)drr[(x - dl) % NS];
          keep = (diff < 0 ? -diff : diff) <= mt.lr_threshold;
        }
      }
      out_row[x] = keep ? (uint16_t)dl : kInvalid;
      pb.mask[rowbase + x] = keep ? 1 : 0;
    }
    __syncthreads();
  }
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

// src: [H][W] map (row pitch src_pitch elements); dst: final map with a byte pitch.
__device__ __forceinline__ void median_tile(const uint16_t* src, int64_t src_pitch, int W, int H,
                                            uint16_t* dst, int64_t dst_pitch_bytes, int item,
                                            MedianSmem& sm) {
  const int ntx = (W + kMedTW - 1) / kMedTW;
  const int x0 = (item % ntx) * kMedTW, y0 = (item / ntx) * kMedTH;
  for (int i = threadIdx.x; i < (kMedTH + 2) * (kMedTW + 2); i += blockDim.x) {
    const int ty = i / (kMedTW + 2), tx = i % (kMedTW + 2);
    const int gx = x0 + tx - 1, gy = y0 + ty - 1;
    sm.t[ty][tx] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? src[(int64_t)gy * src_pitch + gx]
                                                            : kInvalid;
  }
  __syncthreads();
  const int lx = threadIdx.x % kMedTW, ly = threadIdx.x / kMedTW;
  const int x = x0 + lx, y = y0 + ly;
  if (ly < kMedTH && x < W && y < H) {
    uint32_t out = kInvalid;
    if (sm.t[ly + 1][lx + 1] != kInvalid) {
      uint32_t a0 = sm.t[ly][lx], a1 = sm.t[ly][lx + 1], a2 = sm.t[ly][lx + 2];
      uint32_t b0 = sm.t[ly + 1][lx], b1 = sm.t[ly + 1][lx + 1], b2 = sm.t[ly + 1][lx + 2];
      uint32_t c0 = sm.t[ly + 2][lx], c1 = sm.t[ly + 2][lx + 1], c2 = sm.t[ly + 2][lx + 2];
      sort3(a0, a1, a2);
      sort3(b0, b1, b2);
      sort3(c0, c1, c2);
      const uint32_t lo = max(max(a0, b0), c0);
      const uint32_t mid = med3(a1, b1, c1);
      const uint32_t hi = min(min(a2, b2), c2);
      out = med3(lo, mid, hi);
    }
    *reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(dst) + (int64_t)y * dst_pitch_bytes +
                                 2 * (int64_t)x) = (uint16_t)out;
  }
  __syncthreads();
}

}  // namespace r2t
