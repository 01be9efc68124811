// Census transform and Hamming matching cost, as block-level device routines (256 threads).
//
// Census (Sec. 2.1.1, Sec. 2.2.1): bit k of the descriptor of pixel (x, y) is 1 when the k-th
// neighbour of the cw x ch window (visited row by row, left to right, centre skipped) is darker
// than the centre; neighbours outside the image read 0 (zero-valued margin). 5x5 gives 24 bits,
// 9x7 gives 62 bits, both stored as uint64.
// Cost (Eq. image_matching): C(x, y, d) = popcount(CT_L(x, y) ^ CT_R(x - d, y)), 255 if x < d.
#pragma once
#include "common.cuh"

namespace r2t {

constexpr int kCensusTW = 64;  // census tile: 64 x 4 pixels, one per thread
constexpr int kCensusTH = 4;
constexpr int kCostTX = 128;   // cost tile: 128 pixels of one row, all D disparities

__host__ __device__ inline int census_tiles_x(int W) { return (W + kCensusTW - 1) / kCensusTW; }
__host__ __device__ inline int census_tiles_y(int H) { return (H + kCensusTH - 1) / kCensusTH; }
// Work items of the census stage of one pair: both images, all tiles.
__host__ __device__ inline int census_items(int W, int H) {
  return 2 * census_tiles_x(W) * census_tiles_y(H);
}
__host__ __device__ inline int cost_items(int W, int H) { return H * ((W + kCostTX - 1) / kCostTX); }

// Shared memory of the census routine (largest window 9 x 7).
struct CensusSmem {
  uint8_t tile[kCensusTH + 6][kCensusTW + 8];
};

template <int CW, int CH>
__device__ __forceinline__ void census_tile(const Problem& pb, int item, CensusSmem& sm) {
  constexpr int RX = CW / 2, RY = CH / 2;
  constexpr int SW = kCensusTW + 2 * RX, SH = kCensusTH + 2 * RY;
  const int ntx = census_tiles_x(pb.W), nty = census_tiles_y(pb.H);
  const int img = item / (ntx * nty);
  const int t = item % (ntx * nty);
  const int x0 = (t % ntx) * kCensusTW, y0 = (t / ntx) * kCensusTH;
  const uint8_t* src = img ? pb.right : pb.left;
  uint64_t* dst = img ? pb.ctr : pb.ctl;
  for (int i = threadIdx.x; i < SW * SH; i += blockDim.x) {
    const int ty = i / SW, tx = i - ty * SW;
    const int gx = x0 + tx - RX, gy = y0 + ty - RY;
    uint8_t v = 0;
    if (gx >= 0 && gx < pb.W && gy >= 0 && gy < pb.H) v = src[(int64_t)gy * pb.in_pitch + gx];
    sm.tile[ty][tx] = v;
  }
  __syncthreads();
  const int lx = threadIdx.x % kCensusTW, ly = threadIdx.x / kCensusTW;
  const int x = x0 + lx, y = y0 + ly;
  if (ly < kCensusTH && x < pb.W && y < pb.H) {
    const uint32_t c = sm.tile[ly + RY][lx + RX];
    uint64_t bits = 0;
    int k = 0;
#pragma unroll
    for (int j = 0; j < CH; j++) {
#pragma unroll
      for (int i = 0; i < CW; i++) {
        if (j == RY && i == RX) continue;
        bits |= (uint64_t)(sm.tile[ly + j][lx + i] < c) << k;
        k++;
      }
    }
    dst[(int64_t)y * pb.W + x] = bits;
  }
  __syncthreads();
}

__device__ __forceinline__ void census_tile_dispatch(const Problem& pb, const Method& mt, int item,
                                                     CensusSmem& sm) {
  if (mt.cw == 9)
    census_tile<9, 7>(pb, item, sm);
  else
    census_tile<5, 5>(pb, item, sm);
}

struct CostSmem {
  uint64_t r[kCostTX + 256];  // CT_R(x0 - D + 1 .. x0 + kCostTX - 1)
  uint64_t l[kCostTX];
};

// One row segment of kCostTX pixels, all disparities, written as 4-byte words (4 consecutive
// disparities stay consecutive in the volume's order, which moves chunks of 16). The same tile of
// the aggregated volume is cleared here (16-byte stores) and the tile's right-disparity keys are
// set to their maximum, so the later stages can add / atomicMin into them without separate memset
// passes; agg_bytes_per_de is 2, or 4 when wide.
__device__ __forceinline__ void cost_tile(const Problem& pb, int item, CostSmem& sm,
                                          int agg_bytes_per_de) {
  const int ntx = (pb.W + kCostTX - 1) / kCostTX;
  const int y = item / ntx;
  const int x0 = (item - y * ntx) * kCostTX;
  const int D = pb.D;
  const uint64_t* rowr = pb.ctr + (int64_t)y * pb.W;
  const uint64_t* rowl = pb.ctl + (int64_t)y * pb.W;
  for (int i = threadIdx.x; i < kCostTX + D - 1; i += blockDim.x) {
    const int xr = x0 - (D - 1) + i;
    sm.r[i] = (xr >= 0 && xr < pb.W) ? rowr[xr] : 0ull;
  }
  for (int i = threadIdx.x; i < kCostTX; i += blockDim.x)
    sm.l[i] = (x0 + i < pb.W) ? rowl[x0 + i] : 0ull;
  __syncthreads();
  const int nq = D / 4;  // 4-disparity words per pixel
  // exact it / nq for it < 2^16 (nq <= 64): multiply by ceil(2^32 / nq), keep the high word
  const uint32_t inv = (uint32_t)((0xFFFFFFFFull + nq) / nq);
  const int64_t rowe = (int64_t)y * pb.W * D;
  for (int it = threadIdx.x; it < kCostTX * nq; it += blockDim.x) {
    const int px = (int)__umulhi((uint32_t)it, inv), q = it - px * nq;
    const int x = x0 + px;
    if (x >= pb.W) continue;
    const uint64_t cl = sm.l[px];
    uint32_t word = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int d = 4 * q + j;
      uint32_t v = kCostOutside;
      if (x >= d) v = (uint32_t)__popcll(cl ^ sm.r[px + D - 1 - d]);
      word |= v << (8 * j);
    }
    *reinterpret_cast<uint32_t*>(pb.cost + rowe + (int64_t)x * D + vol_pos(4 * q, pb.ord, 4)) = word;
  }
  {
    const int npx = min(kCostTX, pb.W - x0);
    const int64_t bytes = (int64_t)npx * D * agg_bytes_per_de;  // multiple of 32
    uint4* z = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(pb.agg) +
                                        ((int64_t)y * pb.W + x0) * D * agg_bytes_per_de);
    for (int64_t i = threadIdx.x; i < bytes / 16; i += blockDim.x) z[i] = make_uint4(0, 0, 0, 0);
    for (int i = threadIdx.x; i < npx; i += blockDim.x)
      pb.kr[(int64_t)y * pb.W + x0 + i] = 0xFFFFFFFFu;
  }
  __syncthreads();
}

}  // namespace r2t
