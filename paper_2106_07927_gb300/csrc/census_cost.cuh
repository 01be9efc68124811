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

// CT_R(x0 - D + 1 + i) for i < kCostTX + D - 1 sits at r[i & 3][i >> 2]: the lanes of a warp read
// i, i - 4, i - 8, ... (4 disparities apart), which this split keeps on consecutive words.
struct CostSmem {
  uint64_t r[4][(kCostTX + 256) / 4];
  uint64_t l[kCostTX];
};

__device__ __forceinline__ uint32_t pack_bytes(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  return __byte_perm(__byte_perm(a, b, 0x0040), __byte_perm(c, d, 0x0040), 0x5410);
}
// Hamming distance of two descriptors of CT64 ? 64 : 32 bits.
template <bool CT64>
__device__ __forceinline__ uint32_t hamming(uint64_t a, uint64_t b) {
  return CT64 ? (uint32_t)__popcll(a ^ b) : (uint32_t)__popc((uint32_t)a ^ (uint32_t)b);
}

// One row segment of kCostTX pixels, all disparities, written as 4-byte words of 4 consecutive
// disparities. The same tile of the aggregated volume is cleared here (16-byte stores) and the
// tile's right-disparity keys are set to their maximum, so the later stages can add / atomicMin
// into them without separate memset passes; agg_bytes_per_de is 2, or 4 when wide. CT64: the
// census descriptors use more than 32 bits.
//
// Thread t computes word q = t % (D / 4) of pixels t / (D / 4), t / (D / 4) + 256 / (D / 4), ...
// when D / 4 divides 256 (D = 16, 32, 64, 128, 256), so its r phases and offsets are fixed and
// its shared-memory addresses advance by a constant; other D take a generic loop.
template <bool CT64>
__device__ __forceinline__ void cost_tile(const Problem& pb, int item, CostSmem& sm,
                                          int agg_bytes_per_de) {
  const int ntx = (pb.W + kCostTX - 1) / kCostTX;
  const int y = item / ntx;
  const int x0 = (item - y * ntx) * kCostTX;
  const int D = pb.D;
  const int npx = min(kCostTX, pb.W - x0);
  const uint64_t* rowr = pb.ctr + (int64_t)y * pb.W;
  const uint64_t* rowl = pb.ctl + (int64_t)y * pb.W;
  for (int i = threadIdx.x; i < kCostTX + D - 1; i += blockDim.x) {
    const int xr = x0 - (D - 1) + i;
    sm.r[i & 3][i >> 2] = (xr >= 0 && xr < pb.W) ? rowr[xr] : 0ull;
  }
  for (int i = threadIdx.x; i < kCostTX; i += blockDim.x)
    sm.l[i] = (x0 + i < pb.W) ? rowl[x0 + i] : 0ull;
  __syncthreads();
  const int nq = D / 4;  // 4-disparity words per pixel
  uint32_t* out = reinterpret_cast<uint32_t*>(pb.cost + ((int64_t)y * pb.W + x0) * D);
  if (256 % nq == 0 && blockDim.x == 256) {
    const int q = threadIdx.x % nq, step = 256 / nq;  // step is a multiple of 4
    int px = threadIdx.x / nq;
    // d = 4 q + j reads r index px + D - 1 - 4 q - j: phase and row offset per j
    const uint64_t* rp[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int i = px + D - 1 - 4 * q - j;
      rp[j] = &sm.r[i & 3][i >> 2];
    }
    const int dmax = 4 * q + 3;
    for (; px < npx; px += step) {
      const uint64_t cl = sm.l[px];
      uint32_t v0 = hamming<CT64>(cl, *rp[0]), v1 = hamming<CT64>(cl, *rp[1]);
      uint32_t v2 = hamming<CT64>(cl, *rp[2]), v3 = hamming<CT64>(cl, *rp[3]);
      const int x = x0 + px;
      if (x < dmax) {  // x - d < 0: outside the right image
        v0 = x < dmax - 3 ? kCostOutside : v0;
        v1 = x < dmax - 2 ? kCostOutside : v1;
        v2 = x < dmax - 1 ? kCostOutside : v2;
        v3 = kCostOutside;
      }
      out[px * nq + q] = pack_bytes(v0, v1, v2, v3);
#pragma unroll
      for (int j = 0; j < 4; j++) rp[j] += step / 4;
    }
  } else {
    // exact it / nq for it < 2^16 (nq <= 64): multiply by ceil(2^32 / nq), keep the high word
    const uint32_t inv = (uint32_t)((0xFFFFFFFFull + nq) / nq);
    for (int it = threadIdx.x; it < npx * nq; it += blockDim.x) {
      const int px = (int)__umulhi((uint32_t)it, inv), q = it - px * nq;
      const int x = x0 + px;
      const uint64_t cl = sm.l[px];
      uint32_t v[4];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const int d = 4 * q + j;
        const int i = px + D - 1 - d;
        v[j] = x >= d ? hamming<CT64>(cl, sm.r[i & 3][i >> 2]) : (uint32_t)kCostOutside;
      }
      out[it] = pack_bytes(v[0], v[1], v[2], v[3]);
    }
  }
  {
    const int nv = npx * D * agg_bytes_per_de / 16;  // 16-byte pieces, D a multiple of 16
    uint4* z = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(pb.agg) +
                                        ((int64_t)y * pb.W + x0) * D * agg_bytes_per_de);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) z[i] = make_uint4(0, 0, 0, 0);
    for (int i = threadIdx.x; i < npx; i += blockDim.x)
      pb.kr[(int64_t)y * pb.W + x0 + i] = 0xFFFFFFFFu;
  }
  __syncthreads();
}

// Census descriptors of the method's window fit 32 bits when cw * ch - 1 <= 32 (5 x 5).
__device__ __forceinline__ void cost_tile_dispatch(const Problem& pb, const Method& mt, int item,
                                                   CostSmem& sm) {
  if (mt.cw * mt.ch - 1 > 32)
    cost_tile<true>(pb, item, sm, mt.wide ? 4 : 2);
  else
    cost_tile<false>(pb, item, sm, mt.wide ? 4 : 2);
}

}  // namespace r2t
