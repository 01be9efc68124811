// Census transform and the Hamming matching cost, as two block-level device routines (256
// threads each).
//
// Census (Sec. 2.1.1, Sec. 2.2.1): bit k of the descriptor of pixel (x, y) is 1 when the k-th
// neighbour of the cw x ch window (visited row by row, left to right, centre skipped) is darker
// than the centre; neighbours outside the image read 0 (zero-valued margin). 5x5 gives 24 bits,
// 9x7 gives 62 bits, both kept as uint64.
// Cost (Eq. image_matching): C(x, y, d) = popcount(CT_L(x, y) ^ CT_R(x - d, y)), 255 if x < d.
//
// census_tile: 32 x 8 pixels of one image; the window rows around them are staged in shared
// memory (zero outside the image) and each thread computes one descriptor, stored to the pair's
// descriptor map (8 B per pixel and image; 16 B per pixel for both, which stays in L2).
// cost_tile: kCostTX pixels of one row, all D disparities. It stages the row's kCostTX left
// descriptors and the kCostTX + D right ones it reads (x0 - D .. x0 + kCostTX - 1) in shared
// memory, then each thread walks a run of consecutive pixels for one 4-disparity word: the four
// right descriptors of word q at pixel x are CT_R(x - 4q - j), j = 0..3, so from one pixel to the
// next three of them carry over in registers and one is loaded. Separate passes compute every
// descriptor once (a fused tile recomputed the D - 1 right descriptors it shares with its left
// neighbour, and tested every staged byte against the image bounds).
#pragma once
#include "common.cuh"

namespace r2t {

constexpr int kCostTX = 128;  // cost tile: 128 pixels of one row, all D disparities
constexpr int kCtTX = 32, kCtTY = 8;  // census tile: 32 x 8 pixels of one image

__host__ __device__ inline int cost_items(int W, int H) { return H * ((W + kCostTX - 1) / kCostTX); }
// Census tiles of one image; a pair has twice as many (left image first).
__host__ __device__ inline int census_items(int W, int H) {
  return ((W + kCtTX - 1) / kCtTX) * ((H + kCtTY - 1) / kCtTY);
}

struct CensusSmem {
  uint8_t win[kCtTY + 6][kCtTX + 8];  // rows y0 - ry .. y0 + 7 + ry, columns x0 - rx .. x0 + 31 + rx
};
// CT_R(x0 - D + i) sits at r[i & 3][i >> 2]: the lanes of a warp read i, i - 4, i - 8, ... (their
// words are 4 disparities apart), which this split keeps on consecutive words (no bank conflict).
struct CostSmem {
  uint64_t l[kCostTX];                // CT_L(x0 .. x0 + kCostTX - 1)
  uint64_t r[4][(kCostTX + 256) / 4]; // CT_R(x0 - D + i), i < kCostTX + D (0 outside the image)
};

// Census descriptor of the pixel whose window's top-left byte is win[0][i] (row stride kCtTX + 8).
// Bits are accumulated from the last neighbour to the first, each as the sign of
// (neighbour - centre) shifted in from the right, so bit k ends at position k (first 32
// neighbours in the low word).
template <int CW, int CH>
__device__ __forceinline__ uint64_t census_at(const uint8_t (*win)[kCtTX + 8], int i) {
  constexpr int RX = CW / 2, RY = CH / 2;
  const int c = win[RY][i + RX];
  uint32_t lo = 0, hi = 0;
#pragma unroll
  for (int j = CH - 1; j >= 0; j--) {
#pragma unroll
    for (int ii = CW - 1; ii >= 0; ii--) {
      constexpr int centre = RY * CW + RX;
      const int n = j * CW + ii;  // window position, compile time after unrolling
      if (n == centre) continue;
      const int k = n < centre ? n : n - 1;          // bit of this neighbour
      const uint32_t dlt = (uint32_t)((int)win[j][i + ii] - c);  // sign bit: 1 iff darker
      if (k >= 32)
        hi = __funnelshift_l(dlt, hi, 1);  // (hi << 1) | (dlt >> 31)
      else
        lo = __funnelshift_l(dlt, lo, 1);
    }
  }
  return (uint64_t)lo | ((uint64_t)hi << 32);
}

// Census tile `item` of the pair (items [0, census_items) the left image, then the right one)
// into pb.ct: left descriptors at [0, W H), right ones at [W H, 2 W H).
template <int CW, int CH>
__device__ __forceinline__ void census_tile(const Problem& pb, int item, CensusSmem& sm) {
  constexpr int RX = CW / 2, RY = CH / 2, NR = kCtTY + 2 * RY, NC = kCtTX + 2 * RX;
  const int W = pb.W, H = pb.H;
  const int per = census_items(W, H);
  const int img = item >= per ? 1 : 0;
  const int it = item - img * per;
  const int ntx = (W + kCtTX - 1) / kCtTX;
  const int x0 = (it % ntx) * kCtTX, y0 = (it / ntx) * kCtTY;
  const uint8_t* src = img ? pb.right : pb.left;
  for (int k = threadIdx.x; k < NR * NC; k += blockDim.x) {
    const int r = k / NC, c = k - r * NC;
    const int gy = y0 - RY + r, gx = x0 - RX + c;
    sm.win[r][c] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? __ldg(src + (int64_t)gy * pb.in_pitch + gx)
                                                           : (uint8_t)0;
  }
  __syncthreads();
  const int lx = threadIdx.x % kCtTX, ly = threadIdx.x / kCtTX;
  const int x = x0 + lx, y = y0 + ly;
  if (x < W && y < H)
    pb.ct[(int64_t)img * W * H + (int64_t)y * W + x] =
        census_at<CW, CH>(reinterpret_cast<const uint8_t(*)[kCtTX + 8]>(&sm.win[ly][0]), lx);
  __syncthreads();  // the block may take another tile into the same shared memory
}

__device__ __forceinline__ uint32_t pack_bytes(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  return __byte_perm(__byte_perm(a, b, 0x0040), __byte_perm(c, d, 0x0040), 0x5410);
}
// Hamming distance of two descriptors of CT64 ? 64 : 32 bits.
template <bool CT64>
__device__ __forceinline__ uint32_t hamming(uint64_t a, uint64_t b) {
  return CT64 ? (uint32_t)__popcll(a ^ b) : (uint32_t)__popc((uint32_t)a ^ (uint32_t)b);
}

// The cost words of a tile for D = 4 NQ (NQ = 8 .. 64 dividing 256): thread t computes word
// q = t % NQ (d = 4q .. 4q + 3) of the PPR = kCostTX NQ / 256 consecutive pixels
// px0 = (t / NQ) PPR ...; d = 4q + j at tile pixel px0 + k reads right descriptor
// i = a + k - j with a = px0 + D - 4q, a multiple of 4 (PPR is), so its phase (k - j) & 3 and word
// a / 4 + floor((k - j) / 4) are compile-time offsets. From one pixel to the next, three of the
// four descriptors carry over in registers. Tiles whose pixels all have x >= D - 1 skip the test
// for x - d < 0.
template <bool CT64, int NQ>
__device__ __forceinline__ void cost_words(const CostSmem& sm, uint32_t* out, int x0, int npx) {
  constexpr int D = 4 * NQ, PPR = kCostTX * NQ / 256;
  static_assert(PPR % 4 == 0, "runs start on a multiple of 4");
  const int q = threadIdx.x % NQ, px0 = (threadIdx.x / NQ) * PPR;
  const int aw = (px0 + D - 4 * q) >> 2;  // word of descriptor a (phase 0)
  // descriptor a + o for a compile-time offset o >= -3
#define R2T_RD(o) sm.r[(o) & 3][aw + ((o) >> 2)]
  uint64_t r0 = R2T_RD(0), r1 = R2T_RD(-1), r2 = R2T_RD(-2), r3 = R2T_RD(-3);
  uint32_t* o = out + px0 * NQ + q;
  const bool interior = x0 >= D - 1;  // block-uniform
#pragma unroll
  for (int k = 0; k < PPR; k++) {
    if (px0 + k < npx) {
      const uint64_t cl = sm.l[px0 + k];
      uint32_t v0 = hamming<CT64>(cl, r0), v1 = hamming<CT64>(cl, r1);
      uint32_t v2 = hamming<CT64>(cl, r2), v3 = hamming<CT64>(cl, r3);
      if (!interior) {
        const int x = x0 + px0 + k, dmax = 4 * q + 3;
        if (x < dmax) {  // x - d < 0: outside the right image
          v0 = x < dmax - 3 ? kCostOutside : v0;
          v1 = x < dmax - 2 ? kCostOutside : v1;
          v2 = x < dmax - 1 ? kCostOutside : v2;
          v3 = kCostOutside;
        }
      }
      o[k * NQ] = pack_bytes(v0, v1, v2, v3);
    }
    if (k + 1 < PPR) {  // one pixel right: the window of word q moves by one descriptor
      r3 = r2;
      r2 = r1;
      r1 = r0;
      r0 = R2T_RD(k + 1);
    }
  }
#undef R2T_RD
}

// One row segment of kCostTX pixels, all disparities, written as 4-byte words of 4 consecutive
// disparities, from the descriptor map pb.ct. The same tile of the aggregated volume is cleared
// here (16-byte stores) and the tile's right-disparity keys are set to their maximum, so the later
// stages can add / atomicMin into them without separate memset passes; agg_bytes_per_de is 2, or
// 4 when wide.
template <bool CT64>
__device__ __forceinline__ void cost_tile(const Problem& pb, int item, CostSmem& sm,
                                          int agg_bytes_per_de) {
  const int ntx = (pb.W + kCostTX - 1) / kCostTX;
  const int y = item / ntx;
  const int x0 = (item - y * ntx) * kCostTX;
  const int W = pb.W, D = pb.D;
  const int npx = min(kCostTX, W - x0);
  const uint64_t* ctl = pb.ct + (int64_t)y * W;
  const uint64_t* ctr = pb.ct + (int64_t)W * pb.H + (int64_t)y * W;
  for (int i = threadIdx.x; i < kCostTX + D; i += blockDim.x) {
    if (i < kCostTX) sm.l[i] = i < npx ? ctl[x0 + i] : 0ull;
    const int xr = x0 - D + i;  // only x - d >= 0 within the row are read
    sm.r[i & 3][i >> 2] = (xr >= 0 && xr < W) ? ctr[xr] : 0ull;
  }
  __syncthreads();
  const int nq = D / 4;  // 4-disparity words per pixel
  uint32_t* out = reinterpret_cast<uint32_t*>(pb.cost + ((int64_t)y * W + x0) * D);
  if (blockDim.x == 256 && (nq == 8 || nq == 16 || nq == 32 || nq == 64)) {
    switch (nq) {
      case 8: cost_words<CT64, 8>(sm, out, x0, npx); break;
      case 16: cost_words<CT64, 16>(sm, out, x0, npx); break;
      case 32: cost_words<CT64, 32>(sm, out, x0, npx); break;
      default: cost_words<CT64, 64>(sm, out, x0, npx); break;
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
        const int i = px + D - d;
        v[j] = x >= d ? hamming<CT64>(cl, sm.r[i & 3][i >> 2]) : (uint32_t)kCostOutside;
      }
      out[it] = pack_bytes(v[0], v[1], v[2], v[3]);
    }
  }
  {
    const int nv = npx * D * agg_bytes_per_de / 16;  // 16-byte pieces, D a multiple of 16
    uint4* z = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(pb.agg) +
                                        ((int64_t)y * W + x0) * D * agg_bytes_per_de);
    for (int i = threadIdx.x; i < nv; i += blockDim.x) z[i] = make_uint4(0, 0, 0, 0);
    for (int i = threadIdx.x; i < npx; i += blockDim.x) pb.kr[(int64_t)y * W + x0 + i] = 0xFFFFFFFFu;
  }
  __syncthreads();
}

// The two census windows of the method: 9 x 7 (62-bit descriptors) and 5 x 5 (24-bit).
__device__ __forceinline__ void census_tile_dispatch(const Problem& pb, const Method& mt, int item,
                                                     CensusSmem& sm) {
  if (mt.cw == 9)
    census_tile<9, 7>(pb, item, sm);
  else
    census_tile<5, 5>(pb, item, sm);
}
__device__ __forceinline__ void cost_tile_dispatch(const Problem& pb, const Method& mt, int item,
                                                   CostSmem& sm) {
  if (mt.cw == 9)
    cost_tile<true>(pb, item, sm, mt.wide ? 4 : 2);
  else
    cost_tile<false>(pb, item, sm, mt.wide ? 4 : 2);
}

}  // namespace r2t
