// Census transform and the Hamming matching cost, as two block-level device routines (256
// threads each).
//
// Census (Sec. 2.1.1, Sec. 2.2.1): bit k of the descriptor of pixel (x, y) is 1 when the k-th
// neighbour of the cw x ch window (visited row by row, left to right, centre skipped) is darker
// than the centre; neighbours outside the image read 0 (zero-valued margin). 5x5 gives 24 bits,
// 9x7 gives 62 bits, both kept as uint64.
// Cost (Eq. image_matching): C(x, y, d) = popcount(CT_L(x, y) ^ CT_R(x - d, y)), 255 if x < d.
//
// census_tile: 128 x 8 pixels of one image; the window rows around them are staged in shared
// memory as 4-byte words (zero outside the image) and each thread computes the descriptors of four
// neighbouring pixels at once, four byte comparisons per 32-bit operation, stored to the pair's
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
constexpr int kCtTX = 128, kCtTY = 8;  // census tile: 128 x 8 pixels of one image

__host__ __device__ inline int cost_items(int W, int H) { return H * ((W + kCostTX - 1) / kCostTX); }
// Census tiles of one image; a pair has twice as many (left image first).
__host__ __device__ inline int census_items(int W, int H) {
  return ((W + kCtTX - 1) / kCtTX) * ((H + kCtTY - 1) / kCtTY);
}

struct CensusSmem {
  // window rows y0 - ry .. y0 + 7 + ry, columns x0 - 4 .. x0 + 131, as 4-byte words (word w holds
  // columns x0 - 4 + 4 w .. + 3, lowest address in the low byte)
  uint32_t win[kCtTY + 6][kCtTX / 4 + 2];
};
// CT_R(x0 - D + i) sits at r[i & 3][i >> 2]: the lanes of a warp read i, i - 4, i - 8, ... (their
// words are 4 disparities apart), which this split keeps on consecutive words (no bank conflict).
struct CostSmem {
  uint64_t l[kCostTX];                // CT_L(x0 .. x0 + kCostTX - 1)
  uint64_t r[4][(kCostTX + 256) / 4]; // CT_R(x0 - D + i), i < kCostTX + D (0 outside the image)
};

// Bytewise unsigned a < b of four byte lanes, in bit 7 of each byte (other bits undefined).
// t = (a | 0x80) - (b & 0x7F) per byte lies in 1 .. 255, so no borrow crosses a byte, and its bit 7
// says a_low >= b_low (the low seven bits); with the top bits a7, b7:
// a < b = (!a7 & b7) | (a7 == b7 & !(a_low >= b_low)).
__device__ __forceinline__ uint32_t bytes_lt(uint32_t a, uint32_t b_low, uint32_t b) {
  const uint32_t t = (a | 0x80808080u) - b_low;
  return (~a & b) | (~(a ^ b) & ~t);
}

// Census descriptors of the four pixels x .. x + 3 of one row, x = x0 + 4 lane, from the window
// words of rows r0 .. r0 + ch - 1 (r0 = the pixels' row - ry + ry = tile row). The four pixels'
// comparisons with neighbour k run in one word: the neighbour bytes of offset dx are the window
// bytes 4 + dx .. 7 + dx of the three words lane, lane + 1, lane + 2. Neighbour k's four result
// bits (bit 7 of each byte) are shifted into byte lane p of the accumulator of group k / 8, which
// after eight neighbours holds bit k % 8 of pixel p's descriptor byte k / 8 at position k % 8; a
// byte transpose of the accumulators gives the four descriptors.
template <int CW, int CH>
__device__ __forceinline__ void census_x4(const uint32_t (*win)[kCtTX / 4 + 2], int lane,
                                          uint64_t* out) {
  constexpr int RX = CW / 2, RY = CH / 2;
  constexpr int NB = CW * CH - 1;     // descriptor bits
  constexpr int NG = (NB + 7) / 8;    // groups of eight neighbours
  constexpr int centre = RY * CW + RX;
  const uint32_t c = win[RY][lane + 1];
  const uint32_t c_low = c & 0x7F7F7F7Fu;
  uint32_t acc[8];
#pragma unroll
  for (int g = 0; g < 8; g++) acc[g] = 0;
#pragma unroll
  for (int j = 0; j < CH; j++) {
    const uint32_t w0 = win[j][lane], w1 = win[j][lane + 1], w2 = win[j][lane + 2];
#pragma unroll
    for (int i = 0; i < CW; i++) {
      const int n = j * CW + i;  // window position, compile time after unrolling
      if (n == centre) continue;
      const int k = n < centre ? n : n - 1;
      const int o = 4 + i - RX;  // byte offset of the neighbour word in w0 w1 w2
      uint32_t nb;
      if (o == 4)
        nb = w1;
      else if (o == 8)
        nb = w2;
      else if (o < 4)
        nb = __byte_perm(w0, w1, (o) | ((o + 1) << 4) | ((o + 2) << 8) | ((o + 3) << 12));
      else
        nb = __byte_perm(w1, w2, (o - 4) | ((o - 3) << 4) | ((o - 2) << 8) | ((o - 1) << 12));
      acc[k >> 3] = (acc[k >> 3] >> 1) | (bytes_lt(nb, c_low, c) & 0x80808080u);
    }
  }
  if (NB % 8) acc[NG - 1] >>= 8 - NB % 8;  // a last group of fewer than eight bits
  // 4 x 4 byte transposes: descriptor byte g of pixel p = byte p of acc[g]
  uint32_t lo[4], hi[4];
  {
    const uint32_t u0 = __byte_perm(acc[0], acc[1], 0x5140), u1 = __byte_perm(acc[0], acc[1], 0x7362);
    const uint32_t u2 = __byte_perm(acc[2], acc[3], 0x5140), u3 = __byte_perm(acc[2], acc[3], 0x7362);
    lo[0] = __byte_perm(u0, u2, 0x5410);
    lo[1] = __byte_perm(u0, u2, 0x7632);
    lo[2] = __byte_perm(u1, u3, 0x5410);
    lo[3] = __byte_perm(u1, u3, 0x7632);
  }
  if (NG > 4) {
    const uint32_t u0 = __byte_perm(acc[4], acc[5], 0x5140), u1 = __byte_perm(acc[4], acc[5], 0x7362);
    const uint32_t u2 = __byte_perm(acc[6], acc[7], 0x5140), u3 = __byte_perm(acc[6], acc[7], 0x7362);
    hi[0] = __byte_perm(u0, u2, 0x5410);
    hi[1] = __byte_perm(u0, u2, 0x7632);
    hi[2] = __byte_perm(u1, u3, 0x5410);
    hi[3] = __byte_perm(u1, u3, 0x7632);
  } else {
    hi[0] = hi[1] = hi[2] = hi[3] = 0;
  }
#pragma unroll
  for (int p = 0; p < 4; p++) out[p] = (uint64_t)lo[p] | ((uint64_t)hi[p] << 32);
}

// Census tile `item` of the pair (items [0, census_items) the left image, then the right one)
// into pb.ct: left descriptors at [0, W H), right ones at [W H, 2 W H). Warp w computes row
// y0 + w; lane l the pixels x0 + 4 l .. + 3.
template <int CW, int CH>
__device__ __forceinline__ void census_tile(const Problem& pb, int item, CensusSmem& sm) {
  constexpr int RY = CH / 2, NR = kCtTY + 2 * RY, NWD = kCtTX / 4 + 2;
  const int W = pb.W, H = pb.H;
  const int per = census_items(W, H);
  const int img = item >= per ? 1 : 0;
  const int it = item - img * per;
  const int ntx = (W + kCtTX - 1) / kCtTX;
  const int x0 = (it % ntx) * kCtTX, y0 = (it / ntx) * kCtTY;
  const uint8_t* src = img ? pb.right : pb.left;
  for (int k = threadIdx.x; k < NR * NWD; k += blockDim.x) {
    const int r = k / NWD, cw = k - r * NWD;
    const int gy = y0 - RY + r, gx = x0 - 4 + 4 * cw;
    uint32_t v = 0;
    if (gy >= 0 && gy < H) {
      const uint8_t* row = src + (int64_t)gy * pb.in_pitch;
      if (gx >= 0 && gx + 3 < W && ((reinterpret_cast<uintptr_t>(row + gx) & 3) == 0)) {
        v = __ldg(reinterpret_cast<const uint32_t*>(row + gx));
      } else {
#pragma unroll
        for (int b = 0; b < 4; b++)
          if (gx + b >= 0 && gx + b < W) v |= (uint32_t)__ldg(row + gx + b) << (8 * b);
      }
    }
    sm.win[r][cw] = v;
  }
  __syncthreads();
  const int ly = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int x = x0 + 4 * lane, y = y0 + ly;
  if (ly < kCtTY && x < W && y < H) {
    uint64_t d[4];
    census_x4<CW, CH>(reinterpret_cast<const uint32_t(*)[NWD]>(&sm.win[ly][0]), lane, d);
    uint64_t* o = pb.ct + (int64_t)img * W * H + (int64_t)y * W + x;
#pragma unroll
    for (int p = 0; p < 4; p++)
      if (x + p < W) o[p] = d[p];
  }
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
