// Census transform fused with the Hamming matching cost, as a block-level device routine (256
// threads).
//
// Census (Sec. 2.1.1, Sec. 2.2.1): bit k of the descriptor of pixel (x, y) is 1 when the k-th
// neighbour of the cw x ch window (visited row by row, left to right, centre skipped) is darker
// than the centre; neighbours outside the image read 0 (zero-valued margin). 5x5 gives 24 bits,
// 9x7 gives 62 bits, both kept as uint64.
// Cost (Eq. image_matching): C(x, y, d) = popcount(CT_L(x, y) ^ CT_R(x - d, y)), 255 if x < d.
//
// A tile is kCostTX pixels of one row. It stages the ch image rows around the row (left segment
// x0 - rx .. x0 + kCostTX - 1 + rx, right segment x0 - D + 1 - rx .. x0 + kCostTX - 1 + rx, zero
// outside the image) in shared memory, computes the descriptors it needs there (kCostTX left,
// kCostTX + D - 1 right), then all D costs of its pixels. No descriptor map goes through HBM; the
// right descriptors shared by neighbouring tiles are computed by each of them.
#pragma once
#include "common.cuh"

namespace r2t {

constexpr int kCostTX = 128;                 // cost tile: 128 pixels of one row, all D disparities
constexpr int kImgW = kCostTX + 256 + 8;     // widest staged row: kCostTX + D - 1 + 2 rx, D <= 256

__host__ __device__ inline int cost_items(int W, int H) { return H * ((W + kCostTX - 1) / kCostTX); }

// CT_R(x0 - D + 1 + i) for i < kCostTX + D - 1 sits at r[i & 3][i >> 2]: the lanes of a warp read
// i, i - 4, i - 8, ... (4 disparities apart), which this split keeps on consecutive words.
struct CostSmem {
  uint8_t img[2][7][kImgW];  // rows y - ry .. y + ry of the left / right segment
  uint64_t r[4][(kCostTX + 256) / 4];
  uint64_t l[kCostTX];
};

// Census descriptor of the pixel whose window starts at column i of the staged rows. Bits are
// accumulated from the last neighbour to the first, each as the sign of (neighbour - centre)
// shifted in from the right, so bit k ends at position k (first 32 neighbours in the low word).
template <int CW, int CH>
__device__ __forceinline__ uint64_t census_at(const uint8_t (*rows)[kImgW], int i) {
  constexpr int RX = CW / 2, RY = CH / 2;
  const int c = rows[RY][i + RX];
  uint32_t lo = 0, hi = 0;
#pragma unroll
  for (int j = CH - 1; j >= 0; j--) {
#pragma unroll
    for (int ii = CW - 1; ii >= 0; ii--) {
      constexpr int centre = RY * CW + RX;
      const int n = j * CW + ii;  // window position, compile time after unrolling
      if (n == centre) continue;
      const int k = n < centre ? n : n - 1;          // bit of this neighbour
      const uint32_t dlt = (uint32_t)((int)rows[j][i + ii] - c);  // sign bit: 1 iff darker
      if (k >= 32)
        hi = __funnelshift_l(dlt, hi, 1);  // (hi << 1) | (dlt >> 31)
      else
        lo = __funnelshift_l(dlt, lo, 1);
    }
  }
  return (uint64_t)lo | ((uint64_t)hi << 32);
}

__device__ __forceinline__ uint32_t pack_bytes(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  return __byte_perm(__byte_perm(a, b, 0x0040), __byte_perm(c, d, 0x0040), 0x5410);
}
// Hamming distance of two descriptors of CT64 ? 64 : 32 bits.
template <bool CT64>
__device__ __forceinline__ uint32_t hamming(uint64_t a, uint64_t b) {
  return CT64 ? (uint32_t)__popcll(a ^ b) : (uint32_t)__popc((uint32_t)a ^ (uint32_t)b);
}

// The cost words of a tile for D = 4 NQ (NQ dividing 256): thread t computes word q = t % NQ of
// pixels t / NQ + k 256 / NQ, k = 0 .. kCostTX NQ / 256 - 1, unrolled, so every shared-memory
// and global offset is a constant from the thread's base. d = 4 q + j reads the right descriptor
// r index px + D - 1 - 4 q - j (the phase split puts lanes 4 disparities apart on consecutive
// words). Tiles whose pixels all have x >= D - 1 skip the test for x - d < 0.
template <bool CT64, int NQ>
__device__ __forceinline__ void cost_words(const CostSmem& sm, uint32_t* out, int x0, int npx) {
  constexpr int D = 4 * NQ, STEP = 256 / NQ, ITER = kCostTX / STEP;
  const int q = threadIdx.x % NQ, px0 = threadIdx.x / NQ;
  const uint64_t* lp = &sm.l[px0];
  const uint64_t* rp[4];
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const int i = px0 + D - 1 - 4 * q - j;
    rp[j] = &sm.r[i & 3][i >> 2];
  }
  uint32_t* o = out + px0 * NQ + q;
  const bool interior = x0 >= D - 1;  // block-uniform
#pragma unroll
  for (int it = 0; it < ITER; it++) {
    const int px = px0 + it * STEP;
    if (px < npx) {
      const uint64_t cl = lp[it * STEP];
      uint32_t v0 = hamming<CT64>(cl, rp[0][it * STEP / 4]);
      uint32_t v1 = hamming<CT64>(cl, rp[1][it * STEP / 4]);
      uint32_t v2 = hamming<CT64>(cl, rp[2][it * STEP / 4]);
      uint32_t v3 = hamming<CT64>(cl, rp[3][it * STEP / 4]);
      if (!interior) {
        const int x = x0 + px, dmax = 4 * q + 3;
        if (x < dmax) {  // x - d < 0: outside the right image
          v0 = x < dmax - 3 ? kCostOutside : v0;
          v1 = x < dmax - 2 ? kCostOutside : v1;
          v2 = x < dmax - 1 ? kCostOutside : v2;
          v3 = kCostOutside;
        }
      }
      o[it * STEP * NQ] = pack_bytes(v0, v1, v2, v3);
    }
  }
}

// One row segment of kCostTX pixels, all disparities, written as 4-byte words of 4 consecutive
// disparities, from a CW x CH census. The same tile of the aggregated volume is cleared here
// (16-byte stores) and the tile's right-disparity keys are set to their maximum, so the later
// stages can add / atomicMin into them without separate memset passes; agg_bytes_per_de is 2, or 4
// when wide.
//
// Thread t computes word q = t % (D / 4) of pixels t / (D / 4), t / (D / 4) + 256 / (D / 4), ...
// when D / 4 divides 256 (D = 16, 32, 64, 128, 256), so its r phases and offsets are fixed and
// its shared-memory addresses advance by a constant; other D take a generic loop.
template <int CW, int CH>
__device__ __forceinline__ void cost_tile(const Problem& pb, int item, CostSmem& sm,
                                          int agg_bytes_per_de) {
  constexpr int RX = CW / 2, RY = CH / 2;
  constexpr bool CT64 = CW * CH - 1 > 32;
  const int ntx = (pb.W + kCostTX - 1) / kCostTX;
  const int y = item / ntx;
  const int x0 = (item - y * ntx) * kCostTX;
  const int W = pb.W, H = pb.H, D = pb.D;
  const int npx = min(kCostTX, W - x0);
  const int nl = kCostTX + 2 * RX, nr = kCostTX + D - 1 + 2 * RX;  // staged row lengths
  const int xl0 = x0 - RX, xr0 = x0 - (D - 1) - RX;                 // their first columns
  {
    // every thread (of 256) issues all of its loads, up to NQ bytes per staged row, before
    // storing any, so their latencies overlap; nl + nr <= 2 kCostTX + 255 + 4 rx <= 256 NQ
    constexpr int NQ = 3;
    static_assert(2 * kCostTX + 255 + 16 <= 256 * NQ, "staged rows exceed the loads");
    uint8_t v[CH][NQ];
#pragma unroll
    for (int j = 0; j < CH; j++) {
      const int gy = y - RY + j;
      const bool rowin = gy >= 0 && gy < H;
      const uint8_t* lrow = pb.left + (int64_t)gy * pb.in_pitch;
      const uint8_t* rrow = pb.right + (int64_t)gy * pb.in_pitch;
#pragma unroll
      for (int q = 0; q < NQ; q++) {
        const int k = threadIdx.x + 256 * q;
        const bool isr = k >= nl;
        const int gx = (isr ? xr0 - nl : xl0) + k;
        v[j][q] = 0;
        if (k < nl + nr && rowin && gx >= 0 && gx < W) v[j][q] = __ldg(isr ? rrow + gx : lrow + gx);
      }
    }
#pragma unroll
    for (int j = 0; j < CH; j++) {
#pragma unroll
      for (int q = 0; q < NQ; q++) {
        const int k = threadIdx.x + 256 * q;
        if (k < nl + nr) {
          if (k >= nl)
            sm.img[1][j][k - nl] = v[j][q];
          else
            sm.img[0][j][k] = v[j][q];
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kCostTX + (kCostTX + D - 1); i += blockDim.x) {
    if (i < kCostTX) {
      sm.l[i] = census_at<CW, CH>(sm.img[0], i);
    } else {
      const int ir = i - kCostTX;
      const int xr = x0 - (D - 1) + ir;  // only x - d >= 0 are read, so xr < 0 stays unused
      sm.r[ir & 3][ir >> 2] = xr >= 0 ? census_at<CW, CH>(sm.img[1], ir) : 0ull;
    }
  }
  __syncthreads();
  const int nq = D / 4;  // 4-disparity words per pixel
  uint32_t* out = reinterpret_cast<uint32_t*>(pb.cost + ((int64_t)y * pb.W + x0) * D);
  if (blockDim.x == 256 && (nq == 4 || nq == 8 || nq == 16 || nq == 32 || nq == 64)) {
    switch (nq) {
      case 4: cost_words<CT64, 4>(sm, out, x0, npx); break;
      case 8: cost_words<CT64, 8>(sm, out, x0, npx); break;
      case 16: cost_words<CT64, 16>(sm, out, x0, npx); break;
      case 32: cost_words<CT64, 32>(sm, out, x0, npx); break;
      default: cost_words<CT64, 64>(sm, out, x0, npx); break;
    }
  } else if (256 % nq == 0 && blockDim.x == 256) {
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

// The two census windows of the method: 9 x 7 (62-bit descriptors) and 5 x 5 (24-bit).
__device__ __forceinline__ void cost_tile_dispatch(const Problem& pb, const Method& mt, int item,
                                                   CostSmem& sm) {
  if (mt.cw == 9)
    cost_tile<9, 7>(pb, item, sm, mt.wide ? 4 : 2);
  else
    cost_tile<5, 5>(pb, item, sm, mt.wide ? 4 : 2);
}

}  // namespace r2t
