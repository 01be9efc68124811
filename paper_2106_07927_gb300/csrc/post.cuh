// Disparity selection and post-processing, Sec. 2.1.2 - 2.1.3, as block-level routines.
//
// wta_dr_staged: for T consecutive pixels of a row, staged in shared memory as one contiguous
// run, each pixel's aggregated vector S(x, .) is read once, by one warp with its lanes on
// consecutive disparities, and gives
//   D^L(x) = smallest d with the least S(x, d)                                  Eq. (wta)
// as a warp minimum, and its share of
//   D^R(x) = smallest d <= min(D-1, W-1-x) with the least S(x + d, d)          Eq. (right_disparity)
// for every target x' = x - d. The paper gathers S for D^R with strided, uncoalesced reads
// (Sec. 2.2.3); here every source is read once and each of its keys is scattered to its target.
// Keys are S << 8 | d, so the minimum key carries the least S and, among equal S, the smallest d.
// Sub-pixel refinement (Sec. 2.1.3): the parabola through S(x, d-1), S(x, d), S(x, d+1) at
// d = D^L(x) has its minimum at d + delta with
//   delta = (a - b) / (2 (a + b)),  a = S(d-1) - S(d),  b = S(d+1) - S(d),
// taken in fp32 with correctly rounded division and addition; D^L = 0 and D^L = D - 1 have one
// neighbour only and stay integral. a > 0 because d is the smallest minimiser and b >= 0, so the
// denominator is positive and delta lies in (-1/2, 1/2]. It runs in the left-right / median
// stage, one thread per pixel, which reads the three costs (adjacent in the volume) directly.
//
// lr_median_tile: the left-right check of Eq. (LR_check) (App. B) for a tile and its 1-pixel
// frame, then the 3x3 median of the valid pixels (Sec. 2.1.3): element [4] of the nine sorted
// values, where pixels outside the image and invalid pixels read 0xFFFF; invalid pixels stay
// invalid. The selection network (sort the three rows, then the median of {max of minima, median
// of medians, min of maxima}) selects the same element as the paper's five bubble-sort passes
// with fewer comparators.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace r2t {

__host__ __device__ inline int wta_items(int W, int H, int T) { return H * ((W + T - 1) / T); }

// The keys of one pixel x (tile position px): each lane offers its keys to targets x - d with a
// shared-memory atomicMin (consecutive lanes hit consecutive targets, so no bank conflict); returns
// the warp minimum, whose low byte is D^L(x).
template <int NDL, bool EXACT>
__device__ __forceinline__ uint32_t wta_keys(const Problem& pb, int x, int px, uint32_t* keys,
                                             int lane, const uint32_t (&s)[NDL]) {
  const int D = EXACT ? 32 * NDL : pb.D;
  uint32_t* kt = keys + (px + D - 1 - lane);  // kt[-32 i] is the key of target x - d
  uint32_t key[NDL];
  uint32_t kl = 0xFFFFFFFFu;
#pragma unroll
  for (int i = 0; i < NDL; i++) {
    const int d = lane + 32 * i;
    key[i] = (EXACT || d < D) ? (s[i] << 8) | (uint32_t)d : 0xFFFFFFFFu;
    kl = min(kl, key[i]);
  }
  if (EXACT && x >= D - 1) {  // warp-uniform: every target x - d lies in the image
#pragma unroll
    for (int i = 0; i < NDL; i++) atomicMin(kt - 32 * i, key[i]);
  } else {
#pragma unroll
    for (int i = 0; i < NDL; i++) {
      const int d = lane + 32 * i;
      if ((EXACT || d < D) && d <= x) atomicMin(kt - 32 * i, key[i]);
    }
  }
  return __reduce_min_sync(0xffffffffu, kl);
}

// Sub-pixel D^L of pixel p (Sec. 2.1.3) from its integer D^L d and the aggregated costs at d - 1,
// d, d + 1 (saturated to 16 bits as in the uint16 volume).
template <bool WIDE>
__device__ __forceinline__ float refine_subpixel(const Problem& pb, int64_t p, int d) {
  float v = (float)d;
  if (d >= 1 && d <= pb.D - 2) {
    const int64_t i = p * pb.D + d;
    uint32_t sm, s0, sp;
    if (WIDE) {
      const uint32_t* S = reinterpret_cast<const uint32_t*>(pb.agg);
      sm = min(S[i - 1], 65535u);
      s0 = min(S[i], 65535u);
      sp = min(S[i + 1], 65535u);
    } else {
      const uint16_t* S = reinterpret_cast<const uint16_t*>(pb.agg);
      sm = S[i - 1];
      s0 = S[i];
      sp = S[i + 1];
    }
    const int a = (int)(sm - s0), b = (int)(sp - s0);  // a > 0, b >= 0
    v = __fadd_rn(v, __fdiv_rn((float)(a - b), (float)(2 * (a + b))));
  }
  return v;
}

// One tile of T pixels of a row (256 threads): its sums are staged in shared memory first, all
// threads copying the tile's contiguous run of S (n pixels x D sums) with 16-byte cp.async
// copies, so the whole tile is in flight at once; then warp w takes pixels w, w + 8, ... from
// shared memory. Targets whose sources all lie in the tile are stored, the others (at most
// D - 1 per tile side) merged with a global atomicMin. T pixels with T * D * bytes-per-sum
// <= 64 KB (wta_staged_px). Shared memory: the run, then T + D - 1 keys.
__host__ __device__ inline int wta_staged_px(int D, bool wide, int T) {
  const int cap = 65536 / (D * (wide ? 4 : 2));
  return T < cap ? T : cap;
}
__host__ __device__ inline size_t wta_staged_smem_bytes(int D, bool wide, int T) {
  return (size_t)T * D * (wide ? 4 : 2) + (size_t)(T + D - 1) * 4;
}

template <bool WIDE, int NDL, bool EXACT>
__device__ __forceinline__ void wta_dr_staged_t(const Problem& pb, int item, uint8_t* smem,
                                                int T) {
  constexpr int BPE = WIDE ? 4 : 2;
  const int W = pb.W, D = EXACT ? 32 * NDL : pb.D;
  const int ntx = (W + T - 1) / T;
  const int y = item / ntx, x0 = (item - y * ntx) * T;
  const int n = min(T, W - x0);
  const int64_t rowbase = (int64_t)y * W;
  uint32_t* keys = reinterpret_cast<uint32_t*>(smem + (size_t)T * D * BPE);
  {
    const uint8_t* src = reinterpret_cast<const uint8_t*>(pb.agg) + (rowbase + x0) * D * BPE;
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem);
    const int pieces = n * D * BPE / 16;  // D % 16 == 0
    const int64_t vbytes = (int64_t)W * pb.H * D * BPE;  // extent of S (range checks)
    (void)vbytes;
    for (int i = threadIdx.x; i < pieces; i += blockDim.x)
      if (R2T_CHECKED(pb, src + 16 * (int64_t)i, 16, pb.agg, vbytes, 6))
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16 * i),
                     "l"(src + 16 * (int64_t)i));
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  const int ntar = T + D - 1;  // targets x0 - D + 1 .. x0 + T - 1
  for (int i = threadIdx.x; i < ntar; i += blockDim.x) keys[i] = 0xFFFFFFFFu;
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5, warp = threadIdx.x >> 5;
  uint32_t mine = 0;  // lane k keeps the key of the warp's k-th pixel (T / nw <= 32 pixels)
  int it = 0;
  for (int px = warp; px < n; px += nw, it++) {
    uint32_t sv[NDL];
#pragma unroll
    for (int i = 0; i < NDL; i++) {
      const int d = lane + 32 * i;
      sv[i] = 0xFFFFu;
      if (EXACT || d < D) {
        if (WIDE)
          sv[i] = min(reinterpret_cast<const uint32_t*>(smem)[px * D + d], 65535u);
        else
          sv[i] = reinterpret_cast<const uint16_t*>(smem)[px * D + d];
      }
    }
    const uint32_t kl = wta_keys<NDL, EXACT>(pb, x0 + px, px, keys, lane, sv);
    mine = lane == it ? kl : mine;
  }
  if (lane < it && R2T_CHECKED(pb, pb.dl + rowbase + x0 + warp + nw * lane, 2, pb.dl,
                              2 * (int64_t)W * pb.H, 7))
    pb.dl[rowbase + x0 + warp + nw * lane] = (uint16_t)(mine & 0xFFu);  // D^L
  __syncthreads();
  for (int i = threadIdx.x; i < ntar; i += blockDim.x) {
    const int x = x0 - D + 1 + i;
    if (x < 0 || x >= x0 + n) continue;
    const uint32_t k = keys[i];
    if (k == 0xFFFFFFFFu) continue;
    const bool whole = x >= x0 && min(x + D - 1, W - 1) < x0 + n;
    if (whole)
      pb.kr[rowbase + x] = k;
    else
      atomicMin(&pb.kr[rowbase + x], k);
  }
}

template <bool WIDE>
__device__ __forceinline__ void wta_dr_staged(const Problem& pb, int item, uint8_t* smem, int T) {
#define R2T_WTA_STAGED(N)                                 \
  case N:                                                 \
    if (pb.D == 32 * N)                                   \
      wta_dr_staged_t<WIDE, N, true>(pb, item, smem, T);  \
    else                                                  \
      wta_dr_staged_t<WIDE, N, false>(pb, item, smem, T); \
    break;
  switch ((pb.D + 31) / 32) {
    R2T_WTA_STAGED(1)
    R2T_WTA_STAGED(2)
    R2T_WTA_STAGED(3)
    R2T_WTA_STAGED(4)
    R2T_WTA_STAGED(5)
    R2T_WTA_STAGED(6)
    R2T_WTA_STAGED(7)
    default:
      R2T_WTA_STAGED(8)
  }
#undef R2T_WTA_STAGED
}

constexpr int kMedTW = 64;  // median tile: 64 x 4 pixels, one per thread
constexpr int kMedTH = 4;
__host__ __device__ inline int median_items(int W, int H) {
  return ((W + kMedTW - 1) / kMedTW) * ((H + kMedTH - 1) / kMedTH);
}
// Tile plus frame of checked disparities: uint16 values, or (sub-pixel) the bit patterns of
// non-negative floats, which order as unsigned integers do, with +infinity as the invalid value.
template <bool SUB>
struct MedianSmemT {
  typename std::conditional<SUB, uint32_t, uint16_t>::type t[kMedTH + 2][kMedTW + 2];
};
using MedianSmem = MedianSmemT<false>;
constexpr uint32_t kInvalidF = 0x7F800000u;  // +infinity

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

// Disparity of pixel (x, y) after the left-right check (or D^L when the check is off). The check
// always compares the integer D^L with D^R; SUB returns the bits of the sub-pixel D^L it kept.
template <bool SUB, bool WIDE>
__device__ __forceinline__ uint32_t checked_from(const Problem& pb, const Method& mt, int x, int y,
                                                 int dl) {
  constexpr uint32_t inv = SUB ? kInvalidF : kInvalid;
  const int64_t row = (int64_t)y * pb.W;
  if (mt.flags & 1) {
    if (x - dl < 0) return inv;
    // exact check: D^R(x') = D^L of the swapped, flipped pair at W - 1 - x'
    const int dr =
        pb.dp ? (int)pb.dp[row + pb.W - 1 - (x - dl)] : (int)(pb.kr[row + x - dl] & 0xFFu);
    const int diff = dl - dr;
    if ((diff < 0 ? -diff : diff) > mt.lr_threshold) return inv;
  }
  return SUB ? __float_as_uint(refine_subpixel<WIDE>(pb, row + x, dl)) : (uint32_t)dl;
}
template <bool SUB, bool WIDE>
__device__ __forceinline__ uint32_t checked_disp(const Problem& pb, const Method& mt, int x, int y) {
  return checked_from<SUB, WIDE>(pb, mt, x, y, pb.dl[(int64_t)y * pb.W + x]);
}

// Final map of one 64 x 4 tile: LR check (+ median when flags & 2), plus the debug maps D^R and
// the LR mask of the tile's own pixels. SUB writes the float map pb.disp_f (+infinity where
// invalid) from the sub-pixel D^L instead of the uint16 map (WIDE: uint32 aggregated sums).
template <bool SUB, bool WIDE>
__device__ __forceinline__ void lr_median_tile(const Problem& pb, const Method& mt, int item,
                                               MedianSmemT<SUB>& sm) {
  constexpr uint32_t inv = SUB ? kInvalidF : kInvalid;
  const int W = pb.W, H = pb.H;
  const int ntx = (W + kMedTW - 1) / kMedTW;
  const int x0 = (item % ntx) * kMedTW, y0 = (item / ntx) * kMedTH;
  const bool median = (mt.flags & 2) != 0;
  if (median) {
    // the frame and tile (396 values, two per thread of 256): both D^L loads first, then the
    // checks (whose D^R key loads depend on them), so the two load chains overlap
    constexpr int NS = (kMedTH + 2) * (kMedTW + 2);
    static_assert(NS <= 2 * 256, "two staged values per thread");
    int gxs[2], gys[2], dls[2];
    bool ins[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
      const int i = threadIdx.x + 256 * u;
      const int ty = i / (kMedTW + 2), tx = i % (kMedTW + 2);
      gxs[u] = x0 + tx - 1;
      gys[u] = y0 + ty - 1;
      ins[u] = i < NS && gxs[u] >= 0 && gxs[u] < W && gys[u] >= 0 && gys[u] < H;
      dls[u] = ins[u] ? pb.dl[(int64_t)gys[u] * W + gxs[u]] : 0;
    }
#pragma unroll
    for (int u = 0; u < 2; u++) {
      const int i = threadIdx.x + 256 * u;
      if (i < NS)
        sm.t[i / (kMedTW + 2)][i % (kMedTW + 2)] =
            ins[u] ? checked_from<SUB, WIDE>(pb, mt, gxs[u], gys[u], dls[u]) : inv;
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
      if (out != inv) {
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
      pb.mask[p] = sm.t[ly + 1][lx + 1] != inv ? 1 : 0;
    } else {
      out = checked_disp<SUB, WIDE>(pb, mt, x, y);
      pb.mask[p] = out != inv ? 1 : 0;
    }
    pb.dr[p] = pb.dp ? pb.dp[(int64_t)y * W + W - 1 - x] : (uint16_t)(pb.kr[p] & 0xFFu);
    if (SUB)
      *reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(pb.disp_f) +
                                   (int64_t)y * pb.out_pitch + 4 * (int64_t)x) = out;
    else
      *reinterpret_cast<uint16_t*>(reinterpret_cast<uint8_t*>(pb.disp) +
                                   (int64_t)y * pb.out_pitch + 2 * (int64_t)x) = (uint16_t)out;
  }
  if (median) __syncthreads();
}

}  // namespace r2t
