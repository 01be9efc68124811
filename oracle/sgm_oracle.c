/*
 * Plain CPU oracle of the ReS2tAC dense SGM stereo path (Ruf et al., Sensors 2021).
 *
 * TEST INFRASTRUCTURE. This file is the checker of the CUDA library, not part of it: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it. It shares no code,
 * header, table or helper with the CUDA path. It is deliberately slow and literal: one pixel,
 * one disparity, one direction at a time, int32 arithmetic (64- and 128-bit integers for the NCC
 * sums), no floating point on the integer path, no SIMD, no threads, no blocking.
 *
 * What each function computes, with the passage it follows:
 *   r2o_census          census transform, Sec. 2.1.1 and Sec. 2.2.1 (zero-valued margin), the
 *                       centre pixel left out (Sec. 2.3.1).
 *   r2o_cost            Hamming matching cost, Eq. (image_matching) in Sec. 2.1.1; cost 0xFF
 *                       where the matching pixel lies left of the image (Sec. 2.3.2).
 *   r2o_path            one SGM path, Eq. (sgm_path) in Sec. 2.1.2, in the normalised form
 *                       L(p,d) = C(p,d) + min(L(q,d), L(q,d-1)+P1, L(q,d+1)+P1, m+P2) - m,
 *                       q = p - r, m = min_k L(q,k); L = C where the path enters the image.
 *   r2o_aggregate       S(p,d) = sum over paths of L_r(p,d), Eq. (sgm_path_aggr), saturated
 *                       to 65535 (uint16 volume).
 *   r2o_wta             D^L(p) = argmin_d S(p,d), Eq. (wta); the smallest d wins a tie.
 *   r2o_right_disparity D^R(x,y) = argmin_d S((x+d,y),d), Eq. (right_disparity), over the d
 *                       whose pixel x+d lies inside the image; the smallest d wins a tie.
 *   r2o_lr_check        Eq. (LR_check), App. B: keep D^L(p) when x - D^L(p) >= 0 and
 *                       |D^L(p) - D^R(x - D^L(p), y)| <= threshold, else the invalid value.
 *   r2o_median3x3       3x3 median of the valid pixels, Sec. 2.1.3 / Sec. 2.2.4: pixels outside
 *                       the image and invalid pixels count as 0xFFFF; the output is element [4]
 *                       of the 9 sorted values (what five bubble-sort passes leave, App. D).
 *   r2o_cost_right      matching cost with the right image as reference, for the exact
 *                       consistency check (Sec. 3.2.3): C^R(x,y,d) = Hamming distance between
 *                       CT_R(x,y) and CT_L(x+d,y); 255 when x + d > W - 1.
 *   r2o_ncc_cost        the second matching cost, Sec. 2.1.1 and Sec. 2.2.1 ("Inverted and
 *                       truncated version of the normalized cross-correlation"):
 *                       s = 1 - max(0, Phi) with Phi the zero-mean NCC of the n x n patches
 *                       around (x, y) in the reference and (x -/+ d, y) in the matching image
 *                       (zero margin as for the census), scaled to 0..255 as 255 - k with
 *                       k = round(255 max(0, Phi)) decided in exact integer arithmetic.
 *   r2o_s_at            S(p, .) at one pixel from the R path lines through it (each walked from
 *                       the pixel where it enters the image, costs computed on the way): the same
 *                       sums as r2o_aggregate, for sampled checks of images too large for it.
 *   r2o_rectify         rectification (Sec. 2.1.1: the pair is resampled through two maps so
 *                       that epipolar lines lie on image rows): bilinear interpolation of the raw
 *                       image at the map's source coordinate, on a 1/32-pixel grid with integer
 *                       weights (see the function); samples outside the raw image read 0.
 *   r2o_sgm             the whole chain above, in the order of Sec. 2.1. With flag 4 (exact
 *                       check) D^R is the WTA of the right-reference volume aggregated from C^R
 *                       over the same paths, instead of Eq. (right_disparity). The paper gets it
 *                       by swapping and mirroring the pair and matching again; since mirroring
 *                       maps the path set onto itself and permutes both descriptors' bits alike,
 *                       that is the same map (a pin checks the two against each other).
 *   r2o_subpixel        sub-pixel refinement, Sec. 2.1.3 ("Subpixel disparity refinement"): the
 *                       parabola through the aggregated costs at D^L(p) - 1, D^L(p), D^L(p) + 1,
 *                       fitted by solving its 3 x 3 system in fp64; D^L(p) moves to the abscissa
 *                       of its minimum. D^L = 0 and D^L = D - 1 have one neighbour and stay.
 *   r2o_median3x3_f64   the 3x3 median above on a double map (+infinity = invalid).
 *   r2o_sgm_subpixel    the chain with the refinement ("fine" in Tab. throughput): the check
 *                       compares the integer D^L with D^R, keeps the refined value, and the
 *                       median runs on the refined values.
 *
 * Conventions where the paper is silent (each is a reading of the paper, not a statement of it):
 *   - census bit = [neighbour < centre], row-major over the window (rows outer), LSB first;
 *   - disparities d = 0 .. D-1;
 *   - all volumes are [y][x][d] with the disparities of one pixel contiguous (Sec. 2.2.1).
 *
 * Return value of every function: 0 on success, -1 on an invalid argument.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define R2O_INVALID 0xFFFF
#define R2O_COST_OUTSIDE 255

/* Path directions r = (dx, dy), in the order LR, RL, TB, BT, TLBR, TRBL, BLTR, BRTL
 * (Fig. neon_impl_paths, Sec. 2.3.3). Four-path SGM uses the first four (Sec. 3.2). */
static const int R2O_DIRS[8][2] = {
    {+1, 0}, {-1, 0}, {0, +1}, {0, -1}, {+1, +1}, {-1, +1}, {+1, -1}, {-1, -1}};

static int popcount64(uint64_t v) {
  int n = 0;
  while (v) {
    v &= v - 1;
    n++;
  }
  return n;
}

/* Census transform. Bit k of the descriptor of pixel (x,y) is 1 when the k-th neighbour of the
 * w x h window (visited row by row, left to right, centre skipped) is darker than the centre.
 * Neighbours outside the image read 0 (zero-valued margin of Sec. 2.2.1). */
int r2o_census(const uint8_t* img, int64_t pitch, int W, int H, int cw, int ch, uint64_t* out) {
  if (!img || !out || W < 1 || H < 1 || cw < 1 || ch < 1) return -1;
  if ((cw % 2) == 0 || (ch % 2) == 0 || cw * ch - 1 > 64 || pitch < W) return -1;
  int rx = cw / 2, ry = ch / 2;
  for (int y = 0; y < H; y++) {
    for (int x = 0; x < W; x++) {
      int centre = img[(int64_t)y * pitch + x];
      uint64_t bits = 0;
      int k = 0;
      for (int j = -ry; j <= ry; j++) {
        for (int i = -rx; i <= rx; i++) {
          if (i == 0 && j == 0) continue;
          int xx = x + i, yy = y + j;
          int v = 0;
          if (xx >= 0 && xx < W && yy >= 0 && yy < H) v = img[(int64_t)yy * pitch + xx];
          if (v < centre) bits |= (uint64_t)1 << k;
          k++;
        }
      }
      out[(int64_t)y * W + x] = bits;
    }
  }
  return 0;
}

/* Matching cost S(p,d) = Hamming distance between CT_L(x,y) and CT_R(x-d,y) (Eq. image_matching);
 * 255 when x - d < 0. */
int r2o_cost(const uint64_t* ctl, const uint64_t* ctr, int W, int H, int D, uint8_t* cost) {
  if (!ctl || !ctr || !cost || W < 1 || H < 1 || D < 1 || D > 256) return -1;
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++)
      for (int d = 0; d < D; d++) {
        int64_t i = ((int64_t)y * W + x) * D + d;
        if (x - d < 0)
          cost[i] = R2O_COST_OUTSIDE;
        else
          cost[i] = (uint8_t)popcount64(ctl[(int64_t)y * W + x] ^ ctr[(int64_t)y * W + (x - d)]);
      }
  return 0;
}

/* One SGM path L_r over the whole image for the direction r = (dx, dy) (Eq. sgm_path).
 * Pixels are visited so that p - r is always visited before p; a pixel whose predecessor
 * p - r lies outside the image starts its line: L(p,.) = C(p,.). L values never exceed
 * 255 + P2, so uint16 holds them exactly. */
int r2o_path(const uint8_t* cost, int W, int H, int D, int dx, int dy, int P1, int P2,
             uint16_t* L) {
  if (!cost || !L || W < 1 || H < 1 || D < 1 || D > 256) return -1;
  if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || (dx == 0 && dy == 0)) return -1;
  if (P1 < 0 || P2 < P1 || P2 > 16384) return -1;
  for (int yi = 0; yi < H; yi++) {
    int y = (dy >= 0) ? yi : H - 1 - yi;
    for (int xi = 0; xi < W; xi++) {
      int x = (dx >= 0) ? xi : W - 1 - xi;
      int64_t p = ((int64_t)y * W + x) * D;
      int qx = x - dx, qy = y - dy;
      if (qx < 0 || qx >= W || qy < 0 || qy >= H) {
        for (int d = 0; d < D; d++) L[p + d] = cost[p + d];
        continue;
      }
      int64_t q = ((int64_t)qy * W + qx) * D;
      int m = L[q];
      for (int k = 1; k < D; k++)
        if (L[q + k] < m) m = L[q + k];
      for (int d = 0; d < D; d++) {
        int best = L[q + d];
        if (d > 0 && L[q + d - 1] + P1 < best) best = L[q + d - 1] + P1;
        if (d < D - 1 && L[q + d + 1] + P1 < best) best = L[q + d + 1] + P1;
        if (m + P2 < best) best = m + P2;
        L[p + d] = (uint16_t)(cost[p + d] + best - m);
      }
    }
  }
  return 0;
}

/* Matching cost with the right image as reference (exact consistency check, Sec. 3.2.3):
 * C^R(x,y,d) = Hamming distance between CT_R(x,y) and CT_L(x+d,y); 255 when x + d > W - 1. */
int r2o_cost_right(const uint64_t* ctl, const uint64_t* ctr, int W, int H, int D, uint8_t* cost) {
  if (!ctl || !ctr || !cost || W < 1 || H < 1 || D < 1) return -1;
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++)
      for (int d = 0; d < D; d++) {
        int64_t p = ((int64_t)y * W + x) * D + d;
        if (x + d > W - 1)
          cost[p] = 255;
        else
          cost[p] = (uint8_t)popcount64(ctr[(int64_t)y * W + x] ^ ctl[(int64_t)y * W + x + d]);
      }
  return 0;
}

/* Pixel of an image with the zero-valued margin. */
static int px_or_zero(const uint8_t* img, int64_t pitch, int W, int H, int x, int y) {
  if (x < 0 || x >= W || y < 0 || y >= H) return 0;
  return img[(int64_t)y * pitch + x];
}

/* The integer k = round(255 max(0, Phi)), rounded half to even, for Phi = cov / sqrt(vA vB)
 * (Sec. 2.1.1: the cost is the truncated 1 - max(0, Phi); the 8-bit scale 255 is this library's
 * reading). Decided on integers alone, so no floating-point rounding order enters it:
 *   k = 0 when cov <= 0 or a patch is constant (vA = 0 or vB = 0);
 *   otherwise x = 255 Phi lies in (0, 255] (Cauchy-Schwarz) and, for m >= 1,
 *     x >= m - 1/2  <=>  (510 cov)^2 >= (2m - 1)^2 vA vB      (both sides are squares of
 *                                                               non-negative numbers),
 *   so M = floor(x + 1/2) is the largest m in 0..255 for which that holds (m = 0 always does);
 *   x + 1/2 = M exactly (a tie) when the two sides are equal, and a tie rounds to the even one of
 *   M - 1 and M. Products reach 2^72 for 9 x 9 patches: 128-bit integers. */
static int ncc_round_255phi(int64_t cov, int64_t vA, int64_t vB) {
  if (cov <= 0 || vA <= 0 || vB <= 0) return 0;
  const __int128 t = (__int128)(510 * cov) * (__int128)(510 * cov);
  const __int128 v = (__int128)vA * (__int128)vB;
  int lo = 0, hi = 255; /* the largest m with (2m - 1)^2 v <= t lies in [lo, hi] */
  while (lo < hi) {
    int m = (lo + hi + 1) / 2;
    __int128 r = (__int128)(2 * m - 1) * (2 * m - 1) * v;
    if (r <= t)
      lo = m;
    else
      hi = m - 1;
  }
  if (lo >= 1 && (__int128)(2 * lo - 1) * (2 * lo - 1) * v == t && (lo & 1)) lo -= 1;
  return lo;
}

/* Exported for the pins: k of ncc_round_255phi for given (cov, vA, vB). */
int r2o_ncc_round(int64_t cov, int64_t vA, int64_t vB) { return ncc_round_255phi(cov, vA, vB); }

/* Inverted, truncated NCC cost of one patch pair: reference patch centred at (xa, y) of A,
 * matching patch centred at (xb, y) of B, n x n, N = n^2 pixels, zero margin.
 *   sA = sum a, sB = sum b, sAA = sum a^2, sBB = sum b^2, sAB = sum a b   (exact integers)
 *   vA = N sAA - sA^2,  vB = N sBB - sB^2,  cov = N sAB - sA sB           (N^2 (co)variances)
 *   Phi = cov / sqrt(vA vB), taken as 0 when vA or vB is 0 (a constant patch);
 *   cost = 255 - k, k = round(255 max(0, Phi)) (ties to even) from ncc_round_255phi: the
 *   truncated 1 - max(0, Phi) on 0..255, with no floating point anywhere. */
static uint8_t ncc_pair_cost(const uint8_t* A, const uint8_t* B, int64_t pitch, int W, int H,
                             int xa, int xb, int y, int n) {
  int r = n / 2, N = n * n;
  int64_t sA = 0, sB = 0, sAA = 0, sBB = 0, sAB = 0;
  for (int j = -r; j <= r; j++)
    for (int i = -r; i <= r; i++) {
      int a = px_or_zero(A, pitch, W, H, xa + i, y + j);
      int b = px_or_zero(B, pitch, W, H, xb + i, y + j);
      sA += a;
      sB += b;
      sAA += a * a;
      sBB += b * b;
      sAB += a * b;
    }
  int64_t vA = N * sAA - sA * sA, vB = N * sBB - sB * sB, cov = N * sAB - sA * sB;
  return (uint8_t)(255 - ncc_round_255phi(cov, vA, vB));
}

/* NCC cost volume with the left image as reference: C(x,y,d) = ncc_pair_cost(left patch at x,
 * right patch at x - d); 255 when x - d < 0. n = 5 or 9. */
int r2o_ncc_cost(const uint8_t* left, const uint8_t* right, int64_t pitch, int W, int H, int D,
                 int n, uint8_t* cost) {
  if (!left || !right || !cost || W < 1 || H < 1 || D < 1 || n < 1 || !(n & 1)) return -1;
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++)
      for (int d = 0; d < D; d++)
        cost[((int64_t)y * W + x) * D + d] =
            x - d < 0 ? 255 : ncc_pair_cost(left, right, pitch, W, H, x, x - d, y, n);
  return 0;
}

/* NCC cost volume with the right image as reference (exact consistency check):
 * C^R(x,y,d) = ncc_pair_cost(right patch at x, left patch at x + d); 255 when x + d > W - 1. */
int r2o_ncc_cost_right(const uint8_t* left, const uint8_t* right, int64_t pitch, int W, int H,
                       int D, int n, uint8_t* cost) {
  if (!left || !right || !cost || W < 1 || H < 1 || D < 1 || n < 1 || !(n & 1)) return -1;
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++)
      for (int d = 0; d < D; d++)
        cost[((int64_t)y * W + x) * D + d] =
            x + d > W - 1 ? 255 : ncc_pair_cost(right, left, pitch, W, H, x, x + d, y, n);
  return 0;
}

/* Aggregated volume S(p,d) = min(65535, sum_r L_r(p,d)) over the first R directions (R = 4 or 8). */
int r2o_aggregate(const uint8_t* cost, int W, int H, int D, int R, int P1, int P2, uint16_t* S) {
  if (!cost || !S || (R != 4 && R != 8) || W < 1 || H < 1 || D < 1 || D > 256) return -1;
  int64_t n = (int64_t)W * H * D;
  uint32_t* sum = (uint32_t*)calloc((size_t)n, sizeof(uint32_t));
  uint16_t* L = (uint16_t*)malloc((size_t)n * sizeof(uint16_t));
  if (!sum || !L) {
    free(sum);
    free(L);
    return -1;
  }
  int rc = 0;
  for (int r = 0; r < R && rc == 0; r++) {
    rc = r2o_path(cost, W, H, D, R2O_DIRS[r][0], R2O_DIRS[r][1], P1, P2, L);
    for (int64_t i = 0; i < n && rc == 0; i++) sum[i] += L[i];
  }
  for (int64_t i = 0; i < n && rc == 0; i++) S[i] = (uint16_t)(sum[i] > 65535 ? 65535 : sum[i]);
  free(sum);
  free(L);
  return rc;
}

/* Winner-takes-all, Eq. (wta): the smallest d with the least S(p,d). */
int r2o_wta(const uint16_t* S, int W, int H, int D, uint16_t* DL) {
  if (!S || !DL || W < 1 || H < 1 || D < 1) return -1;
  for (int64_t p = 0; p < (int64_t)W * H; p++) {
    int best = S[p * D], bd = 0;
    for (int d = 1; d < D; d++)
      if (S[p * D + d] < best) {
        best = S[p * D + d];
        bd = d;
      }
    DL[p] = (uint16_t)bd;
  }
  return 0;
}

/* Approximate right disparity, Eq. (right_disparity): D^R(x,y) is the smallest d in
 * [0, min(D-1, W-1-x)] with the least S((x+d,y),d). */
int r2o_right_disparity(const uint16_t* S, int W, int H, int D, uint16_t* DR) {
  if (!S || !DR || W < 1 || H < 1 || D < 1) return -1;
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      int best = -1, bd = 0;
      for (int d = 0; d < D && x + d < W; d++) {
        int v = S[((int64_t)y * W + x + d) * D + d];
        if (best < 0 || v < best) {
          best = v;
          bd = d;
        }
      }
      DR[(int64_t)y * W + x] = (uint16_t)bd;
    }
  return 0;
}

/* Left-right consistency check, Eq. (LR_check). mask = 1 where the disparity is kept. */
int r2o_lr_check(const uint16_t* DL, const uint16_t* DR, int W, int H, int threshold,
                 uint16_t* Dout, uint8_t* mask) {
  if (!DL || !DR || !Dout || W < 1 || H < 1 || threshold < 0) return -1;
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      int64_t p = (int64_t)y * W + x;
      int dl = DL[p];
      int keep = 0;
      if (x - dl >= 0) {
        int dr = DR[(int64_t)y * W + (x - dl)];
        int diff = dl - dr;
        if (diff < 0) diff = -diff;
        keep = diff <= threshold;
      }
      Dout[p] = keep ? (uint16_t)dl : (uint16_t)R2O_INVALID;
      if (mask) mask[p] = (uint8_t)keep;
    }
  return 0;
}

/* 3x3 median: for each valid pixel, element [4] of its sorted 3x3 neighbourhood, where pixels
 * outside the image and invalid pixels read 0xFFFF; invalid pixels stay invalid. */
int r2o_median3x3(const uint16_t* Din, int W, int H, uint16_t* Dout) {
  if (!Din || !Dout || W < 1 || H < 1 || Din == Dout) return -1;
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      int64_t p = (int64_t)y * W + x;
      if (Din[p] == R2O_INVALID) {
        Dout[p] = R2O_INVALID;
        continue;
      }
      int v[9], n = 0;
      for (int j = -1; j <= 1; j++)
        for (int i = -1; i <= 1; i++) {
          int xx = x + i, yy = y + j;
          v[n++] = (xx >= 0 && xx < W && yy >= 0 && yy < H) ? Din[(int64_t)yy * W + xx]
                                                            : R2O_INVALID;
        }
      for (int a = 1; a < 9; a++) { /* insertion sort */
        int t = v[a], b = a - 1;
        while (b >= 0 && v[b] > t) {
          v[b + 1] = v[b];
          b--;
        }
        v[b + 1] = t;
      }
      Dout[p] = (uint16_t)v[4];
    }
  return 0;
}

/* Matching cost volume of the method selected by flags: bit 3 = NCC over cw x ch (= n x n),
 * else census over cw x ch and its Hamming distance. right_ref: the right image is the reference
 * (exact consistency check). */
static int method_cost(const uint8_t* left, const uint8_t* right, int64_t pitch, int W, int H,
                       int D, int cw, int ch, int flags, int right_ref, uint8_t* cost) {
  if (flags & 8)
    return right_ref ? r2o_ncc_cost_right(left, right, pitch, W, H, D, cw, cost)
                     : r2o_ncc_cost(left, right, pitch, W, H, D, cw, cost);
  int64_t npx = (int64_t)W * H;
  uint64_t* ctl = (uint64_t*)malloc((size_t)npx * 8);
  uint64_t* ctr = (uint64_t*)malloc((size_t)npx * 8);
  int rc = -1;
  if (ctl && ctr) {
    rc = r2o_census(left, pitch, W, H, cw, ch, ctl);
    if (!rc) rc = r2o_census(right, pitch, W, H, cw, ch, ctr);
    if (!rc)
      rc = right_ref ? r2o_cost_right(ctl, ctr, W, H, D, cost) : r2o_cost(ctl, ctr, W, H, D, cost);
  }
  free(ctl);
  free(ctr);
  return rc;
}

/* Exact right disparity map (Sec. 3.2.3): WTA of the volume aggregated from C^R. */
static int r2o_exact_right(const uint8_t* left, const uint8_t* right, int64_t pitch, int W,
                           int H, int D, int cw, int ch, int P1, int P2, int R, int flags,
                           uint16_t* DR) {
  int64_t nde = (int64_t)W * H * D;
  uint8_t* cost = (uint8_t*)malloc((size_t)nde);
  uint16_t* S = (uint16_t*)malloc((size_t)nde * 2);
  int rc = -1;
  if (cost && S) {
    rc = method_cost(left, right, pitch, W, H, D, cw, ch, flags, 1, cost);
    if (!rc) rc = r2o_aggregate(cost, W, H, D, R, P1, P2, S);
    if (!rc) rc = r2o_wta(S, W, H, D, DR);
  }
  free(cost);
  free(S);
  return rc;
}

/* Whole pipeline (Sec. 2.1). flags: bit 0 = left-right check, bit 1 = median, bit 2 = exact D^R
 * (Sec. 3.2.3), bit 3 = NCC cost over a cw x ch (n x n) patch instead of the census.
 * The optional outputs (may be NULL): cost [H][W][D] uint8, S [H][W][D] uint16, D^L, D^R,
 * the left-right mask. disp receives the final map. */
int r2o_sgm(const uint8_t* left, const uint8_t* right, int64_t pitch, int W, int H, int D,
            int cw, int ch, int P1, int P2, int R, int flags, int lr_threshold, uint16_t* disp,
            uint8_t* cost_out, uint16_t* S_out, uint16_t* DL_out, uint16_t* DR_out,
            uint8_t* mask_out) {
  if (!left || !right || !disp || W < 1 || H < 1 || D < 1 || D > 256) return -1;
  int64_t npx = (int64_t)W * H, nde = npx * D;
  uint8_t* cost = (uint8_t*)malloc((size_t)nde);
  uint16_t* S = (uint16_t*)malloc((size_t)nde * 2);
  uint16_t* DL = (uint16_t*)malloc((size_t)npx * 2);
  uint16_t* DR = (uint16_t*)malloc((size_t)npx * 2);
  uint16_t* Dlr = (uint16_t*)malloc((size_t)npx * 2);
  uint8_t* mask = (uint8_t*)malloc((size_t)npx);
  int rc = -1;
  if (cost && S && DL && DR && Dlr && mask) {
    rc = method_cost(left, right, pitch, W, H, D, cw, ch, flags, 0, cost);
    if (!rc) rc = r2o_aggregate(cost, W, H, D, R, P1, P2, S);
    if (!rc) rc = r2o_wta(S, W, H, D, DL);
    if (!rc) rc = (flags & 4) ? r2o_exact_right(left, right, pitch, W, H, D, cw, ch, P1, P2, R,
                                                flags, DR)
                              : r2o_right_disparity(S, W, H, D, DR);
    if (!rc) {
      if (flags & 1) {
        rc = r2o_lr_check(DL, DR, W, H, lr_threshold, Dlr, mask);
      } else {
        memcpy(Dlr, DL, (size_t)npx * 2);
        memset(mask, 1, (size_t)npx);
      }
    }
    if (!rc) {
      if (flags & 2)
        rc = r2o_median3x3(Dlr, W, H, disp);
      else
        memcpy(disp, Dlr, (size_t)npx * 2);
    }
    if (!rc && cost_out) memcpy(cost_out, cost, (size_t)nde);
    if (!rc && S_out) memcpy(S_out, S, (size_t)nde * 2);
    if (!rc && DL_out) memcpy(DL_out, DL, (size_t)npx * 2);
    if (!rc && DR_out) memcpy(DR_out, DR, (size_t)npx * 2);
    if (!rc && mask_out) memcpy(mask_out, mask, (size_t)npx);
  }
  free(cost);
  free(S);
  free(DL);
  free(DR);
  free(Dlr);
  free(mask);
  return rc;
}

/* Solves the 3 x 3 system M c = v in place by Gaussian elimination with partial pivoting;
 * returns -1 if M is singular. */
static int solve3(double M[3][3], double v[3], double c[3]) {
  for (int k = 0; k < 3; k++) {
    int piv = k;
    for (int i = k + 1; i < 3; i++)
      if (fabs(M[i][k]) > fabs(M[piv][k])) piv = i;
    if (M[piv][k] == 0.0) return -1;
    if (piv != k) {
      for (int j = 0; j < 3; j++) {
        double t = M[k][j];
        M[k][j] = M[piv][j];
        M[piv][j] = t;
      }
      double t = v[k];
      v[k] = v[piv];
      v[piv] = t;
    }
    for (int i = k + 1; i < 3; i++) {
      double f = M[i][k] / M[k][k];
      for (int j = k; j < 3; j++) M[i][j] -= f * M[k][j];
      v[i] -= f * v[k];
    }
  }
  for (int i = 2; i >= 0; i--) {
    double t = v[i];
    for (int j = i + 1; j < 3; j++) t -= M[i][j] * c[j];
    c[i] = t / M[i][i];
  }
  return 0;
}

/* Sub-pixel refinement of D^L (Sec. 2.1.3). For each pixel with 1 <= d = D^L(p) <= D - 2, the
 * parabola s(t) = c0 t^2 + c1 t + c2 through (-1, S(p, d-1)), (0, S(p, d)), (1, S(p, d+1)), t
 * measured from d, is solved for, and the abscissa of its minimum, -c1 / (2 c0), is added to d.
 * A parabola that does not open upwards has no minimum; the WTA winner makes that impossible
 * (S(d-1) > S(d) <= S(d+1)), and such a pixel is reported as an error. Other pixels keep d. */
int r2o_subpixel(const uint16_t* S, const uint16_t* DL, int W, int H, int D, double* out) {
  if (!S || !DL || !out || W < 1 || H < 1 || D < 1) return -1;
  for (int64_t p = 0; p < (int64_t)W * H; p++) {
    int d = DL[p];
    if (d >= D) return -1;
    out[p] = (double)d;
    if (d < 1 || d > D - 2) continue;
    double M[3][3], v[3], c[3];
    for (int k = 0; k < 3; k++) {
      double t = (double)(k - 1);
      M[k][0] = t * t;
      M[k][1] = t;
      M[k][2] = 1.0;
      v[k] = (double)S[p * D + d - 1 + k];
    }
    if (solve3(M, v, c) != 0 || !(c[0] > 0.0)) return -1;
    out[p] = (double)d + -c[1] / (2.0 * c[0]);
  }
  return 0;
}

/* 3x3 median of a double map: for each valid (finite) pixel, element [4] of its sorted 3x3
 * neighbourhood, where pixels outside the image and invalid pixels read +infinity; invalid
 * pixels stay +infinity. */
int r2o_median3x3_f64(const double* Din, int W, int H, double* Dout) {
  if (!Din || !Dout || W < 1 || H < 1 || Din == Dout) return -1;
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      int64_t p = (int64_t)y * W + x;
      if (isinf(Din[p])) {
        Dout[p] = INFINITY;
        continue;
      }
      double v[9];
      int n = 0;
      for (int j = -1; j <= 1; j++)
        for (int i = -1; i <= 1; i++) {
          int xx = x + i, yy = y + j;
          v[n++] = (xx >= 0 && xx < W && yy >= 0 && yy < H) ? Din[(int64_t)yy * W + xx]
                                                            : INFINITY;
        }
      for (int a = 1; a < 9; a++) { /* insertion sort */
        double t = v[a];
        int b = a - 1;
        while (b >= 0 && v[b] > t) {
          v[b + 1] = v[b];
          b--;
        }
        v[b + 1] = t;
      }
      Dout[p] = v[4];
    }
  return 0;
}

/* Whole pipeline with the sub-pixel refinement (flags as r2o_sgm). disp receives the final
 * double map (+infinity where invalid); refined (may be NULL) the refined D^L before the check. */
int r2o_sgm_subpixel(const uint8_t* left, const uint8_t* right, int64_t pitch, int W, int H,
                     int D, int cw, int ch, int P1, int P2, int R, int flags, int lr_threshold,
                     double* disp, double* refined) {
  if (!left || !right || !disp || W < 1 || H < 1 || D < 1 || D > 256) return -1;
  int64_t npx = (int64_t)W * H, nde = npx * D;
  uint8_t* cost = (uint8_t*)malloc((size_t)nde);
  uint16_t* S = (uint16_t*)malloc((size_t)nde * 2);
  uint16_t* DL = (uint16_t*)malloc((size_t)npx * 2);
  uint16_t* DR = (uint16_t*)malloc((size_t)npx * 2);
  uint16_t* Dlr = (uint16_t*)malloc((size_t)npx * 2);
  uint8_t* mask = (uint8_t*)malloc((size_t)npx);
  double* ref = (double*)malloc((size_t)npx * 8);
  double* chk = (double*)malloc((size_t)npx * 8);
  int rc = -1;
  if (cost && S && DL && DR && Dlr && mask && ref && chk) {
    rc = method_cost(left, right, pitch, W, H, D, cw, ch, flags, 0, cost);
    if (!rc) rc = r2o_aggregate(cost, W, H, D, R, P1, P2, S);
    if (!rc) rc = r2o_wta(S, W, H, D, DL);
    if (!rc) rc = (flags & 4) ? r2o_exact_right(left, right, pitch, W, H, D, cw, ch, P1, P2, R,
                                                flags, DR)
                              : r2o_right_disparity(S, W, H, D, DR);
    if (!rc) rc = r2o_subpixel(S, DL, W, H, D, ref);
    if (!rc) {
      if (flags & 1) {
        rc = r2o_lr_check(DL, DR, W, H, lr_threshold, Dlr, mask);
      } else {
        memset(mask, 1, (size_t)npx);
      }
    }
    if (!rc) {
      for (int64_t p = 0; p < npx; p++) chk[p] = mask[p] ? ref[p] : INFINITY;
      if (flags & 2)
        rc = r2o_median3x3_f64(chk, W, H, disp);
      else
        memcpy(disp, chk, (size_t)npx * 8);
    }
    if (!rc && refined) memcpy(refined, ref, (size_t)npx * 8);
  }
  free(cost);
  free(S);
  free(DL);
  free(DR);
  free(Dlr);
  free(mask);
  free(ref);
  free(chk);
  return rc;
}

/* Rectification of one image through its map (Sec. 2.1.1). For every output pixel (x, y) the
 * map gives the source coordinate (mx, my) in the raw image (float32, mapx / mapy rows of
 * map_pitch bytes). The coordinate is put on a 1/32-pixel grid, X = rint(32 mx), Y = rint(32 my)
 * (the product by 32 is exact in float; rint rounds ties to even); a coordinate that is not
 * finite or has |32 m| >= 2^24 yields 0. With x0 = floor(X / 32), fx = X - 32 x0 (y likewise) the
 * output is the bilinear interpolation with integer weights summing to 1024, rounded:
 *   (I(x0,y0)(32-fx)(32-fy) + I(x0+1,y0) fx (32-fy) + I(x0,y0+1)(32-fx) fy
 *    + I(x0+1,y0+1) fx fy + 512) >> 10,
 * where samples outside the raw image (rw x rh) read 0. */
int r2o_rectify(const uint8_t* raw, int64_t raw_pitch, int rw, int rh, const float* mapx,
                const float* mapy, int64_t map_pitch, int W, int H, uint8_t* out,
                int64_t out_pitch) {
  if (!raw || !mapx || !mapy || !out || rw < 1 || rh < 1 || W < 1 || H < 1) return -1;
  for (int y = 0; y < H; y++)
    for (int x = 0; x < W; x++) {
      const float* mxr = (const float*)((const uint8_t*)mapx + (int64_t)y * map_pitch);
      const float* myr = (const float*)((const uint8_t*)mapy + (int64_t)y * map_pitch);
      float sx = mxr[x] * 32.0f, sy = myr[x] * 32.0f;
      int v = 0;
      if (isfinite(sx) && isfinite(sy) && fabsf(sx) < 16777216.0f && fabsf(sy) < 16777216.0f) {
        int X = (int)rintf(sx), Y = (int)rintf(sy);
        int x0 = (int)floor(X / 32.0), y0 = (int)floor(Y / 32.0);
        int fx = X - 32 * x0, fy = Y - 32 * y0;
        int p00 = px_or_zero(raw, raw_pitch, rw, rh, x0, y0);
        int p10 = px_or_zero(raw, raw_pitch, rw, rh, x0 + 1, y0);
        int p01 = px_or_zero(raw, raw_pitch, rw, rh, x0, y0 + 1);
        int p11 = px_or_zero(raw, raw_pitch, rw, rh, x0 + 1, y0 + 1);
        v = (p00 * (32 - fx) * (32 - fy) + p10 * fx * (32 - fy) + p01 * (32 - fx) * fy +
             p11 * fx * fy + 512) >> 10;
      }
      out[(int64_t)y * out_pitch + x] = (uint8_t)v;
    }
  return 0;
}

/* Census descriptor of one pixel (the definition of r2o_census). */
static uint64_t census_px(const uint8_t* img, int64_t pitch, int W, int H, int cw, int ch, int x,
                          int y) {
  int rx = cw / 2, ry = ch / 2, centre = img[(int64_t)y * pitch + x], k = 0;
  uint64_t bits = 0;
  for (int j = -ry; j <= ry; j++)
    for (int i = -rx; i <= rx; i++) {
      if (i == 0 && j == 0) continue;
      if (px_or_zero(img, pitch, W, H, x + i, y + j) < centre) bits |= (uint64_t)1 << k;
      k++;
    }
  return bits;
}

/* Aggregated sums at the single pixel (x, y): for each of the first R directions r, the line of
 * pixels p_0, p_1, .., p_k = (x, y) with p_{i+1} = p_i + r and p_0 where the line enters the image;
 * L(p_0, .) = C(p_0, .), then the recurrence of r2o_path along the line. out[d] = min(65535,
 * sum_r L_r(x, y, d)). flags bit 3 selects the NCC cost over a cw x cw patch, as in r2o_sgm. */
int r2o_s_at(const uint8_t* left, const uint8_t* right, int64_t pitch, int W, int H, int D,
             int cw, int ch, int P1, int P2, int R, int flags, int x, int y, uint16_t* out) {
  if (!left || !right || !out || x < 0 || x >= W || y < 0 || y >= H || D < 1 || D > 256) return -1;
  if ((R != 4 && R != 8) || P1 < 0 || P2 < P1 || P2 > 16384) return -1;
  static const int dirs[8][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1},
                                 {1, 1}, {-1, 1}, {1, -1}, {-1, -1}};
  int32_t sum[256] = {0};
  int Lq[256], Lp[256], C[256];
  for (int r = 0; r < R; r++) {
    int dx = dirs[r][0], dy = dirs[r][1];
    int k = 0;  /* steps back to the entry pixel */
    while (x - (k + 1) * dx >= 0 && x - (k + 1) * dx < W && y - (k + 1) * dy >= 0 &&
           y - (k + 1) * dy < H)
      k++;
    for (int i = 0; i <= k; i++) {
      int px = x - (k - i) * dx, py = y - (k - i) * dy;
      if (flags & 8) {
        for (int d = 0; d < D; d++)
          C[d] = px - d < 0 ? 255 : ncc_pair_cost(left, right, pitch, W, H, px, px - d, py, cw);
      } else {
        uint64_t cl = census_px(left, pitch, W, H, cw, ch, px, py);
        for (int d = 0; d < D; d++)
          C[d] = px - d < 0 ? 255
                            : popcount64(cl ^ census_px(right, pitch, W, H, cw, ch, px - d, py));
      }
      if (i == 0) {
        for (int d = 0; d < D; d++) Lp[d] = C[d];
      } else {
        int m = Lq[0];
        for (int d = 1; d < D; d++)
          if (Lq[d] < m) m = Lq[d];
        for (int d = 0; d < D; d++) {
          int best = Lq[d];
          if (d > 0 && Lq[d - 1] + P1 < best) best = Lq[d - 1] + P1;
          if (d < D - 1 && Lq[d + 1] + P1 < best) best = Lq[d + 1] + P1;
          if (m + P2 < best) best = m + P2;
          Lp[d] = C[d] + best - m;
        }
      }
      memcpy(Lq, Lp, sizeof(int) * D);
    }
    for (int d = 0; d < D; d++) sum[d] += Lq[d];
  }
  for (int d = 0; d < D; d++) out[d] = (uint16_t)(sum[d] > 65535 ? 65535 : sum[d]);
  return 0;
}
