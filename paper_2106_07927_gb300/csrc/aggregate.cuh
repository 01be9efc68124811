// SGM path aggregation, Eq. (sgm_path) and Eq. (sgm_path_aggr) of Sec. 2.1.2.
//
// For one direction r and a pixel p with predecessor q = p - r inside the image,
//   L_r(p,d) = C(p,d) + min(L_r(q,d), L_r(q,d-1) + P1, L_r(q,d+1) + P1, m + P2) - m,
//   m = min_k L_r(q,k),
// and L_r(p,d) = C(p,d) where the path enters the image. With P1 <= P2 the four-term min equals
// the paper's min over d' of L_r(q,d') + V(d,d'); subtracting m keeps L_r <= 255 + P2 so every
// value fits 16 bits. S(p,d) = sum_r L_r(p,d), saturated at 65535.
//
// GB300 mapping (not the paper's): every path line is a sequential chain, so one group of LPL
// lanes walks one line with the D disparities spread over the lanes, DPL per lane, held as
// packed u16x2 registers. Both directions of a line (LR/RL, TB/BT, TLBR/BRTL, TRBL/BLTR) run in
// the same group as two independent chains, which doubles the instruction-level parallelism of
// the latency-bound recurrence. Neighbouring disparities cross lanes by one shuffle each way;
// the group minimum m is one redux.sync. Path costs are added into S with 64-bit atomic adds of
// four packed u16 lanes (no carry can cross a lane while 8 (255 + P2) <= 65535; above that the
// sums are kept as uint32, "wide"). Integer addition is associative, so the result does not
// depend on the order in which the eight directions arrive.
#pragma once
#include "common.cuh"

namespace r2t {

template <int DPL>
struct RawCost;
template <>
struct RawCost<2> {
  typedef uint32_t T;
  static __device__ __forceinline__ T load(const uint8_t* p) {
    return (uint32_t)__ldg(reinterpret_cast<const unsigned short*>(p));
  }
  static __device__ __forceinline__ void unpack(T r, uint32_t (&c)[1]) {
    c[0] = __byte_perm(r, 0u, 0x4140);
  }
};
template <>
struct RawCost<4> {
  typedef uint32_t T;
  static __device__ __forceinline__ T load(const uint8_t* p) {
    return __ldg(reinterpret_cast<const unsigned int*>(p));
  }
  static __device__ __forceinline__ void unpack(T r, uint32_t (&c)[2]) {
    c[0] = __byte_perm(r, 0u, 0x4140);
    c[1] = __byte_perm(r, 0u, 0x4342);
  }
};
template <>
struct RawCost<8> {
  typedef uint2 T;
  static __device__ __forceinline__ T load(const uint8_t* p) {
    return __ldg(reinterpret_cast<const uint2*>(p));
  }
  static __device__ __forceinline__ void unpack(T r, uint32_t (&c)[4]) {
    c[0] = __byte_perm(r.x, 0u, 0x4140);
    c[1] = __byte_perm(r.x, 0u, 0x4342);
    c[2] = __byte_perm(r.y, 0u, 0x4140);
    c[3] = __byte_perm(r.y, 0u, 0x4342);
  }
};

// Number of path lines of a pair: rows (+ columns) (+ 2 (W + H - 1) diagonals).
__host__ __device__ inline int agg_num_lines(int W, int H, int num_paths) {
  return num_paths == 8 ? H + W + 2 * (W + H - 1) : H + W;
}

// Line li (0 .. agg_num_lines - 1) -> entry pixel, unit step and length. The longest axis comes
// first so its chains start earliest. Axes: 0 rows (LR/RL), 1 columns (TB/BT), 2 diagonals
// x - y = const (TLBR/BRTL), 3 anti-diagonals x + y = const (TRBL/BLTR).
struct LineGeom {
  int sx, sy, dx, dy, len;
};
// Axis order of the line index space (the longer of rows / columns first, then the diagonals)
// and the number of axes (2 or 4).
__host__ __device__ inline int axis_order(int W, int H, int num_paths, int (&order)[4]) {
  if (W >= H) {
    order[0] = 0; order[1] = 2; order[2] = 3; order[3] = 1;
  } else {
    order[0] = 1; order[1] = 2; order[2] = 3; order[3] = 0;
  }
  if (num_paths == 4) order[1] = order[3];
  return num_paths == 8 ? 4 : 2;
}

// The axes as contiguous segments [begin, end) of the line index space, with the longest line
// of each; returns the number of segments.
__host__ __device__ inline int agg_segments(int W, int H, int num_paths, int* begin, int* end,
                                            int* maxlen) {
  const int nl[4] = {H, W, W + H - 1, W + H - 1};
  const int mn = W < H ? W : H;
  const int ml[4] = {W, H, mn, mn};
  int order[4];
  const int naxes = axis_order(W, H, num_paths, order);
  int b = 0;
  for (int a = 0; a < naxes; a++) {
    begin[a] = b;
    b += nl[order[a]];
    end[a] = b;
    maxlen[a] = ml[order[a]];
  }
  return naxes;
}

__host__ __device__ inline LineGeom line_geom(int li, int W, int H, int num_paths) {
  int nl[4] = {H, W, W + H - 1, W + H - 1};
  int order[4];
  const int naxes = axis_order(W, H, num_paths, order);
  int axis = -1, i = li;
  for (int a = 0; a < naxes; a++) {
    int n = nl[order[a]];
    if (i < n) {
      axis = order[a];
      break;
    }
    i -= n;
  }
  LineGeom g;
  g.len = 0;
  g.sx = g.sy = g.dx = g.dy = 0;
  if (axis == 0) {
    g.sx = 0; g.sy = i; g.dx = 1; g.dy = 0; g.len = W;
  } else if (axis == 1) {
    g.sx = i; g.sy = 0; g.dx = 0; g.dy = 1; g.len = H;
  } else if (axis == 2) {
    int k = i - (H - 1);
    g.sx = k > 0 ? k : 0;
    g.sy = k < 0 ? -k : 0;
    g.dx = 1; g.dy = 1;
    g.len = (W - g.sx) < (H - g.sy) ? (W - g.sx) : (H - g.sy);
  } else if (axis == 3) {
    int k = i;
    g.sy = k - (W - 1) > 0 ? k - (W - 1) : 0;
    g.sx = k - g.sy;
    g.dx = -1; g.dy = 1;
    g.len = (g.sx + 1) < (H - g.sy) ? (g.sx + 1) : (H - g.sy);
  }
  return g;
}

// One step of one chain: L <- L_r(p, .) from L = L_r(q, .), m = min_k L_r(q, k), c = C(p, .).
template <int DPL, int LPL>
__device__ __forceinline__ void chain_step(uint32_t (&L)[DPL / 2], uint32_t& m,
                                           const uint32_t (&c)[DPL / 2], bool active, int lig,
                                           uint32_t P1P1, uint32_t P2P2) {
  constexpr int NP = DPL / 2;
  uint32_t up = __shfl_up_sync(0xffffffffu, L[NP - 1], 1, LPL);  // hi half: d = first - 1
  uint32_t dn = __shfl_down_sync(0xffffffffu, L[0], 1, LPL);     // lo half: d = last + 1
  if (lig == 0) up = kSent << 16;
  if (lig == LPL - 1) dn = kSent;
  // X[k] = (L(d0 - 1), L(d0)) for pair k starting at d0; X[k + 1] = (L(d0 + 1), L(d0 + 2)).
  uint32_t X[NP + 1];
  X[0] = __byte_perm(up, L[0], 0x5432);
#pragma unroll
  for (int k = 1; k < NP; k++) X[k] = __byte_perm(L[k - 1], L[k], 0x5432);
  X[NP] = __byte_perm(L[NP - 1], dn, 0x5432);
  const uint32_t mm = m * 0x10001u;
  const uint32_t mP2 = mm + P2P2;
  uint32_t lmin = 0xFFFFFFFFu;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    uint32_t t = vmin2(X[k], X[k + 1]) + P1P1;   // min(L(d-1), L(d+1)) + P1, no lane carry
    uint32_t u = vmin2(vmin2(L[k], t), mP2);     // >= m in both halves
    uint32_t ln = u + c[k] - mm;                 // each half in [0, 255 + P2]
    ln = active ? ln : (kSent * 0x10001u);
    L[k] = ln;
    lmin = vmin2(lmin, ln);
  }
  uint32_t lm = min(lmin & 0xFFFFu, lmin >> 16);
  if (LPL == 32) {
    lm = __reduce_min_sync(0xffffffffu, lm);
  } else {
#pragma unroll
    for (int o = LPL / 2; o >= 1; o >>= 1) lm = min(lm, __shfl_xor_sync(0xffffffffu, lm, o, LPL));
  }
  m = lm;
}

template <int DPL, bool WIDE>
__device__ __forceinline__ void add_to_sum(void* aggp, const uint32_t (&L)[DPL / 2]) {
  constexpr int NP = DPL / 2;
  if (!WIDE) {
    if (DPL == 2) {
      atomicAdd(reinterpret_cast<unsigned int*>(aggp), L[0]);
    } else {
#pragma unroll
      for (int k = 0; k < NP; k += 2)
        atomicAdd(reinterpret_cast<unsigned long long*>(aggp) + k / 2,
                  (unsigned long long)L[k] | ((unsigned long long)L[k + 1] << 32));
    }
  } else {
#pragma unroll
    for (int k = 0; k < NP; k++)
      atomicAdd(reinterpret_cast<unsigned long long*>(aggp) + k,
                (unsigned long long)(L[k] & 0xFFFFu) | ((unsigned long long)(L[k] >> 16) << 32));
  }
}

// Aggregates the lines [line0, min(line0 + 32 / LPL, line_end)) of one pair with one warp: lane
// group g walks line line0 + g in both directions and adds both chains into S.
template <int DPL, int LPL, bool WIDE>
__device__ __forceinline__ void agg_warp_lines(const Problem& pb, const Method& mt, int line0,
                                               int line_end) {
  typedef RawCost<DPL> RC;
  typedef typename RC::T Raw;
  constexpr int NP = DPL / 2;
  constexpr int U = 4;  // steps loaded ahead
  const int lane = threadIdx.x & 31;
  const int lig = lane % LPL;
  const int li = line0 + lane / LPL;
  const int W = pb.W, H = pb.H, D = pb.D;
  const int nl = min(agg_num_lines(W, H, mt.num_paths), line_end);
  LineGeom g;
  if (li < nl) {
    g = line_geom(li, W, H, mt.num_paths);
  } else {
    g.sx = g.sy = g.dx = g.dy = 0;
    g.len = 0;
  }
  const int maxlen = __reduce_max_sync(0xffffffffu, (unsigned)g.len);
  if (maxlen == 0) return;
  const bool active = lig * DPL < D;
  const int64_t stride = ((int64_t)g.dy * W + g.dx) * D;  // elements per step
  const int64_t off_f = ((int64_t)g.sy * W + g.sx) * D + lig * DPL;
  const int64_t off_b = off_f + (int64_t)(g.len > 0 ? g.len - 1 : 0) * stride;
  const uint8_t* cf = pb.cost + off_f;
  const uint8_t* cb = pb.cost + off_b;
  const uint32_t P1P1 = (uint32_t)mt.P1 * 0x10001u, P2P2 = (uint32_t)mt.P2 * 0x10001u;

  uint32_t Lf[NP], Lb[NP];
#pragma unroll
  for (int k = 0; k < NP; k++) Lf[k] = Lb[k] = active ? 0u : kSent * 0x10001u;
  uint32_t mf = 0, mb = 0;

  Raw rf[U], rb[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    const bool live = active && u < g.len;
    rf[u] = live ? RC::load(cf + (int64_t)u * stride) : Raw();
    rb[u] = live ? RC::load(cb - (int64_t)u * stride) : Raw();
  }
  for (int t0 = 0; t0 < maxlen; t0 += U) {
    Raw nf[U], nb[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int t = t0 + U + u;
      const bool live = active && t < g.len;
      nf[u] = live ? RC::load(cf + (int64_t)t * stride) : Raw();
      nb[u] = live ? RC::load(cb - (int64_t)t * stride) : Raw();
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int t = t0 + u;
      if (t < maxlen) {
        uint32_t c[NP];
        RC::unpack(rf[u], c);
        chain_step<DPL, LPL>(Lf, mf, c, active, lig, P1P1, P2P2);
        RC::unpack(rb[u], c);
        chain_step<DPL, LPL>(Lb, mb, c, active, lig, P1P1, P2P2);
        if (active && t < g.len) {
          const int64_t ef = off_f + (int64_t)t * stride;
          const int64_t eb = off_b - (int64_t)t * stride;
          if (WIDE) {
            add_to_sum<DPL, true>(reinterpret_cast<uint32_t*>(pb.agg) + ef, Lf);
            add_to_sum<DPL, true>(reinterpret_cast<uint32_t*>(pb.agg) + eb, Lb);
          } else {
            add_to_sum<DPL, false>(reinterpret_cast<uint16_t*>(pb.agg) + ef, Lf);
            add_to_sum<DPL, false>(reinterpret_cast<uint16_t*>(pb.agg) + eb, Lb);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      rf[u] = nf[u];
      rb[u] = nb[u];
    }
  }
}

}  // namespace r2t
