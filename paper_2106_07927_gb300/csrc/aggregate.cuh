// SGM path aggregation, Eq. (sgm_path) and Eq. (sgm_path_aggr) of Sec. 2.1.2.
//
// For one direction r and a pixel p with predecessor q = p - r inside the image,
//   L_r(p,d) = C(p,d) + min(L_r(q,d), L_r(q,d-1) + P1, L_r(q,d+1) + P1, m(q) + P2) - m(q),
//   m(q) = min_k L_r(q,k),
// and L_r(p,d) = C(p,d) where the path enters the image. With P1 <= P2 the four-term min equals
// the paper's min over d' of L_r(q,d') + V(d,d'); subtracting m keeps L_r <= 255 + P2 so every
// value fits 16 bits. S(p,d) = sum_r L_r(p,d), saturated at 65535.
//
// GB300 mapping (not the paper's). Every path line is a sequential chain; a group of lanes walks
// one chain with the D disparities spread over its lanes, held as packed u16x2 registers.
// Neighbouring disparities cross lanes by one shuffle each way. S is accumulated with atomic adds
// of packed u16 sums (64-bit red.add in the row kernel, TMA bulk add-reductions of 32-bit words in
// the sheared kernel): no carry can cross a half while num_paths (255 + P2) <= 65535; above that
// the sums are uint32 ("wide"). Integer addition is associative, so the order in which directions
// arrive does not change S. Two kernels split the paths:
//  - rows (LR, RL), the longest chains when W >= H. A group of 8..32 lanes walks a row with 2..8
//    disparities per lane, either both directions interleaved (two chains for ILP) or one
//    direction per group, and forms m with a pipelined reduction: writing
//    g(q,d) = min(L(q,d), L(q,d-1) + P1, L(q,d+1) + P1) and h(p,d) = C(p,d) + g(q,d),
//      L(p,d) = min(h(p,d) - m(q), C(p,d) + P2),
//      m(p)   = min(min_d h(p,d) - m(q), min_d C(p,d) + P2),
//    so the group minima of h and of C (redux.sync) do not wait for m(q) and overlap the next
//    step. Costs are fetched several steps ahead into a register ring.
//  - sheared columns (TB, BT and, with 8 paths, the four diagonals). Each such path is walked row
//    by row as W sheared chains of length H (see agg_shear), so the chains of one warp sit on
//    adjacent pixels at every step. Lane groups hold 8, 16 or 32 disparities per lane and one or
//    two chains per lane; the warp's cost vectors of a step (adjacent, so contiguous in memory)
//    are copied into a shared-memory ring with cp.async several steps ahead, and its new L values
//    are staged in shared memory and added to S by one bulk reduction per step (two where the
//    run wraps around the image edge). Pairs of steps that meet no wrap, restart or last-row
//    event take a fast path without those tests (see agg_shear_t).
#pragma once
#include "common.cuh"

namespace r2t {

// Row kernel configuration for D disparities: dpl in {2, 4, 8}, lanes = next power of two
// >= D / dpl (at least 8).
__host__ __device__ inline int long_dpl_default(int D) { return D <= 64 ? 2 : (D <= 128 ? 4 : 8); }
__host__ __device__ inline int long_lanes(int D, int dpl) {
  const int l = pow2ceil((D + dpl - 1) / dpl);
  return l < 8 ? 8 : l;
}
// Work units of the row kernel of one pair: rows (both directions per lane group) or chains
// (one direction per lane group, chain 2 y walks row y left to right, chain 2 y + 1 back).
__host__ __device__ inline int row_units(int H, bool split) { return split ? 2 * H : H; }

// Adds 4 packed u16 sums (2 registers) into S at element e (uint16 or, when wide, uint32).
template <bool WIDE>
__device__ __forceinline__ void add4(void* agg, int64_t e, uint32_t a, uint32_t b) {
  if (!WIDE) {
    atomicAdd(reinterpret_cast<unsigned long long*>(reinterpret_cast<uint16_t*>(agg) + e),
              (unsigned long long)a | ((unsigned long long)b << 32));
  } else {
    unsigned long long* p =
        reinterpret_cast<unsigned long long*>(reinterpret_cast<uint32_t*>(agg) + e);
    atomicAdd(p, (unsigned long long)(a & 0xFFFFu) | ((unsigned long long)(a >> 16) << 32));
    atomicAdd(p + 1, (unsigned long long)(b & 0xFFFFu) | ((unsigned long long)(b >> 16) << 32));
  }
}
template <bool WIDE>
__device__ __forceinline__ void add2(void* agg, int64_t e, uint32_t a) {
  if (!WIDE)
    atomicAdd(reinterpret_cast<unsigned int*>(reinterpret_cast<uint16_t*>(agg) + e), a);
  else
    atomicAdd(reinterpret_cast<unsigned long long*>(reinterpret_cast<uint32_t*>(agg) + e),
              (unsigned long long)(a & 0xFFFFu) | ((unsigned long long)(a >> 16) << 32));
}
// A lane's DPL consecutive sums, starting at element e.
template <int DPL, bool WIDE>
__device__ __forceinline__ void add_lane(void* agg, int64_t e, const uint32_t (&L)[DPL / 2]) {
  constexpr int NP = DPL / 2;
  if (DPL == 2) {
    add2<WIDE>(agg, e, L[0]);
  } else {
    add4<WIDE>(agg, e, L[0], L[1 % NP]);
    if (DPL == 8) add4<WIDE>(agg, e + 4, L[2 % NP], L[3 % NP]);
  }
}

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

__device__ __forceinline__ void unpack4(uint32_t r, uint32_t& lo, uint32_t& hi) {
  lo = __byte_perm(r, 0u, 0x4140);
  hi = __byte_perm(r, 0u, 0x4342);
}

// Both halves of the result hold min(lo(v), hi(v)).
__device__ __forceinline__ uint32_t halves_min(uint32_t v) {
  return vmin2(v, __byte_perm(v, v, 0x1032));
}

// Minimum over a group of LPL lanes (aligned, LPL a power of two) of a value whose halves are
// equal. A whole warp uses redux.sync. Smaller groups use xor shuffles in radix-4 rounds (three
// independent shuffles per round), so a group of 8 or 16 lanes needs two shuffle latencies instead
// of three or four. A redux.sync with a different member mask per group measured about 15 times
// slower than a full-warp one and is not used.
template <int LPL>
__device__ __forceinline__ uint32_t group_min(uint32_t v) {
  if constexpr (LPL == 32) {
    return __reduce_min_sync(0xffffffffu, v);
  } else {
#pragma unroll
    for (int a = 1; a < LPL; a *= 4) {
      if (4 * a <= LPL) {
        const uint32_t v1 = __shfl_xor_sync(0xffffffffu, v, a, LPL);
        const uint32_t v2 = __shfl_xor_sync(0xffffffffu, v, 2 * a, LPL);
        const uint32_t v3 = __shfl_xor_sync(0xffffffffu, v, 3 * a, LPL);
        v = vmin2(vmin2(v, v1), vmin2(v2, v3));
      } else {
        v = vmin2(v, __shfl_xor_sync(0xffffffffu, v, a, LPL));
      }
    }
    return v;
  }
}

// (L(d0 - 1), L(d0)) for every pair k of a lane, from the lane's registers and its neighbours.
template <int NP, int LPL>
__device__ __forceinline__ void neighbours(const uint32_t (&L)[NP], int lig, uint32_t (&X)[NP + 1]) {
  uint32_t up = kSent << 16, dn = kSent;
  if (LPL > 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, L[NP - 1], 1, LPL);   // hi half: d0 - 1
    const uint32_t w = __shfl_down_sync(0xffffffffu, L[0], 1, LPL);      // lo half: last + 1
    up = lig == 0 ? up : u;
    dn = lig == LPL - 1 ? dn : w;
  }
  X[0] = __byte_perm(up, L[0], 0x5432);
#pragma unroll
  for (int k = 1; k < NP; k++) X[k] = __byte_perm(L[k - 1], L[k], 0x5432);
  X[NP] = __byte_perm(L[NP - 1], dn, 0x5432);
}

// ------------------------------------------------------------------------------- rows
// One pipelined step. In: L = L(q, .), mm = m(q) in both halves, c = C(p, .). Out: L(p, .),
// m(p) in both halves.
template <int DPL, int LPL, bool FULL>
__device__ __forceinline__ void long_step(uint32_t (&L)[DPL / 2], uint32_t& mm,
                                          const uint32_t (&c)[DPL / 2], bool active, int lig,
                                          uint32_t P1P1, uint32_t P2P2) {
  constexpr int NP = DPL / 2;
  uint32_t X[NP + 1];
  neighbours<NP, LPL>(L, lig, X);
  uint32_t h[NP];
  uint32_t hmin = 0xFFFFFFFFu, cmin = 0xFFFFFFFFu;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    const uint32_t g = vmin2(L[k], vmin2(X[k], X[k + 1]) + P1P1);  // <= L(q,d), no lane carry
    h[k] = g + c[k];
    hmin = vmin2(hmin, h[k]);
    cmin = vmin2(cmin, c[k]);
  }
  hmin = halves_min(hmin);
  cmin = halves_min(cmin);
  if (!FULL) {
    hmin = active ? hmin : 0xFFFFFFFFu;
    cmin = active ? cmin : 0xFFFFFFFFu;
  }
  const uint32_t aa = group_min<LPL>(hmin);  // min_d h(p, d), both halves
  const uint32_t cc = group_min<LPL>(cmin);  // min_d C(p, d), both halves
#pragma unroll
  for (int k = 0; k < NP; k++) {
    const uint32_t ln = vmin2(h[k] - mm, c[k] + P2P2);  // h >= m(q) in both halves
    L[k] = (FULL || active) ? ln : kSent * 0x10001u;
  }
  mm = vmin2(aa - mm, cc + P2P2);
}

// The same step for the two chains of a row, written stage by stage (neighbour shuffles of both,
// arithmetic of both, group minima of both, updates of both) so that one chain's shuffle and
// redux latencies overlap the other chain's work.
template <int DPL, int LPL, bool FULL>
__device__ __forceinline__ void long_step2(uint32_t (&Lf)[DPL / 2], uint32_t& mf,
                                           const uint32_t (&cf)[DPL / 2], uint32_t (&Lb)[DPL / 2],
                                           uint32_t& mb, const uint32_t (&cb)[DPL / 2],
                                           bool active, int lig, uint32_t P1P1, uint32_t P2P2) {
  constexpr int NP = DPL / 2;
  uint32_t Xf[NP + 1], Xb[NP + 1];
  neighbours<NP, LPL>(Lf, lig, Xf);
  neighbours<NP, LPL>(Lb, lig, Xb);
  uint32_t hf[NP], hb[NP];
  uint32_t hminf = 0xFFFFFFFFu, cminf = 0xFFFFFFFFu, hminb = 0xFFFFFFFFu, cminb = 0xFFFFFFFFu;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    hf[k] = vmin2(Lf[k], vmin2(Xf[k], Xf[k + 1]) + P1P1) + cf[k];
    hb[k] = vmin2(Lb[k], vmin2(Xb[k], Xb[k + 1]) + P1P1) + cb[k];
    hminf = vmin2(hminf, hf[k]);
    hminb = vmin2(hminb, hb[k]);
    cminf = vmin2(cminf, cf[k]);
    cminb = vmin2(cminb, cb[k]);
  }
  hminf = halves_min(hminf);
  hminb = halves_min(hminb);
  cminf = halves_min(cminf);
  cminb = halves_min(cminb);
  if (!FULL) {
    hminf = active ? hminf : 0xFFFFFFFFu;
    hminb = active ? hminb : 0xFFFFFFFFu;
    cminf = active ? cminf : 0xFFFFFFFFu;
    cminb = active ? cminb : 0xFFFFFFFFu;
  }
  const uint32_t aaf = group_min<LPL>(hminf), aab = group_min<LPL>(hminb);
  const uint32_t ccf = group_min<LPL>(cminf), ccb = group_min<LPL>(cminb);
#pragma unroll
  for (int k = 0; k < NP; k++) {
    const uint32_t lf = vmin2(hf[k] - mf, cf[k] + P2P2);  // h >= m(q) in both halves
    const uint32_t lb = vmin2(hb[k] - mb, cb[k] + P2P2);
    Lf[k] = (FULL || active) ? lf : kSent * 0x10001u;
    Lb[k] = (FULL || active) ? lb : kSent * 0x10001u;
  }
  mf = vmin2(aaf - mf, ccf + P2P2);
  mb = vmin2(aab - mb, ccb + P2P2);
}

// Units [unit0, min(unit0 + 32 / LPL, unit_end)) of the row kernel, one per lane group (see
// row_units). FULL: every lane of a group owns disparities (D == LPL * DPL). Lane member lig owns
// disparities [lig DPL, (lig + 1) DPL). Costs are loaded U steps ahead into a register ring that
// each step refills in place.
template <int DPL, int LPL, bool WIDE, bool FULL, bool SPLIT>
__device__ __forceinline__ void agg_rows(const Problem& pb, const Method& mt, int unit0,
                                         int unit_end) {
  typedef RawCost<DPL> RC;
  typedef typename RC::T Raw;
  constexpr int NP = DPL / 2;
  constexpr int U = DPL == 8 ? 8 : 16;  // steps loaded ahead
  const int lane = threadIdx.x & 31;
  const int lig = lane % LPL;
  const int W = pb.W, H = pb.H, D = pb.D;
  const int nu = min(row_units(H, SPLIT), unit_end);
  const int ui = unit0 + lane / LPL;
  if (LPL == 32 && ui >= nu) return;  // one unit per warp: uniform
  const bool valid = ui < nu;
  const int y = valid ? (SPLIT ? ui >> 1 : ui) : 0;
  const bool active = FULL ? valid : (valid && lig * DPL < D);
  const int d0 = active ? lig * DPL : 0;
  const int64_t pl = (int64_t)y * W, pr = pl + W - 1;  // first and last pixel of the row
  const uint32_t P1P1 = (uint32_t)mt.P1 * 0x10001u, P2P2 = (uint32_t)mt.P2 * 0x10001u;
  const int64_t nde = (int64_t)W * H * D;  // extent of the volumes (range checks)
  (void)nde;
  if constexpr (SPLIT) {
    const bool back = (ui & 1) != 0;
    const int64_t estride = back ? -(int64_t)D : (int64_t)D;
    const uint8_t* cp = pb.cost + (back ? pr : pl) * D + d0;  // next load
    int64_t e = (back ? pr : pl) * D + d0;
    uint32_t L[NP];
#pragma unroll
    for (int k = 0; k < NP; k++) L[k] = active ? 0u : kSent * 0x10001u;
    uint32_t mm = 0;
    Raw r[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      r[u] = (active && u < W && R2T_CHECKED(pb, cp, DPL, pb.cost, nde, 1)) ? RC::load(cp) : Raw();
      if (u + 1 < W) cp += estride;
    }
    int t0 = 0;
    // Blocks whose steps and refills all lie inside the row (t0 + 2U < W) test for neither and
    // add through a running pointer; the last blocks take the tested loop below.
    constexpr int BPE = WIDE ? 4 : 2;
    for (; t0 + 2 * U < W; t0 += U) {
      uint8_t* sp = reinterpret_cast<uint8_t*>(pb.agg) + e * BPE;
#pragma unroll
      for (int u = 0; u < U; u++) {
        uint32_t c[NP];
        RC::unpack(r[u], c);
        long_step<DPL, LPL, FULL>(L, mm, c, active, lig, P1P1, P2P2);
        r[u] = (active && R2T_CHECKED(pb, cp, DPL, pb.cost, nde, 1)) ? RC::load(cp)
                                                                      : Raw();  // step t0 + u + U
        cp += estride;
        if (active && R2T_CHECKED(pb, sp, DPL * BPE, pb.agg, nde * BPE, 2))
          add_lane<DPL, WIDE>(sp, 0, L);
        sp += estride * BPE;
      }
      e += U * estride;
    }
    for (; t0 < W; t0 += U) {
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int t = t0 + u;
        if (t >= W) break;
        uint32_t c[NP];
        RC::unpack(r[u], c);
        long_step<DPL, LPL, FULL>(L, mm, c, active, lig, P1P1, P2P2);
        r[u] = (active && t + U < W && R2T_CHECKED(pb, cp, DPL, pb.cost, nde, 1))
                   ? RC::load(cp)
                   : Raw();  // step t + U
        if (t + U + 1 < W) cp += estride;
        if (active && R2T_CHECKED(pb, reinterpret_cast<uint8_t*>(pb.agg) + e * BPE, DPL * BPE,
                                  pb.agg, nde * BPE, 2))
          add_lane<DPL, WIDE>(pb.agg, e, L);
        e += estride;
      }
    }
  } else {
    const int64_t estride = D;
    const uint8_t* cf = pb.cost + pl * D + d0;  // next load of each direction
    const uint8_t* cb = pb.cost + pr * D + d0;
    int64_t ef = pl * D + d0, eb = pr * D + d0;
    uint32_t Lf[NP], Lb[NP];
#pragma unroll
    for (int k = 0; k < NP; k++) Lf[k] = Lb[k] = active ? 0u : kSent * 0x10001u;
    uint32_t mf = 0, mb = 0;
    Raw rf[U], rb[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const bool ok = active && u < W;
      rf[u] = (ok && R2T_CHECKED(pb, cf, DPL, pb.cost, nde, 1)) ? RC::load(cf) : Raw();
      rb[u] = (ok && R2T_CHECKED(pb, cb, DPL, pb.cost, nde, 1)) ? RC::load(cb) : Raw();
      if (u + 1 < W) {
        cf += estride;
        cb -= estride;
      }
    }
    for (int t0 = 0; t0 < W; t0 += U) {
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int t = t0 + u;
        if (t >= W) break;
        uint32_t c1[NP], c2[NP];
        RC::unpack(rf[u], c1);
        RC::unpack(rb[u], c2);
        long_step2<DPL, LPL, FULL>(Lf, mf, c1, Lb, mb, c2, active, lig, P1P1, P2P2);
        // refill this slot with step t + U (the pointers sit there already)
        const bool ok = active && t + U < W;
        rf[u] = (ok && R2T_CHECKED(pb, cf, DPL, pb.cost, nde, 1)) ? RC::load(cf) : Raw();
        rb[u] = (ok && R2T_CHECKED(pb, cb, DPL, pb.cost, nde, 1)) ? RC::load(cb) : Raw();
        if (t + U + 1 < W) {
          cf += estride;
          cb -= estride;
        }
        if (active && R2T_CHECKED(pb, reinterpret_cast<uint8_t*>(pb.agg) + ef * (WIDE ? 4 : 2),
                                  DPL * (WIDE ? 4 : 2), pb.agg, nde * (WIDE ? 4 : 2), 2))
          add_lane<DPL, WIDE>(pb.agg, ef, Lf);
        if (active && R2T_CHECKED(pb, reinterpret_cast<uint8_t*>(pb.agg) + eb * (WIDE ? 4 : 2),
                                  DPL * (WIDE ? 4 : 2), pb.agg, nde * (WIDE ? 4 : 2), 2))
          add_lane<DPL, WIDE>(pb.agg, eb, Lb);
        ef += estride;
        eb -= estride;
      }
    }
  }
}

// The row walk of agg_rows (one direction per lane group) with the costs recomputed from the
// census descriptor map instead of read from the cost volume: for the lane's disparities
// d0 + j at pixel x, C = popcount(CT_L(x) ^ CT_R(x - d0 - j)), Eq. (image_matching), and 255 where
// x < d0 + j. CT_L(x) and the one right descriptor that enters the lane's window of DPL right
// descriptors at pixel x (CT_R(x - d0) going right, CT_R(x - d0 - DPL + 1) going left) are loaded
// UR steps ahead; the window slides by one descriptor per step.
template <int DPL, int LPL, bool WIDE, bool FULL>
__device__ __forceinline__ void agg_rows_recompute(const Problem& pb, const Method& mt, int unit0,
                                                   int unit_end) {
  constexpr int NP = DPL / 2, UR = 8;
  const int lane = threadIdx.x & 31;
  const int lig = lane % LPL;
  const int W = pb.W, H = pb.H, D = pb.D;
  const int nu = min(row_units(H, true), unit_end);
  const int ui = unit0 + lane / LPL;
  if (LPL == 32 && ui >= nu) return;  // one unit per warp: uniform
  const bool valid = ui < nu;
  const int y = valid ? ui >> 1 : 0;
  const bool active = FULL ? valid : (valid && lig * DPL < D);
  const int d0 = active ? lig * DPL : 0;
  const bool back = (ui & 1) != 0;
  const int step = back ? -1 : 1;
  const uint64_t* cl = pb.ct + (int64_t)y * W;
  const uint64_t* cr = pb.ct + (int64_t)W * H + (int64_t)y * W;
  const int enter = back ? d0 + DPL - 1 : d0;  // the entering right descriptor is CT_R(x - enter)
  const uint32_t P1P1 = (uint32_t)mt.P1 * 0x10001u, P2P2 = (uint32_t)mt.P2 * 0x10001u;
  const int64_t nde = (int64_t)W * H * D;  // extent of the volumes (range checks)
  (void)nde;
  constexpr int BPE = WIDE ? 4 : 2;
  const int64_t estride = back ? -(int64_t)D : (int64_t)D;
  int64_t e = ((int64_t)y * W + (back ? W - 1 : 0)) * D + d0;
  uint64_t sl[UR], sr[UR];
  int xf = back ? W - 1 : 0;  // pixel of the next load
#pragma unroll
  for (int u = 0; u < UR; u++) {
    sl[u] = 0;
    sr[u] = 0;
    if (active && u < W) {
      sl[u] = cl[xf];
      const int xr = xf - enter;
      if (xr >= 0) sr[u] = cr[xr];
    }
    if (u + 1 < W) xf += step;
  }
  // the window of the pixel before the first: going right every entry lies left of the image
  // (cost 255 anyway); going left win[j] = CT_R(W - d0 - j), j >= 1
  uint64_t win[DPL];
#pragma unroll
  for (int j = 0; j < DPL; j++) {
    win[j] = 0;
    const int xr = W - d0 - j;
    if (back && active && j >= 1 && xr >= 0 && xr < W) win[j] = cr[xr];
  }
  uint32_t L[NP];
#pragma unroll
  for (int k = 0; k < NP; k++) L[k] = active ? 0u : kSent * 0x10001u;
  uint32_t mm = 0;
  for (int t0 = 0; t0 < W; t0 += UR) {
#pragma unroll
    for (int u = 0; u < UR; u++) {
      const int t = t0 + u;
      if (t >= W) break;
      const int x = back ? W - 1 - t : t;
      if (back) {
#pragma unroll
        for (int j = 0; j + 1 < DPL; j++) win[j] = win[j + 1];
        win[DPL - 1] = sr[u];
      } else {
#pragma unroll
        for (int j = DPL - 1; j > 0; j--) win[j] = win[j - 1];
        win[0] = sr[u];
      }
      uint32_t cv[DPL];
#pragma unroll
      for (int j = 0; j < DPL; j++)
        cv[j] = x < d0 + j ? (uint32_t)kCostOutside : (uint32_t)__popcll(sl[u] ^ win[j]);
      uint32_t c[NP];
#pragma unroll
      for (int k = 0; k < NP; k++) c[k] = cv[2 * k] | (cv[2 * k + 1] << 16);
      long_step<DPL, LPL, FULL>(L, mm, c, active, lig, P1P1, P2P2);
      if (active && t + UR < W) {  // refill this slot with step t + UR (pixel xf)
        sl[u] = cl[xf];
        const int xr = xf - enter;
        sr[u] = xr >= 0 ? cr[xr] : 0ull;
      }
      if (t + UR + 1 < W) xf += step;
      if (active && R2T_CHECKED(pb, reinterpret_cast<uint8_t*>(pb.agg) + e * BPE, DPL * BPE,
                                pb.agg, nde * BPE, 2))
        add_lane<DPL, WIDE>(pb.agg, e, L);
      e += estride;
    }
  }
}

// ------------------------------------------------------------------------------- sheared columns
// Kinds of sheared chain: 0 TB, 1 BT, 2 TLBR, 3 BRTL, 4 TRBL, 5 BLTR. Chain j of a kind with shear
// s (0 for kinds 0-1, +1 for 2-3, -1 for 4-5) visits pixel x = (j + s y) mod W of every row y,
// top-down for the even kinds and bottom-up for the odd ones, so one step moves it by
// (dx, dy) = (s, 1) or (-s, -1): the direction r of its path. Where x wraps around (x = 0 after a
// step with dx = +1, x = W - 1 after dx = -1) the pixel's predecessor lies outside the image: a
// new line of the path enters there and the chain restarts with L = C. Every pixel lies on exactly
// one chain of each kind, j = (x - s y) mod W, so the W chains of a kind cover its path once.
constexpr int kShearRing = 8;  // steps in the cost ring; 2 steps per cp.async group, 6 in flight

__host__ __device__ inline int shear_kinds(int num_paths) { return num_paths == 8 ? 6 : 2; }
__host__ __device__ inline int shear_dpl_default(int D) { return 16; }
// Two chains per lane at D = 128: the step's bookkeeping serves both and the halved warp count
// competes less with the concurrent row kernel (aggregation stage 5 % faster at 1242 x 375, in
// 0.229 ms instead of 0.242); one at the other D, where it was not measured.
__host__ __device__ inline int shear_cpl_default(int D) { return D == 128 ? 2 : 1; }
__host__ __device__ inline int shear_width(int D, int dpl) { return pow2ceil(D / dpl); }
// Warp items of one pair: kinds x groups of cpl * 32 / width adjacent chains (cpl chains per lane).
__host__ __device__ inline int shear_items(int W, int D, int dpl, int num_paths, int cpl) {
  const int ch = cpl * (32 / shear_width(D, dpl));
  return shear_kinds(num_paths) * ((W + ch - 1) / ch);
}
// Shared memory of one warp: the cost ring (kShearRing steps of cpl * 32 / width pixel vectors of
// D bytes, at most 32 cpl dpl bytes per step) and the staging buffers of the steps' sums.
__host__ __device__ inline int shear_ring_bytes(int dpl, int cpl) { return kShearRing * 32 * dpl * cpl; }
__host__ __device__ inline int shear_stage_bytes(int dpl, bool wide, int cpl) {
  return 32 * dpl * cpl * (wide ? 4 : 2);
}
// Ring plus two staging buffers (steps alternate between them).
__host__ __device__ inline int shear_smem_bytes(int dpl, bool wide, int cpl) {
  return shear_ring_bytes(dpl, cpl) + 2 * shear_stage_bytes(dpl, wide, cpl);
}

// Position, in 16-byte pieces, of piece i of pixel slot c in a buffer of pixel vectors of pp
// pieces each. When pp is a power of two the pieces of slot c are permuted by c, so lanes that
// access the same piece index of adjacent pixels hit different shared-memory banks.
__device__ __forceinline__ int swz(int c, int i, int pp) {
  return c * pp + ((pp & (pp - 1)) == 0 ? (i ^ (c & (pp - 1))) : i);
}

__device__ __forceinline__ uint4 lds128(uint32_t a) {
  uint4 r;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
               : "r"(a));
  return r;
}
__device__ __forceinline__ void sts128(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w)
               : "memory");
}
__device__ __forceinline__ unsigned long long lds64(uint32_t a) {
  unsigned long long r;
  asm volatile("ld.shared.u64 %0, [%1];" : "=l"(r) : "r"(a));
  return r;
}

// Warp item of the sheared-column kernel: CH = CPL * 32 / WD adjacent chains of one kind, WD lanes
// per chain and CPL chains per lane (lane (c, lig) walks chains c, c + 32 / WD, ...), DPL
// disparities per lane and chain (member lig owns [lig DPL, (lig + 1) DPL)). FULL: every lane owns
// disparities (D == WD * DPL). SH0: the kind has shear 0 (columns), so its runs never wrap and its
// chains never restart. ring / stage: this warp's shear_ring_bytes(DPL, CPL) and
// 2 shear_stage_bytes(DPL, WIDE, CPL) bytes of shared memory, 16-byte aligned.
//
// Per step (one row): the warp's costs were copied 6 steps earlier by all lanes, each lane taking
// 16-byte pieces of the contiguous pixel run so that every copy instruction is coalesced; after
// cp.async.wait_group and __syncwarp each lane reads its own pieces. The new L values go to a
// staging buffer in the volume's layout, which one bulk reduction adds into S. Lanes of chains
// past the image's last column
// (and, FULL, every lane) compute unconditionally; only their copies and adds are skipped. With
// CPL = 2 the step's bookkeeping (syncs, ring slots, run pointers) serves twice the chains and the
// two chains' arithmetic interleaves.
//
// Events - a run that wraps around the image edge (copy or add in two parts), a chain that
// restarts because a new line of the path enters, a cursor that wraps, the last rows - happen only
// in a window of about CH + 8 steps each time the run passes the edge column, and near the end.
// Between them the walk takes pairs of steps on a fast path that tests for none of them (ring slot
// and staging buffer follow from the step index); each event step takes the general path.
template <int DPL, int WD, int CPL, bool WIDE, bool FULL, bool SH0>
__device__ __forceinline__ void agg_shear_t(const Problem& pb, const Method& mt, int kind, int j0,
                                            uint8_t* ring, uint8_t* stage) {
  constexpr int NP = DPL / 2;
  constexpr int CPW = 32 / WD;                // chains per warp and lane slot
  constexpr int CH = CPW * CPL;               // chains of the warp item
  constexpr int KS = kShearRing;
  constexpr int BPE = WIDE ? 4 : 2;           // bytes per sum
  constexpr int CW = DPL < 16 ? DPL : 16;     // disparities per cost read (8 or 16 bytes)
  constexpr int NVC = DPL / CW;               // cost reads a lane makes per chain and step
  constexpr int NCP = CPL * DPL >= 16 ? CPL * DPL / 16 : 1;  // 16-byte pieces a lane copies per step
  constexpr int NVS = DPL * BPE / 16;         // sum pieces a lane stages per chain and step
  constexpr int NA = NP < 4 ? NP : 4;         // independent accumulators of a lane's minimum
  static_assert(KS == 8, "two copied steps per group, three groups ahead");
  const int lane = threadIdx.x & 31;
  const int lig = lane % WD, c = lane / WD;
  const int W = pb.W, H = pb.H;
  const int D = FULL ? WD * DPL : pb.D;
  const int PP = D / 16;        // cost pieces per pixel
  const int PS = D * BPE / 16;  // sum pieces per pixel
  const int n = min(CH, W - j0);  // chains of this warp item
  const int sh = SH0 ? 0 : (kind < 4 ? 1 : -1);
  const bool back = (kind & 1) != 0;
  const int dy = back ? -1 : 1, dx = back ? -sh : sh;
  const int ystart = back ? H - 1 : 0;
  int xs = (j0 + sh * ystart) % W;  // pixel of chain 0 in the current row
  if (xs < 0) xs += W;
  const bool owns = FULL || lig * DPL < D;  // the lane holds disparities of its chains
  const int slot_bytes = CH * D;
  const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
  const uint32_t stage_s = (uint32_t)__cvta_generic_to_shared(stage);
  const int stage_bytes = CH * D * BPE;  // one step's run of sums (two such buffers)
  const uint32_t P1P1 = (uint32_t)mt.P1 * 0x10001u, P2P2 = (uint32_t)mt.P2 * 0x10001u;
  // bytes from one step's run to the next (before any wrap correction)
  const int64_t cstride = ((int64_t)dy * W + dx) * D, astride = cstride * BPE;
  const int64_t cwrap = (int64_t)W * D, awrap = cwrap * BPE;  // one row, subtracted at a wrap
  const int64_t nde = (int64_t)W * H * D;  // extent of the volumes (range checks)
  (void)nde;

  // Per-lane pieces, fixed for the whole walk: cost piece v of the step's run (chain cp_c[v],
  // shared offset cp_s[v] inside a ring slot); the lane's own cost pieces (rd_s) and sum pieces
  // (st_s, in the run's memory order) of each of its chains. A run that does not wrap around the
  // image edge is contiguous in memory, so piece v then sits 16 (lane + 32 v) bytes after the
  // run's start.
  int cp_c[NCP], cp_s[NCP], rd_s[CPL][NVC], st_s[CPL][NVS];
  bool act[CPL];  // the lane's chain g exists and the lane owns disparities of it
#pragma unroll
  for (int v = 0; v < NCP; v++) {
    const int p = lane + 32 * v;
    const int pc = p / PP, pi = p - pc * PP;
    cp_c[v] = pc < n ? pc : -1;
    cp_s[v] = swz(pc, pi, PP) * 16;
  }
#pragma unroll
  for (int g = 0; g < CPL; g++) {
    const int cg = c + CPW * g;
    act[g] = owns && cg < n;
#pragma unroll
    for (int v = 0; v < NVC; v++) {
      const int b = lig * DPL + v * CW;  // byte of the pixel's cost vector
      rd_s[g][v] = swz(cg, b >> 4, PP) * 16 + (b & 15);
    }
#pragma unroll
    for (int v = 0; v < NVS; v++) st_s[g][v] = (cg * PS + lig * NVS + v) * 16;
  }
  auto slot_of = [&](int t) { return ring_s + (uint32_t)((t & (KS - 1)) * slot_bytes); };

  // copy cursor: global start of the next copied step's run and its column
  const uint8_t* crun = pb.cost + ((int64_t)ystart * W + xs) * D;
  int xc = xs;
  // General copy of step tc (past the last row: nothing), its run possibly wrapping around the
  // image edge.
  auto copy_step = [&](int tc) {
    if (tc < H) {
      const uint32_t cslot = slot_of(tc);
      if (SH0 || xc + n <= W) {  // contiguous run
        const uint8_t* src = crun + 16 * lane;
#pragma unroll
        for (int v = 0; v < NCP; v++)
          if (cp_c[v] >= 0 && R2T_CHECKED(pb, src + 512 * v, 16, pb.cost, nde, 3))
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(cslot + cp_s[v]),
                         "l"(src + 512 * v));
      } else {
#pragma unroll
        for (int v = 0; v < NCP; v++) {
          if (cp_c[v] >= 0) {
            const int p = lane + 32 * v;
            const int pc = cp_c[v], pi = p - pc * PP;
            const int back_w = xc + pc >= W ? W : 0;  // wrapped to the row's start
            const uint8_t* a = crun + ((int64_t)pc - back_w) * D + pi * 16;
            if (R2T_CHECKED(pb, a, 16, pb.cost, nde, 3))
              asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(cslot + cp_s[v]),
                           "l"(a));
          }
        }
      }
      crun += cstride;
      if (!SH0) {
        xc += dx;
        if (xc >= W) {
          xc -= W;
          crun -= cwrap;
        } else if (xc < 0) {
          xc += W;
          crun += cwrap;
        }
      }
    }
  };
  // Fast copy of steps tc and tc + 1: both before the last row, both runs contiguous, and the
  // cursor does not wrap after them.
  auto copy_two = [&](int tc) {
    const uint32_t s0 = slot_of(tc), s1 = slot_of(tc + 1);
    const uint8_t* src = crun + 16 * lane;
#pragma unroll
    for (int v = 0; v < NCP; v++)
      if (cp_c[v] >= 0 && R2T_CHECKED(pb, src + 512 * v, 16, pb.cost, nde, 3))
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s0 + cp_s[v]),
                     "l"(src + 512 * v));
#pragma unroll
    for (int v = 0; v < NCP; v++)
      if (cp_c[v] >= 0 && R2T_CHECKED(pb, src + cstride + 512 * v, 16, pb.cost, nde, 3))
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s1 + cp_s[v]),
                     "l"(src + cstride + 512 * v));
    crun += 2 * cstride;
    if (!SH0) xc += 2 * dx;
  };

  uint32_t L[CPL][NP], mm[CPL];
#pragma unroll
  for (int g = 0; g < CPL; g++) {
#pragma unroll
    for (int k = 0; k < NP; k++) L[g][k] = owns ? 0u : kSent * 0x10001u;
    mm[g] = 0;
  }
  uint8_t* arun = reinterpret_cast<uint8_t*>(pb.agg) + ((int64_t)ystart * W + xs) * D * BPE;

  // The step's cost pieces, all loaded before any is used.
  auto load_costs = [&](int t, uint4 (&raw)[CPL][NVC]) {
    const uint32_t cur = slot_of(t);
#pragma unroll
    for (int g = 0; g < CPL; g++)
#pragma unroll
      for (int v = 0; v < NVC; v++)
        if (CW == 16) {
          raw[g][v] = owns ? lds128(cur + rd_s[g][v]) : make_uint4(0, 0, 0, 0);
        } else {
          const unsigned long long r8 = owns ? lds64(cur + rd_s[g][v]) : 0ull;
          raw[g][v] = make_uint4((uint32_t)r8, (uint32_t)(r8 >> 32), 0u, 0u);
        }
  };
  // One step of the recurrence on every chain of the lane, L and mm in place, and its sums into
  // staging buffer par (the step's parity).
  auto update = [&](int par, const uint4 (&raw)[CPL][NVC]) {
    // Neighbour pairs are formed on the fly from the old L: xp = (L(d0 - 1), L(d0)) of pair k,
    // xn the same for pair k + 1; L[k] is overwritten only after both were formed.
    uint32_t xp[CPL], dn[CPL], mP2[CPL], lm[CPL][NA];
#pragma unroll
    for (int g = 0; g < CPL; g++) {
      uint32_t up = kSent << 16;
      dn[g] = kSent;
      if (WD > 1) {
        const uint32_t a = __shfl_up_sync(0xffffffffu, L[g][NP - 1], 1, WD);
        const uint32_t b = __shfl_down_sync(0xffffffffu, L[g][0], 1, WD);
        up = lig == 0 ? up : a;
        dn[g] = lig == WD - 1 ? dn[g] : b;
      }
      xp[g] = __byte_perm(up, L[g][0], 0x5432);
      mP2[g] = mm[g] + P2P2;
#pragma unroll
      for (int a = 0; a < NA; a++) lm[g][a] = 0xFFFFFFFFu;
    }
#pragma unroll
    for (int v = 0; v < NVC; v++) {  // CW disparities (CW / 2 pairs) per cost read
      uint32_t cst[CPL][8];
#pragma unroll
      for (int g = 0; g < CPL; g++) {
        unpack4(raw[g][v].x, cst[g][0], cst[g][1]);
        unpack4(raw[g][v].y, cst[g][2], cst[g][3]);
        unpack4(raw[g][v].z, cst[g][4], cst[g][5]);
        unpack4(raw[g][v].w, cst[g][6], cst[g][7]);
      }
#pragma unroll
      for (int j = 0; j < CW / 2; j++) {
        const int k = (CW / 2) * v + j;
#pragma unroll
        for (int g = 0; g < CPL; g++) {
          const uint32_t xn =
              __byte_perm(L[g][k], k + 1 < NP ? L[g][(k + 1) % NP] : dn[g], 0x5432);
          const uint32_t tt = vmin2(xp[g], xn) + P1P1;
          const uint32_t uu = vmin2(vmin2(L[g][k], tt), mP2[g]);  // >= m(q) in both halves
          const uint32_t ln = uu + cst[g][j] - mm[g];             // each half in [0, 255 + P2]
          L[g][k] = owns ? ln : kSent * 0x10001u;
          lm[g][k % NA] = vmin2(lm[g][k % NA], L[g][k]);
          xp[g] = xn;
        }
      }
    }
#pragma unroll
    for (int g = 0; g < CPL; g++) {
#pragma unroll
      for (int w = 1; w < NA; w *= 2)
#pragma unroll
        for (int a = 0; a + w < NA; a += 2 * w) lm[g][a] = vmin2(lm[g][a], lm[g][a + w]);
      mm[g] = group_min<WD>(halves_min(lm[g][0]));
    }
    const uint32_t sbuf = stage_s + (uint32_t)(par * stage_bytes);
#pragma unroll
    for (int g = 0; g < CPL; g++) {
      if (FULL || act[g]) {
#pragma unroll
        for (int v = 0; v < NVS; v++) {
          const uint32_t a = sbuf + (uint32_t)st_s[g][v];
          if (!WIDE)
            sts128(a, L[g][4 * v], L[g][4 * v + 1], L[g][4 * v + 2], L[g][4 * v + 3]);
          else
            sts128(a, L[g][2 * v] & 0xFFFFu, L[g][2 * v] >> 16, L[g][2 * v + 1] & 0xFFFFu,
                   L[g][2 * v + 1] >> 16);
        }
      }
    }
    // The run's sums go to S with bulk reductions issued by lane 0 (below): the tensor memory
    // accelerator adds the staged 32-bit words (two packed u16 sums each, which cannot carry into
    // each other, or one u32 sum when wide) into S atomically, element by element. The staging
    // writes are made visible to that async proxy first.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
  };
  // The bulk add of the step's run from staging buffer par (n1 pixels from arun, the rest from
  // the row's start).
  auto add_run = [&](int par, int n1) {
    if (lane == 0) {
      const uint32_t sbuf = stage_s + (uint32_t)(par * stage_bytes);
      if (R2T_CHECKED(pb, arun, (int64_t)n1 * D * BPE, pb.agg, nde * BPE, 4))
        asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u32 [%0], [%1], %2;"
                     ::"l"(arun), "r"(sbuf), "r"(n1 * D * BPE) : "memory");
      if (!SH0 && n1 < n &&
          R2T_CHECKED(pb, arun - (int64_t)xs * D * BPE, (int64_t)(n - n1) * D * BPE, pb.agg,
                      nde * BPE, 5))
        asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u32 [%0], [%1], %2;"
                     ::"l"(arun - (int64_t)xs * D * BPE), "r"(sbuf + n1 * D * BPE),
                     "r"((n - n1) * D * BPE)
                     : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  };
  // Start of every step: the bulk add issued two steps ago has read the staging buffer this step
  // refills (bulk groups are per thread: lanes other than lane 0 have none and pass at once); on
  // even steps, issue the copies of steps t + 6, t + 7 (fast or general) and wait for steps t,
  // t + 1.
  auto begin_step = [&](int t, bool even, bool fast) {
    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
    __syncwarp();  // every lane is done with the ring slot refilled below and with the staging
    if (even) {
      if (fast) {
        copy_two(t + KS - 2);
      } else {
        copy_step(t + KS - 2);
        copy_step(t + KS - 1);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      asm volatile("cp.async.wait_group 3;" ::: "memory");
      __syncwarp();
    }
  };
  // Pairs of fast steps from even step t: for steps t .. t + 7 (the pair and its copies) the runs
  // neither wrap nor restart a chain and the cursors do not wrap. Going right that holds while
  // 1 <= xs and xs + 7 <= min(W - n, W - 2); going left while 8 <= xs <= W - n - 1 (a chain
  // restarts at column 0 going right, W - 1 going left).
  auto fast_pairs = [&](int t) -> int {
    const int qh = H - KS - t;  // the pair's copies must be of rows before H
    if (qh < 0) return 0;
    int q = qh >> 1;
    if (!SH0) {
      if (dx > 0) {
        const int lim = min(W - n, W - 2) - (KS - 1);
        if (xs < 1 || xs > lim) return 0;
        q = min(q, (lim - xs) >> 1);
      } else {
        if (xs < KS || xs > W - n - 1) return 0;
        q = min(q, (xs - KS) >> 1);
      }
    }
    return q + 1;
  };

  // prologue: steps 0 .. 5 in flight as three groups of two
#pragma unroll
  for (int s = 0; s < KS - 2; s += 2) {
    copy_step(s);
    copy_step(s + 1);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  int t = 0;
  while (t < H) {
    for (int np = (t & 1) ? 0 : fast_pairs(t); np > 0; np--, t += 2) {
#pragma unroll
      for (int u = 0; u < 2; u++) {
        uint4 raw[CPL][NVC];
        begin_step(t + u, u == 0, true);
        load_costs(t + u, raw);
        update(u, raw);
        add_run(u, n);
        arun += astride;
        if (!SH0) xs += dx;
      }
    }
    if (t >= H) break;
    // general step
    uint4 raw[CPL][NVC];
    const int par = t & 1;
    begin_step(t, par == 0, false);
    load_costs(t, raw);
    if (!SH0 && t > 0) {  // a new line of the path enters where a chain reaches the edge: L = C
      const int edge = dx > 0 ? 0 : W - 1;
      bool hit[CPL], any = false;
#pragma unroll
      for (int g = 0; g < CPL; g++) {
        hit[g] = (xs + c + CPW * g) % W == edge;
        any |= hit[g];
      }
      if (__any_sync(0xffffffffu, any)) {
#pragma unroll
        for (int g = 0; g < CPL; g++) {
          if (hit[g]) {
#pragma unroll
            for (int k = 0; k < NP; k++) L[g][k] = owns ? 0u : kSent * 0x10001u;
            mm[g] = 0;
          }
        }
      }
    }
    update(par, raw);
    add_run(par, (!SH0 && xs + n > W) ? W - xs : n);  // pixels before the wrap
    arun += astride;
    if (!SH0) {
      xs += dx;
      if (xs >= W) {  // chain 0 left the row at one side: back in at the other
        xs -= W;
        arun -= awrap;
      } else if (xs < 0) {
        xs += W;
        arun += awrap;
      }
    }
    t++;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // adds complete
  __syncwarp();
}

// Warp item `item` of a pair's sheared-column work (see shear_items). Items run kind by kind in
// the order TB, TLBR, TRBL, BT, BRTL, BLTR: the three downward kinds first, then the three upward
// ones. Warps that start together walk the same rows at about the same time, so when the downward
// kinds' warps are resident together they add into the same band of S while it is in L2 (one
// DRAM round trip of that band instead of one per kind); the upward kinds share the band moving
// up. Kind-major order with both directions of a kind together kept them apart on images whose
// warps do not all fit on the GPU at once (1920 x 1080, D = 256: 27.6 B of DRAM traffic per
// disparity estimate for the six kinds).
__device__ __forceinline__ int shear_kind_of(int k, int num_kinds) {
  return num_kinds == 6 ? (k < 3 ? 2 * k : 2 * (k - 3) + 1) : k;
}

template <int DPL, int WD, int CPL, bool WIDE, bool FULL>
__device__ __forceinline__ void agg_shear(const Problem& pb, const Method& mt, int item,
                                          uint8_t* ring, uint8_t* stage) {
  constexpr int CH = CPL * (32 / WD);
  const int G = (pb.W + CH - 1) / CH;
  const int k = item / G;
  const int kind = shear_kind_of(k, shear_kinds(mt.num_paths));
  const int j0 = (item - k * G) * CH;
  if (kind < 2)
    agg_shear_t<DPL, WD, CPL, WIDE, FULL, true>(pb, mt, kind, j0, ring, stage);
  else
    agg_shear_t<DPL, WD, CPL, WIDE, FULL, false>(pb, mt, kind, j0, ring, stage);
}

}  // namespace r2t
