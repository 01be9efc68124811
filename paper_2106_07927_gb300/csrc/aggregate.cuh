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
// one line with the D disparities spread over its lanes, held as packed u16x2 registers.
// Neighbouring disparities cross lanes by one shuffle each way; the line's costs are added into
// S with 64-bit atomic adds of four packed u16 lanes (no carry can cross a lane while
// num_paths (255 + P2) <= 65535; above that the sums are uint32, "wide"). Integer addition is
// associative, so the order in which directions arrive does not change S.
// Two kernels split the lines:
//  - the long axis (rows when W >= H, else columns) holds the longest chains, which bound the
//    kernel's duration. One warp walks a line in both directions (two chains for ILP) with few
//    disparities per lane, and forms m with a pipelined reduction: writing
//    g(q,d) = min(L(q,d), L(q,d-1) + P1, L(q,d+1) + P1) and h(p,d) = C(p,d) + g(q,d),
//      L(p,d) = min(h(p,d) - m(q), C(p,d) + P2),
//      m(p)   = min(min_d h(p,d) - m(q), min_d C(p,d) + P2),
//    so the group minima of h and of C (redux.sync) do not wait for m(q) and overlap the next
//    step.
//  - the other axes (short lines, many of them) run one chain per small lane group with 32
//    disparities per lane, which amortises shuffles and reductions over much more arithmetic.
// Costs are fetched several steps ahead (registers in the first kernel, a per-lane cp.async ring
// in shared memory in the second). The cost and S vectors use a blocked disparity order
// (VolOrder) matched to the second kernel, so each lane group's copies and atomic adds touch
// contiguous memory in both kernels.
#pragma once
#include "common.cuh"

namespace r2t {

struct LineGeom {
  int sx, sy, dx, dy, len;
};

// Axes: 0 rows (LR/RL), 1 columns (TB/BT), 2 diagonals x - y = const (TLBR/BRTL),
// 3 anti-diagonals x + y = const (TRBL/BLTR). Line i of an axis, walked forward.
__host__ __device__ inline int axis_lines(int axis, int W, int H) {
  return axis == 0 ? H : (axis == 1 ? W : W + H - 1);
}
__host__ __device__ inline LineGeom axis_line(int axis, int i, int W, int H) {
  LineGeom g;
  if (axis == 0) {
    g.sx = 0; g.sy = i; g.dx = 1; g.dy = 0; g.len = W;
  } else if (axis == 1) {
    g.sx = i; g.sy = 0; g.dx = 0; g.dy = 1; g.len = H;
  } else if (axis == 2) {
    const int k = i - (H - 1);
    g.sx = k > 0 ? k : 0;
    g.sy = k < 0 ? -k : 0;
    g.dx = 1; g.dy = 1;
    g.len = (W - g.sx) < (H - g.sy) ? (W - g.sx) : (H - g.sy);
  } else {
    g.sy = i - (W - 1) > 0 ? i - (W - 1) : 0;
    g.sx = i - g.sy;
    g.dx = -1; g.dy = 1;
    g.len = (g.sx + 1) < (H - g.sy) ? (g.sx + 1) : (H - g.sy);
  }
  return g;
}
__host__ __device__ inline int long_axis(int W, int H) { return W >= H ? 0 : 1; }
// Axes of the second kernel: the other straight axis, plus both diagonals with 8 paths.
__host__ __device__ inline int bulk_axes(int W, int H, int num_paths, int (&axes)[3]) {
  axes[0] = 1 - long_axis(W, H);
  if (num_paths == 8) {
    axes[1] = 2;
    axes[2] = 3;
    return 3;
  }
  return 1;
}
__host__ __device__ inline int bulk_num_lines(int W, int H, int num_paths) {
  int axes[3];
  const int na = bulk_axes(W, H, num_paths, axes);
  int n = 0;
  for (int a = 0; a < na; a++) n += axis_lines(axes[a], W, H);
  return n;
}
__host__ __device__ inline LineGeom bulk_line(int li, int W, int H, int num_paths) {
  int axes[3];
  const int na = bulk_axes(W, H, num_paths, axes);
  for (int a = 0; a < na; a++) {
    const int n = axis_lines(axes[a], W, H);
    if (li < n) return axis_line(axes[a], li, W, H);
    li -= n;
  }
  LineGeom g;
  g.sx = g.sy = g.dx = g.dy = g.len = 0;
  return g;
}

// Kernel configurations for D disparities. Long axis: dpl in {2, 4, 8}, lanes = next power of
// two >= D / dpl (at least 8). Other axes: bulk_dpl(D) disparities per lane, group width = next
// power of two >= D / dpl.
__host__ __device__ inline int long_dpl_default(int D) { return D <= 64 ? 2 : (D <= 128 ? 4 : 8); }
__host__ __device__ inline int long_lanes(int D, int dpl) {
  const int l = pow2ceil((D + dpl - 1) / dpl);
  return l < 8 ? 8 : l;
}
__host__ __device__ inline int bulk_width(int D) { return pow2ceil(D / bulk_dpl(D)); }

// Slots (steps) of the per-lane cp.async ring of the other-axes kernel. Two steps form one commit
// group and each pair of steps waits with cp.async.wait_group 3, so six steps are in flight.
constexpr int kBulkRing = 8;
__host__ __device__ inline int bulk_ring_bytes(int dpl) { return kBulkRing * (dpl / 16) * 32 * 16; }

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

// Minimum over a group of LPL lanes of a value whose halves are equal.
template <int LPL>
__device__ __forceinline__ uint32_t group_min(uint32_t v) {
  if (LPL == 32) return __reduce_min_sync(0xffffffffu, v);
#pragma unroll
  for (int o = LPL / 2; o >= 1; o >>= 1) v = vmin2(v, __shfl_xor_sync(0xffffffffu, v, o, LPL));
  return v;
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

// ------------------------------------------------------------------------------- long axis
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

// The same step for the two chains of a line, written stage by stage (neighbour shuffles of both,
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

// Lines [line0, min(line0 + 32 / LPL, line_end)) of the long axis, both directions each.
// FULL: every lane of a group owns disparities (D == LPL * DPL). Costs are loaded U steps ahead
// into a register ring that each step refills in place.
template <int DPL, int LPL, bool WIDE, bool FULL>
__device__ __forceinline__ void agg_long_lines(const Problem& pb, const Method& mt, int line0,
                                               int line_end) {
  typedef RawCost<DPL> RC;
  typedef typename RC::T Raw;
  constexpr int NP = DPL / 2;
  constexpr int U = DPL == 8 ? 8 : 16;  // steps loaded ahead
  const int lane = threadIdx.x & 31;
  const int lig = lane % LPL;
  const int W = pb.W, H = pb.H, D = pb.D;
  const int la = long_axis(W, H);
  const int nl = min(axis_lines(la, W, H), line_end);
  const int li = line0 + lane / LPL;
  if (LPL == 32 && li >= nl) return;  // one line per warp: uniform
  const bool valid = li < nl;
  const LineGeom g = axis_line(la, valid ? li : 0, W, H);  // every line of the axis has len
  const int len = g.len;
  const bool active = FULL ? valid : (valid && lig * DPL < D);
  const int d0 = active ? lig * DPL : 0;
  const int coff = vol_pos(d0, pb.ord, 4);  // DPL consecutive bytes
  const int soff0 = vol_pos(d0, pb.ord, 2);  // first 4 (or 2) sums
  const int soff1 = DPL == 8 ? vol_pos(d0 + 4, pb.ord, 2) - soff0 : 0;
  const int64_t pstride = (int64_t)g.dy * W + g.dx;  // pixels per step
  const int64_t estride = pstride * D;                // volume elements per step
  const int64_t pf = (int64_t)g.sy * W + g.sx;
  const int64_t pbk = pf + (int64_t)(len - 1) * pstride;
  const uint32_t P1P1 = (uint32_t)mt.P1 * 0x10001u, P2P2 = (uint32_t)mt.P2 * 0x10001u;
  const uint8_t* cf = pb.cost + pf * D + coff;  // next load of each direction
  const uint8_t* cb = pb.cost + pbk * D + coff;
  int64_t ef = pf * D + soff0, eb = pbk * D + soff0;

  uint32_t Lf[NP], Lb[NP];
#pragma unroll
  for (int k = 0; k < NP; k++) Lf[k] = Lb[k] = active ? 0u : kSent * 0x10001u;
  uint32_t mf = 0, mb = 0;

  Raw rf[U], rb[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    const bool ok = active && u < len;
    rf[u] = ok ? RC::load(cf) : Raw();
    rb[u] = ok ? RC::load(cb) : Raw();
    if (u + 1 < len) {
      cf += estride;
      cb -= estride;
    }
  }
  for (int t0 = 0; t0 < len; t0 += U) {
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int t = t0 + u;
      if (t >= len) break;
      uint32_t c1[NP], c2[NP];
      RC::unpack(rf[u], c1);
      RC::unpack(rb[u], c2);
      long_step2<DPL, LPL, FULL>(Lf, mf, c1, Lb, mb, c2, active, lig, P1P1, P2P2);
      // refill this slot with step t + U (the pointers sit there already)
      const bool ok = active && t + U < len;
      rf[u] = ok ? RC::load(cf) : Raw();
      rb[u] = ok ? RC::load(cb) : Raw();
      if (t + U + 1 < len) {
        cf += estride;
        cb -= estride;
      }
      if (active) {
        if (DPL == 2) {
          add2<WIDE>(pb.agg, ef, Lf[0]);
          add2<WIDE>(pb.agg, eb, Lb[0]);
        } else {
          add4<WIDE>(pb.agg, ef, Lf[0], Lf[1 % NP]);
          add4<WIDE>(pb.agg, eb, Lb[0], Lb[1 % NP]);
          if (DPL == 8) {
            add4<WIDE>(pb.agg, ef + soff1, Lf[2 % NP], Lf[3 % NP]);
            add4<WIDE>(pb.agg, eb + soff1, Lb[2 % NP], Lb[3 % NP]);
          }
        }
      }
      ef += estride;
      eb -= estride;
    }
  }
}

// ------------------------------------------------------------------------------- other axes
// Chains [chain0, min(chain0 + 32 / WD, chain_end)): chain c walks line c / 2 of the other axes,
// forward when c is even, backward when odd. WD lanes per chain, DPL disparities per lane.
// FULL: every lane owns disparities (D == WD * DPL). Each lane copies its own 16-byte cost
// pieces into `ring` (this warp's kBulkRing * (DPL / 16) * 32 uint4) with cp.async and waits
// only for its own copies, kBulkRing - 1 steps ahead.
template <int DPL, int WD, bool WIDE, bool FULL>
__device__ __forceinline__ void agg_bulk_chains(const Problem& pb, const Method& mt, int chain0,
                                                int chain_end, uint4* ring) {
  constexpr int NP = DPL / 2;
  constexpr int NV = DPL / 16;  // 16-byte cost vectors per lane and step
  constexpr int KS = kBulkRing;
  const int lane = threadIdx.x & 31;
  const int lig = lane % WD;
  const int W = pb.W, H = pb.H, D = pb.D;
  const int nc = min(2 * bulk_num_lines(W, H, mt.num_paths), chain_end);
  const int ci = chain0 + lane / WD;
  const bool valid = ci < nc;
  LineGeom g = bulk_line(valid ? ci >> 1 : 0, W, H, mt.num_paths);
  if (!valid) g.len = 0;
  const int maxlen = (int)__reduce_max_sync(0xffffffffu, (unsigned)g.len);
  if (maxlen == 0) return;
  const bool back = (ci & 1) != 0;
  const bool active = FULL ? valid : (valid && lig * DPL < D);
  int64_t pstride = (int64_t)g.dy * W + g.dx;
  int64_t px = (int64_t)g.sy * W + g.sx;
  if (back) {
    px += (int64_t)(g.len - 1) * pstride;
    pstride = -pstride;
  }
  const int64_t estride = pstride * D;
  // lane member lig owns disparities [lig * DPL, (lig + 1) * DPL): its cost piece v sits at
  // cbo + v * cvs bytes and its sum chunk k at sbo + k * svs elements of the pixel vector
  const int cvs = FULL ? WD * 16 : (pb.ord.blocked ? (D / DPL) * 16 : 16);
  const int svs = FULL ? WD * 4 : (pb.ord.blocked ? (D / DPL) * 4 : 4);
  const int cbo = (FULL || pb.ord.blocked) ? lig * 16 : lig * DPL;
  const int sbo = (FULL || pb.ord.blocked) ? lig * 4 : lig * DPL;
  const uint8_t* cp = pb.cost + px * D + cbo;  // next step to copy
  int64_t e = px * D + sbo;                     // element of this step's first sum
  const uint32_t P1P1 = (uint32_t)mt.P1 * 0x10001u, P2P2 = (uint32_t)mt.P2 * 0x10001u;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(ring);

  uint32_t L[NP];
#pragma unroll
  for (int k = 0; k < NP; k++) L[k] = active ? 0u : kSent * 0x10001u;
  uint32_t mm = 0;

  // copies step s into its ring slot (s % KS) and moves the copy pointer on
  auto copy_step = [&](int s) {
    if (active && s < g.len) {
#pragma unroll
      for (int v = 0; v < NV; v++)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         sbase + (uint32_t)((((s % KS) * NV + v) * 32 + lane) * 16)),
                     "l"(cp + v * cvs));
      if (s + 1 < g.len) cp += estride;
    }
  };
  // prologue: steps 0 .. 5 in flight as three groups of two
#pragma unroll
  for (int s = 0; s < KS - 2; s += 2) {
    copy_step(s);
    copy_step(s + 1);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int t0 = 0; t0 < maxlen; t0 += KS) {
#pragma unroll
    for (int u = 0; u < KS; u++) {
      const int t = t0 + u;
      if (t >= maxlen) break;
      if ((u & 1) == 0) {  // issue steps t + 6, t + 7, then wait for steps t, t + 1
        copy_step(t + KS - 2);
        copy_step(t + KS - 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 3;" ::: "memory");
      }
      uint32_t c[NP];
#pragma unroll
      for (int v = 0; v < NV; v++) {
        const uint4 r = ring[(u * NV + v) * 32 + lane];
        unpack4(r.x, c[8 * v + 0], c[8 * v + 1]);
        unpack4(r.y, c[8 * v + 2], c[8 * v + 3]);
        unpack4(r.z, c[8 * v + 4], c[8 * v + 5]);
        unpack4(r.w, c[8 * v + 6], c[8 * v + 7]);
      }
      uint32_t X[NP + 1];
      neighbours<NP, WD>(L, lig, X);
      const uint32_t mP2 = mm + P2P2;
      uint32_t lmin = 0xFFFFFFFFu;
#pragma unroll
      for (int k = 0; k < NP; k++) {
        const uint32_t tt = vmin2(X[k], X[k + 1]) + P1P1;
        const uint32_t uu = vmin2(vmin2(L[k], tt), mP2);  // >= m(q) in both halves
        const uint32_t ln = uu + c[k] - mm;                // each half in [0, 255 + P2]
        L[k] = (FULL || active) ? ln : kSent * 0x10001u;
        lmin = vmin2(lmin, L[k]);
      }
      mm = group_min<WD>(halves_min(lmin));
      if (active && t < g.len) {
#pragma unroll
        for (int k = 0; k < NP / 2; k++) add4<WIDE>(pb.agg, e + k * svs, L[2 * k], L[2 * k + 1]);
      }
      e += estride;
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

}  // namespace r2t
