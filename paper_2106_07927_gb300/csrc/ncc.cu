// Second matching cost of the method: the inverted, truncated normalised cross-correlation
// (Sec. 2.1.1: s = 1 - max(0, Phi); Sec. 2.2.1: patch statistics precomputed per pixel, then the
// matching), over n x n patches (n = 5 or 9) with the zero-valued margin of the census.
//
// For the reference patch a (around x) and the matching patch b (around x - d), N = n^2:
//   vA = N sum a^2 - (sum a)^2,  vB likewise,  cov = N sum a b - sum a sum b   (exact integers)
//   Phi = cov / sqrt(vA vB)  (0 when vA or vB is 0)
// and the 8-bit cost 255 - k with k = round(255 max(0, Phi)), ties to even. k is a function of
// the three integers alone. The kernel estimates x = 255 Phi in fp32 (iA = 1 / sqrt(vA),
// jB = 255 / sqrt(vB) per pixel, q = (cov iA) jB, each correctly rounded): the relative error of q
// is at most about 9 * 2^-24, under 1.4e-4 absolute for x <= 255. Where q lies farther than
// 1/1024 from the nearest k + 1/2, rint(q) is k. Closer to a boundary the boundary f + 1/2
// (f = floor q) is settled on integers: x > f + 1/2 <=> (510 cov)^2 > (2f + 1)^2 vA vB (128-bit
// products), equality being a tie that goes to the even one of f and f + 1. A cov <= 0 gives 255.
//
// ncc_stats_kernel: per pixel, the patch sum and the factor (iA for the reference image, jB for
// the matching one), as one 8-byte pair, and the exact variance v.
// ncc_cost_kernel: a band of kNccTY rows x TX pixels x all D per block of 256 threads; thread
// (x, g) owns disparities 4g .. 4g + 3 of pixel x. Down the band it forms, per image row, the
// dot products of the patch rows (dp4a over byte words realigned from shared memory) and keeps
// the last n of them in a register ring, so sum a b over the patch costs one row of work per
// output row instead of n. It also clears the tile's aggregated sums and right-disparity keys,
// as the census cost kernel does.
#include <algorithm>

#include "launch.h"

namespace r2t {

namespace {

constexpr int kNccTY = 32;                        // output rows per block
constexpr int kNccMaxRows = kNccTY + 8;           // staged rows, n <= 9
constexpr int kNccLStride = 80;                   // >= TX + 2r + 8 for TX <= 64
constexpr int kNccRStride = 288;                  // >= TX + D - 1 + 2r + 3 + 8 for D <= 256

__host__ __device__ inline int ncc_tx(int D) { return 256 / (D / 4); }  // pixels per block

// Patch sum and factor of every pixel of one image (blocks of 32 x 8): {sum a, bits of f} with
// f = 1 / sqrt(float(vA)) (reference image) or 255 / ... as fl(255 * f) (matching image, scale255).
template <int N_>
__global__ void __launch_bounds__(256) ncc_stats_kernel(const uint8_t* img, int64_t pitch, int W,
                                                        int H, uint2* st, int32_t* sv,
                                                        bool scale255) {
  constexpr int R = N_ / 2, TW = 32 + 2 * R;
  __shared__ uint8_t t[8 + 2 * R][TW];
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8;
  for (int ty = 0; ty < 8 + 2 * R; ty++)
    for (int tx = threadIdx.x; tx < TW; tx += 256) {
      const int gx = x0 + tx - R, gy = y0 + ty - R;
      t[ty][tx] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? img[(int64_t)gy * pitch + gx] : 0;
    }
  __syncthreads();
  const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
  const int x = x0 + lx, y = y0 + ly;
  if (x >= W || y >= H) return;
  int s1 = 0, s2 = 0;
#pragma unroll
  for (int j = 0; j < N_; j++)
#pragma unroll
    for (int i = 0; i < N_; i++) {
      const int v = t[ly + j][lx + i];
      s1 += v;
      s2 += v * v;
    }
  const int v = N_ * N_ * s2 - s1 * s1;  // <= N^2 255^2 / 4 < 2^27
  float f = v > 0 ? __fdiv_rn(1.0f, __fsqrt_rn(__int2float_rn(v))) : 0.0f;
  if (scale255) f = __fmul_rn(255.0f, f);
  st[(int64_t)y * W + x] = make_uint2((uint32_t)s1, __float_as_uint(f));
  sv[(int64_t)y * W + x] = v;
}

// Half-width of the band around k + 1/2 inside which the rounding is settled on integers; the
// fp32 estimate is within 1.4e-4 of 255 Phi.
constexpr float kNccTieBand = 1.0f / 1024.0f;

// k = round(255 Phi) for cov > 0 when the estimate q lies within kNccTieBand of f + 1/2,
// f = floor(q): the true value lies on one side of f + 1/2, found from
// (510 cov)^2 vs (2f + 1)^2 vA vB (both < 2^72, compared as 128-bit unsigned); equal is a tie.
__device__ __noinline__ uint32_t ncc_exact_k(int cov, int va, int vb, float q) {
  const int f = (int)floorf(q);
  const unsigned long long a = 510ull * (unsigned long long)cov;  // < 2^36
  const unsigned long long tl = a * a, th = __umul64hi(a, a);
  const unsigned long long r =
      (unsigned long long)(2 * f + 1) * (unsigned long long)(2 * f + 1) * (unsigned long long)va;
  const unsigned long long rl = r * (unsigned long long)vb;
  const unsigned long long rh = __umul64hi(r, (unsigned long long)vb);
  int k;
  if (th > rh || (th == rh && tl > rl))
    k = f + 1;  // above the boundary
  else if (th < rh || tl < rl)
    k = f;      // below it
  else
    k = (f & 1) ? f + 1 : f;  // on it: the even neighbour
  return (uint32_t)min(k, 255);
}

// The fp32 estimate q = (cov * iA) * jB of 255 Phi for one patch pair from its sums (cov is
// returned too).
__device__ __forceinline__ float ncc_estimate(int nn, int sab, int sa, float ia, uint2 mb,
                                              int& cov) {
  cov = nn * sab - sa * (int)mb.x;  // |cov| < 2^27
  return __fmul_rn(__fmul_rn(__int2float_rn(cov), ia), __uint_as_float(mb.y));
}

// k = rint(q) clamped to 0 .. 255.
__device__ __forceinline__ uint32_t ncc_round(float q) {
  uint32_t k;
  asm("cvt.rni.sat.u8.f32 %0, %1;" : "=r"(k) : "f"(q));
  return k;
}

template <int N_>
__global__ void __launch_bounds__(256, N_ == 5 ? 4 : 3)
    ncc_cost_kernel(Problem pb, int agg_bytes_per_de, const uint2* st, const int32_t* sv) {
  constexpr int R = N_ / 2;
  constexpr int NW = (N_ + 3) / 4;  // dot-product words of a patch row
  __shared__ __align__(16) uint8_t sl[kNccMaxRows][kNccLStride];
  __shared__ __align__(16) uint8_t sr[kNccMaxRows][kNccRStride];
  extern __shared__ __align__(16) uint8_t sst_ring[];  // 9 x 9: N_ x 256 x 16 bytes of ring
  const int W = pb.W, H = pb.H, D = pb.D;
  const int TX = ncc_tx(D), G = D / 4;
  const int ntx = (W + TX - 1) / TX;
  const int x0 = (blockIdx.x % ntx) * TX, y0 = (blockIdx.x / ntx) * kNccTY;
  const int nrows = min(kNccTY, H - y0) + 2 * R;  // staged rows y0 - R .. y0 + ny - 1 + R
  const int lbase = x0 - R;                       // image column of sl[.][0]
  const int rbase = x0 - (D - 1) - R - 3;         // image column of sr[.][0]
  const int lw = TX + 2 * R + 8, rw = TX + D - 1 + 2 * R + 3 + 8;
  // staged columns c < lw are the left segment, c >= lw the right one (lw + rw <= 2 * 256)
  for (int r0 = 0; r0 < nrows; r0 += 4) {
    uint8_t v[4][2];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int gy = y0 - R + r0 + u;
      const bool rowin = r0 + u < nrows && gy >= 0 && gy < H;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int c = threadIdx.x + 256 * h;
        const bool isr = c >= lw;
        const int gx = isr ? rbase + (c - lw) : lbase + c;
        v[u][h] = 0;
        if (rowin && c < lw + rw && gx >= 0 && gx < W)
          v[u][h] = __ldg((isr ? pb.right : pb.left) + (int64_t)gy * pb.in_pitch + gx);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int c = threadIdx.x + 256 * h;
        if (r0 + u < nrows && c < lw + rw) {
          if (c >= lw)
            sr[r0 + u][c - lw] = v[u][h];
          else
            sl[r0 + u][c] = v[u][h];
        }
      }
  }
  __syncthreads();

  // clear the aggregated sums and reset the right-disparity keys of the tile's pixels: per row
  // one contiguous run of nx pixels (16-byte pieces, D % 16 == 0)
  {
    const int ny = min(kNccTY, H - y0), nx = min(TX, W - x0);
    const int pieces = nx * D * agg_bytes_per_de / 16;
    for (int row = 0; row < ny; row++) {
      const int64_t p = (int64_t)(y0 + row) * W + x0;
      uint4* z = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(pb.agg) +
                                          p * D * agg_bytes_per_de);
      for (int i = threadIdx.x; i < pieces; i += 256) z[i] = make_uint4(0, 0, 0, 0);
      if (threadIdx.x < nx) pb.kr[p + threadIdx.x] = 0xFFFFFFFFu;
    }
  }
  const int g = threadIdx.x % G, xl = threadIdx.x / G;
  const int x = x0 + xl;
  if (xl >= TX || x >= W) return;  // no barrier follows
  const int nn = N_ * N_;
  const int64_t npx = (int64_t)W * H;
  // this thread's windows: left bytes [xl, xl + N_) of sl; right bytes [s0, s0 + N_ + 3) of sr
  // hold the windows of d = 4g + 3, 4g + 2, 4g + 1, 4g (d = 4g + k starts at s0 + 3 - k)
  const int s0 = xl + D - 1 - 4 * g;
  const int lsh = 8 * (xl & 3), rsh = 8 * (s0 & 3);
  const uint32_t lmask = (N_ % 4) ? (0xFFFFFFFFu >> (8 * (4 - N_ % 4))) : 0xFFFFFFFFu;
  const uint32_t* lrow = reinterpret_cast<const uint32_t*>(&sl[0][xl & ~3]);
  const uint32_t* rrow = reinterpret_cast<const uint32_t*>(&sr[0][s0 & ~3]);
  // statistics: the reference pixel, and the matching pixels x - 4g - k (k = 0 .. 3); the
  // buffer has 256 entries of slack in front, so x - 4g - k < 0 still reads inside it
  // (pointer of the next output row, advanced by one image row per output row)
  const uint2* sa_p = st + (int64_t)y0 * W + x;
  const int64_t mo = npx - 4 * g;  // matching pixel x - 4g, same row
  uint32_t* out = reinterpret_cast<uint32_t*>(pb.cost + ((int64_t)y0 * W + x) * D) + g;
  const int out_row = W * D / 4;  // uint32 words per image row
  bool inside[4];                 // x - d >= 0 for d = 4g + k
#pragma unroll
  for (int k = 0; k < 4; k++) inside[k] = x - 4 * g - k >= 0;
  // The last N_ rows' dot products: in registers for 5 x 5; in shared memory for 9 x 9 (slot j of
  // this thread at sring[j * 256 + thread], 16 bytes), which keeps the 9 x 9 kernel's registers
  // low enough for more resident blocks.
  constexpr bool RSM = N_ > 5;
  int ring[RSM ? 1 : N_][4];
  int4* sring = reinterpret_cast<int4*>(sst_ring);
  int vs[4] = {0, 0, 0, 0};
#pragma unroll
  for (int j = 0; j < (RSM ? 1 : N_); j++)
#pragma unroll
    for (int k = 0; k < 4; k++) ring[j][k] = 0;
  if (RSM) {
#pragma unroll
    for (int j = 0; j < N_; j++) sring[j * 256 + threadIdx.x] = make_int4(0, 0, 0, 0);
  }

  // one staged row t: its four row dot products enter the ring (slot j = t mod N_); from
  // t = 2R on, the patch of output row t - 2R is complete and its costs are written
  auto row_step = [&](int t, int j) {
    uint32_t lwd[NW], rwd[NW + 1];
    {
      uint32_t raw[NW + 1];
#pragma unroll
      for (int m = 0; m <= NW; m++) raw[m] = lrow[t * (kNccLStride / 4) + m];
#pragma unroll
      for (int m = 0; m < NW; m++) lwd[m] = __funnelshift_r(raw[m], raw[m + 1], lsh);
      lwd[NW - 1] &= lmask;
    }
    {
      uint32_t raw[NW + 2];
#pragma unroll
      for (int m = 0; m <= NW + 1; m++) raw[m] = rrow[t * (kNccRStride / 4) + m];
#pragma unroll
      for (int m = 0; m <= NW; m++) rwd[m] = __funnelshift_r(raw[m], raw[m + 1], rsh);
    }
    int h[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int o = 3 - k;  // byte offset of the window of d = 4g + k
      uint32_t a = 0;
#pragma unroll
      for (int m = 0; m < NW; m++)
        a = __dp4a(lwd[m], o ? __funnelshift_r(rwd[m], rwd[m + 1], 8 * o) : rwd[m], a);
      h[k] = (int)a;
    }
    if (RSM) {
      int4* slot = &sring[j * 256 + threadIdx.x];
      const int4 old = *slot;
      *slot = make_int4(h[0], h[1], h[2], h[3]);
      vs[0] += h[0] - old.x;
      vs[1] += h[1] - old.y;
      vs[2] += h[2] - old.z;
      vs[3] += h[3] - old.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; k++) {
        vs[k] += h[k] - ring[RSM ? 0 : j][k];
        ring[RSM ? 0 : j][k] = h[k];
      }
    }
    if (t >= 2 * R) {  // output row y0 + t - 2R
      const uint2 a = *sa_p;
      const uint2* mb = sa_p + mo;
      float q[4];
      int cov[4];
      uint32_t c[4];
      float far = 0.0f;  // the largest distance of a q from its rounded value
#pragma unroll
      for (int k = 0; k < 4; k++) {
        q[k] = ncc_estimate(nn, vs[k], (int)a.x, __uint_as_float(a.y), mb[-k], cov[k]);
        c[k] = 255u - ncc_round(q[k]);
        far = fmaxf(far, fabsf(q[k] - rintf(q[k])));
      }
      if (far > 0.5f - kNccTieBand) {  // some q near a k + 1/2 boundary: settle it on integers
        const int32_t* va = sv + (sa_p - st);  // exact variances, same indexing as the stats
#pragma unroll
        for (int k = 0; k < 4; k++)
          if (inside[k] && cov[k] > 0 && fabsf(q[k] - rintf(q[k])) > 0.5f - kNccTieBand)
            c[k] = 255u - ncc_exact_k(cov[k], *va, va[mo - k], q[k]);
      }
#pragma unroll
      for (int k = 0; k < 4; k++) c[k] = inside[k] ? c[k] : (uint32_t)kCostOutside;
      *out = c[0] | (c[1] << 8) | (c[2] << 16) | (c[3] << 24);
      sa_p += W;
      out += out_row;
    }
  };
  int t0 = 0;
  for (; t0 + N_ <= nrows; t0 += N_) {
#pragma unroll
    for (int j = 0; j < N_; j++) row_step(t0 + j, j);
  }
#pragma unroll
  for (int j = 0; j < N_; j++)
    if (t0 + j < nrows) row_step(t0 + j, j);
}

template <int N_>
cudaError_t launch_ncc_n(const Problem& pb, const Method& mt, cudaStream_t s) {
  const int64_t npx = (int64_t)pb.W * pb.H;
  const dim3 sg((pb.W + 31) / 32, (pb.H + 7) / 8);
  ncc_stats_kernel<N_><<<sg, 256, 0, s>>>(pb.left, pb.in_pitch, pb.W, pb.H, pb.nst, pb.nsv,
                                          false);
  ncc_stats_kernel<N_><<<sg, 256, 0, s>>>(pb.right, pb.in_pitch, pb.W, pb.H, pb.nst + npx,
                                          pb.nsv + npx, true);
  const int TX = ncc_tx(pb.D);
  const int blocks = ((pb.W + TX - 1) / TX) * ((pb.H + kNccTY - 1) / kNccTY);
  const int ring_smem = N_ > 5 ? N_ * 256 * 16 : 0;
  if (ring_smem)
    cudaFuncSetAttribute(ncc_cost_kernel<N_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         ring_smem);
  ncc_cost_kernel<N_><<<blocks, 256, ring_smem, s>>>(pb, mt.wide ? 4 : 2, pb.nst, pb.nsv);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ncc_cost(const Problem& pb, const Method& mt, cudaStream_t s) {
  if (!pb.nst || !pb.nsv || pb.D % 16 != 0 || pb.D > 256) return cudaErrorInvalidValue;
  if (mt.cw == 5) return launch_ncc_n<5>(pb, mt, s);
  if (mt.cw == 9) return launch_ncc_n<9>(pb, mt, s);
  return cudaErrorInvalidValue;
}

}  // namespace r2t
