// Second matching cost of the method: the inverted, truncated normalised cross-correlation
// (Sec. 2.1.1: s = 1 - max(0, Phi); Sec. 2.2.1: patch statistics precomputed per pixel, then the
// matching), over n x n patches (n = 5 or 9) with the zero-valued margin of the census.
//
// For the reference patch a (around x) and the matching patch b (around x - d), N = n^2:
//   vA = N sum a^2 - (sum a)^2,  vB likewise,  cov = N sum a b - sum a sum b   (exact integers)
//   Phi = cov / sqrt(vA vB)  (0 when vA or vB is 0)
// and the 8-bit cost 255 - clamp(rint(255 max(0, Phi)), 0, 255), scaled in a fixed sequence of
// correctly rounded fp32 operations: iA = 1 / sqrt(float(vA)) (0 when vA = 0), iB likewise,
// q = ((float(cov) * iA) * iB) * 255, cost = 255 - clamp(rint(q), 0, 255). A cov <= 0 gives 255.
//
// ncc_stats_kernel: per pixel of both images, sum a over the patch and iA.
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

// Sum a and 1 / sqrt(vA) of the n x n patch around every pixel of one image (blocks of 32 x 8).
template <int N_>
__global__ void __launch_bounds__(256) ncc_stats_kernel(const uint8_t* img, int64_t pitch, int W,
                                                        int H, int32_t* sum, float* inv) {
  constexpr int R = N_ / 2;
  __shared__ uint8_t t[8 + 2 * R][32 + 2 * R];
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8;
  for (int i = threadIdx.x; i < (8 + 2 * R) * (32 + 2 * R); i += 256) {
    const int ty = i / (32 + 2 * R), tx = i % (32 + 2 * R);
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
  const int64_t p = (int64_t)y * W + x;
  sum[p] = s1;
  inv[p] = v > 0 ? __fdiv_rn(1.0f, __fsqrt_rn(__int2float_rn(v))) : 0.0f;
}

// The 8-bit cost of one patch pair from its sums.
__device__ __forceinline__ uint32_t ncc_cost_of(int nn, int sab, int sa, int sb, float ia,
                                                float ib) {
  const int cov = nn * sab - sa * sb;  // |cov| < 2^29
  float q = __fmul_rn(__int2float_rn(cov), ia);
  q = __fmul_rn(q, ib);
  q = __fmul_rn(q, 255.0f);
  const int k = min(max(__float2int_rn(q), 0), 255);
  return (uint32_t)(255 - k);
}

template <int N_>
__global__ void __launch_bounds__(256) ncc_cost_kernel(Problem pb, int agg_bytes_per_de,
                                                       const int32_t* sum, const float* inv) {
  constexpr int R = N_ / 2;
  constexpr int NW = (N_ + 3) / 4;  // dot-product words of a patch row
  __shared__ __align__(16) uint8_t sl[kNccMaxRows][kNccLStride];
  __shared__ __align__(16) uint8_t sr[kNccMaxRows][kNccRStride];
  const int W = pb.W, H = pb.H, D = pb.D;
  const int TX = ncc_tx(D), G = D / 4;
  const int ntx = (W + TX - 1) / TX;
  const int x0 = (blockIdx.x % ntx) * TX, y0 = (blockIdx.x / ntx) * kNccTY;
  const int nrows = min(kNccTY, H - y0) + 2 * R;  // staged rows y0 - R .. y0 + ny - 1 + R
  const int lbase = x0 - R;                       // image column of sl[.][0]
  const int rbase = x0 - (D - 1) - R - 3;         // image column of sr[.][0]
  const int lw = TX + 2 * R + 8, rw = TX + D - 1 + 2 * R + 3 + 8;
  for (int i = threadIdx.x; i < nrows * (lw + rw); i += 256) {
    const int row = i / (lw + rw), c = i % (lw + rw);
    const int gy = y0 - R + row;
    const bool isr = c >= lw;
    const int gx = isr ? rbase + (c - lw) : lbase + c;
    uint8_t v = 0;
    if (gy >= 0 && gy < H && gx >= 0 && gx < W)
      v = (isr ? pb.right : pb.left)[(int64_t)gy * pb.in_pitch + gx];
    if (isr)
      sr[row][c - lw] = v;
    else
      sl[row][c] = v;
  }
  __syncthreads();

  const int g = threadIdx.x % G, xl = threadIdx.x / G;
  const int x = x0 + xl;
  const bool active = xl < TX && x < W;
  const int nn = N_ * N_;
  // this thread's windows: left bytes [xl, xl + N_) of sl; right bytes [s0, s0 + N_ + 3) of sr
  // hold the windows of d = 4g + 3, 4g + 2, 4g + 1, 4g (d = 4g + k starts at s0 + 3 - k)
  const int s0 = xl + D - 1 - 4 * g;
  const uint32_t lmask = (N_ % 4) ? (0xFFFFFFFFu >> (8 * (4 - N_ % 4))) : 0xFFFFFFFFu;
  int ring[N_][4];
  int vs[4] = {0, 0, 0, 0};
#pragma unroll
  for (int j = 0; j < N_; j++)
#pragma unroll
    for (int k = 0; k < 4; k++) ring[j][k] = 0;

  for (int t0 = 0; t0 < nrows; t0 += N_) {
#pragma unroll
    for (int j = 0; j < N_; j++) {
      const int t = t0 + j;  // staged row
      if (t < nrows && active) {
        // left words, realigned to start at xl
        uint32_t lwd[NW];
        {
          const uint32_t* p = reinterpret_cast<const uint32_t*>(&sl[t][xl & ~3]);
          uint32_t raw[NW + 1];
#pragma unroll
          for (int m = 0; m <= NW; m++) raw[m] = p[m];
#pragma unroll
          for (int m = 0; m < NW; m++) lwd[m] = __funnelshift_r(raw[m], raw[m + 1], 8 * (xl & 3));
          lwd[NW - 1] &= lmask;
        }
        // right words, realigned to start at s0
        uint32_t rwd[NW + 1];
        {
          const uint32_t* p = reinterpret_cast<const uint32_t*>(&sr[t][s0 & ~3]);
          uint32_t raw[NW + 2];
#pragma unroll
          for (int m = 0; m <= NW + 1; m++) raw[m] = p[m];
#pragma unroll
          for (int m = 0; m <= NW; m++) rwd[m] = __funnelshift_r(raw[m], raw[m + 1], 8 * (s0 & 3));
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const int o = 3 - k;  // byte offset of the window of d = 4g + k
          uint32_t h = 0;
#pragma unroll
          for (int m = 0; m < NW; m++)
            h = __dp4a(lwd[m], o ? __funnelshift_r(rwd[m], rwd[m + 1], 8 * o) : rwd[m], h);
          vs[k] += (int)h - ring[j][k];
          ring[j][k] = (int)h;
        }
      }
      if (t < nrows && t >= 2 * R && active) {
        const int y = y0 + t - 2 * R;  // the patch rows y - R .. y + R are all in the ring
        const int64_t p = (int64_t)y * W + x;
        const int sa = sum[p];
        const float ia = inv[p];
        uint32_t c[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const int d = 4 * g + k;
          c[k] = kCostOutside;
          if (x - d >= 0) {
            const int64_t q = p - d + (int64_t)W * H;  // matching image's statistics
            c[k] = ncc_cost_of(nn, vs[k], sa, sum[q], ia, inv[q]);
          }
        }
        reinterpret_cast<uint32_t*>(pb.cost + p * D)[g] =
            c[0] | (c[1] << 8) | (c[2] << 16) | (c[3] << 24);
      }
    }
  }
  // clear the aggregated sums and reset the right-disparity keys of the tile's pixels
  const int ny = min(kNccTY, H - y0), nx = min(TX, W - x0);
  const int per_px = D * agg_bytes_per_de / 16;  // 16-byte pieces per pixel (D % 16 == 0)
  for (int i = threadIdx.x; i < ny * nx * per_px; i += 256) {
    const int piece = i % per_px, pxi = i / per_px;
    const int64_t p = (int64_t)(y0 + pxi / nx) * W + x0 + pxi % nx;
    reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(pb.agg) + p * D * agg_bytes_per_de)[piece] =
        make_uint4(0, 0, 0, 0);
  }
  for (int i = threadIdx.x; i < ny * nx; i += 256)
    pb.kr[(int64_t)(y0 + i / nx) * W + x0 + i % nx] = 0xFFFFFFFFu;
}

template <int N_>
cudaError_t launch_ncc_n(const Problem& pb, const Method& mt, cudaStream_t s) {
  const int64_t npx = (int64_t)pb.W * pb.H;
  const dim3 sg((pb.W + 31) / 32, (pb.H + 7) / 8);
  ncc_stats_kernel<N_><<<sg, 256, 0, s>>>(pb.left, pb.in_pitch, pb.W, pb.H, pb.nsum, pb.ninv);
  ncc_stats_kernel<N_><<<sg, 256, 0, s>>>(pb.right, pb.in_pitch, pb.W, pb.H, pb.nsum + npx,
                                          pb.ninv + npx);
  const int TX = ncc_tx(pb.D);
  const int blocks = ((pb.W + TX - 1) / TX) * ((pb.H + kNccTY - 1) / kNccTY);
  ncc_cost_kernel<N_><<<blocks, 256, 0, s>>>(pb, mt.wide ? 4 : 2, pb.nsum, pb.ninv);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ncc_cost(const Problem& pb, const Method& mt, cudaStream_t s) {
  if (!pb.nsum || !pb.ninv || pb.D % 16 != 0 || pb.D > 256) return cudaErrorInvalidValue;
  if (mt.cw == 5) return launch_ncc_n<5>(pb, mt, s);
  if (mt.cw == 9) return launch_ncc_n<9>(pb, mt, s);
  return cudaErrorInvalidValue;
}

}  // namespace r2t
