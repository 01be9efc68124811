// Rectification (Sec. 2.1.1: the pair is resampled through two maps from the calibration so that
// epipolar lines lie on image rows), the step before the census. For every output pixel the map
// gives the source coordinate (mx, my) in the raw image; it is put on a 1/32-pixel grid,
// X = rint(32 mx), Y = rint(32 my) (the product by 32 is exact in float), and the output is the
// bilinear interpolation with integer weights that sum to 1024, rounded:
//   (I(x0,y0)(32-fx)(32-fy) + I(x0+1,y0) fx (32-fy) + I(x0,y0+1)(32-fx) fy + I(x0+1,y0+1) fx fy
//    + 512) >> 10,   x0 = floor(X / 32), fx = X - 32 x0 (y likewise),
// with samples outside the raw image reading 0; a coordinate that is not finite or has
// |32 m| >= 2^24 gives 0. Integer arithmetic after the grid step, so the result is exact.
//
// One thread per output pixel, both images of a pair in one launch (blockIdx.y). The maps are
// read once (coalesced, 8 B per pixel); the four source bytes come through the L1 cache, since
// neighbouring outputs sample neighbouring sources.
#include <algorithm>

#include "launch.h"

namespace r2t {

namespace {

__device__ __forceinline__ int raw_at(const uint8_t* raw, int64_t pitch, int rw, int rh, int x,
                                      int y) {
  return (x >= 0 && x < rw && y >= 0 && y < rh) ? (int)__ldg(raw + (int64_t)y * pitch + x) : 0;
}

__global__ void __launch_bounds__(256) rectify_kernel(RectifyJob j0, RectifyJob j1) {
  const RectifyJob& j = blockIdx.y == 0 ? j0 : j1;
  const int64_t n = (int64_t)j.W * j.H;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(i / j.W), x = (int)(i - (int64_t)y * j.W);
    const float sx = __fmul_rn(
        __ldg(reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(j.mapx) +
                                             (int64_t)y * j.map_pitch) + x), 32.0f);
    const float sy = __fmul_rn(
        __ldg(reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(j.mapy) +
                                             (int64_t)y * j.map_pitch) + x), 32.0f);
    int v = 0;
    if (fabsf(sx) < 16777216.0f && fabsf(sy) < 16777216.0f) {  // false for NaN and infinity
      const int X = __float2int_rn(sx), Y = __float2int_rn(sy);
      const int x0 = X >> 5, y0 = Y >> 5;  // floor(X / 32): arithmetic shift
      const int fx = X & 31, fy = Y & 31;
      const int p00 = raw_at(j.raw, j.raw_pitch, j.rw, j.rh, x0, y0);
      const int p10 = raw_at(j.raw, j.raw_pitch, j.rw, j.rh, x0 + 1, y0);
      const int p01 = raw_at(j.raw, j.raw_pitch, j.rw, j.rh, x0, y0 + 1);
      const int p11 = raw_at(j.raw, j.raw_pitch, j.rw, j.rh, x0 + 1, y0 + 1);
      v = (p00 * (32 - fx) * (32 - fy) + p10 * fx * (32 - fy) + p01 * (32 - fx) * fy +
           p11 * fx * fy + 512) >> 10;
    }
    j.out[(int64_t)y * j.out_pitch + x] = (uint8_t)v;
  }
}

}  // namespace

cudaError_t launch_rectify(const RectifyJob* jobs, int n, cudaStream_t s) {
  if (n < 1 || n > 2) return cudaErrorInvalidValue;
  int64_t most = 0;
  for (int i = 0; i < n; i++) most = std::max<int64_t>(most, (int64_t)jobs[i].W * jobs[i].H);
  const int grid = (int)std::min<int64_t>((most + 255) / 256, 152 * 8);
  rectify_kernel<<<dim3(grid, n), 256, 0, s>>>(jobs[0], jobs[n - 1]);
  return cudaGetLastError();
}

}  // namespace r2t
