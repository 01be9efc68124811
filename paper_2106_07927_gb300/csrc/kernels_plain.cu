// Plain single-pair launches of the SGM stages (one kernel per stage, all on the caller's stream).
#include "aggregate.cuh"
#include "census_cost.cuh"
#include "launch.h"
#include "post.cuh"

namespace r2t {

__global__ void __launch_bounds__(256) census_kernel(Problem pb, Method mt) {
  __shared__ CensusSmem sm;
  census_tile_dispatch(pb, mt, blockIdx.x, sm);
}

__global__ void __launch_bounds__(256) cost_kernel(Problem pb, int agg_bytes_per_de) {
  __shared__ CostSmem sm;
  cost_tile(pb, blockIdx.x, sm, agg_bytes_per_de);
}

template <int DPL, int LPL, bool WIDE>
__global__ void __launch_bounds__(512) aggregate_kernel(Problem pb, Method mt) {
  const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  agg_warp_lines<DPL, LPL, WIDE>(pb, mt, warp * (32 / LPL), 0x7FFFFFFF);
}

template <bool WIDE>
__global__ void __launch_bounds__(256) wta_lr_kernel(Problem pb, Method mt, int T) {
  extern __shared__ __align__(16) uint16_t wsm[];
  const int y = blockIdx.x;
  uint16_t* out_row = (mt.flags & 2) ? pb.dlr + (int64_t)y * pb.W
                                     : reinterpret_cast<uint16_t*>(
                                           reinterpret_cast<uint8_t*>(pb.disp) + y * pb.out_pitch);
  wta_lr_row<WIDE>(pb, mt, y, T, wsm, out_row);
}

__global__ void __launch_bounds__(256) median_kernel(Problem pb) {
  __shared__ MedianSmem sm;
  median_tile(pb.dlr, pb.W, pb.W, pb.H, pb.disp, pb.out_pitch, blockIdx.x, sm);
}

__global__ void agg_to_u16_kernel(const uint32_t* src, uint16_t* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (uint16_t)min(src[i], 65535u);
}

Tuning default_tuning(int D) {
  Tuning t;
  t.agg_dpl = D <= 64 ? 2 : (D <= 128 ? 4 : 8);
  t.agg_warps = 4;
  t.wta_chunk = wta_default_chunk(D);
  return t;
}

bool tuning_valid(const Tuning& t, int D) {
  if (t.agg_dpl != 2 && t.agg_dpl != 4 && t.agg_dpl != 8) return false;
  if (D % t.agg_dpl != 0) return false;
  if ((D + t.agg_dpl - 1) / t.agg_dpl > 32) return false;
  if (t.agg_warps < 1 || t.agg_warps > 16) return false;
  if (t.wta_chunk < 32 || t.wta_chunk > 256 || t.wta_chunk % 32 != 0) return false;
  if (wta_smem_bytes(D, t.wta_chunk) > 200 * 1024) return false;
  return true;
}

template <int DPL, int LPL, bool WIDE>
static cudaError_t launch_agg_t(const Problem& pb, const Method& mt, int warps, cudaStream_t s) {
  const int nl = agg_num_lines(pb.W, pb.H, mt.num_paths);
  const int lines_per_warp = 32 / LPL;
  const int nwarp = (nl + lines_per_warp - 1) / lines_per_warp;
  const int grid = (nwarp + warps - 1) / warps;
  aggregate_kernel<DPL, LPL, WIDE><<<grid, warps * 32, 0, s>>>(pb, mt);
  return cudaGetLastError();
}

template <bool WIDE>
static cudaError_t launch_agg_w(const Problem& pb, const Method& mt, const Tuning& tn,
                                cudaStream_t s) {
  const int lpl = agg_lanes_for(pb.D, tn.agg_dpl);
  switch (tn.agg_dpl * 100 + lpl) {
    case 208: return launch_agg_t<2, 8, WIDE>(pb, mt, tn.agg_warps, s);
    case 216: return launch_agg_t<2, 16, WIDE>(pb, mt, tn.agg_warps, s);
    case 232: return launch_agg_t<2, 32, WIDE>(pb, mt, tn.agg_warps, s);
    case 408: return launch_agg_t<4, 8, WIDE>(pb, mt, tn.agg_warps, s);
    case 416: return launch_agg_t<4, 16, WIDE>(pb, mt, tn.agg_warps, s);
    case 432: return launch_agg_t<4, 32, WIDE>(pb, mt, tn.agg_warps, s);
    case 808: return launch_agg_t<8, 8, WIDE>(pb, mt, tn.agg_warps, s);
    case 816: return launch_agg_t<8, 16, WIDE>(pb, mt, tn.agg_warps, s);
    case 832: return launch_agg_t<8, 32, WIDE>(pb, mt, tn.agg_warps, s);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t launch_aggregate(const Problem& pb, const Method& mt, const Tuning& tn,
                                    cudaStream_t s) {
  return mt.wide ? launch_agg_w<true>(pb, mt, tn, s) : launch_agg_w<false>(pb, mt, tn, s);
}

cudaError_t run_pipeline(const Problem& pb, const Method& mt, const Tuning& tn, cudaStream_t s,
                         int* launches, cudaEvent_t* ev) {
  int n = 0;
  cudaError_t e;
  if (ev) cudaEventRecord(ev[0], s);
  census_kernel<<<census_items(pb.W, pb.H), 256, 0, s>>>(pb, mt);
  n++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[1], s);
  cost_kernel<<<cost_items(pb.W, pb.H), 256, 0, s>>>(pb, mt.wide ? 4 : 2);
  n++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[2], s);
  if ((e = launch_aggregate(pb, mt, tn, s)) != cudaSuccess) return e;
  n++;
  if (ev) cudaEventRecord(ev[3], s);
  const size_t smem = wta_smem_bytes(pb.D, tn.wta_chunk);
  if (mt.wide) {
    cudaFuncSetAttribute(wta_lr_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    wta_lr_kernel<true><<<pb.H, 256, smem, s>>>(pb, mt, tn.wta_chunk);
  } else {
    cudaFuncSetAttribute(wta_lr_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    wta_lr_kernel<false><<<pb.H, 256, smem, s>>>(pb, mt, tn.wta_chunk);
  }
  n++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[4], s);
  if (mt.flags & 2) {
    median_kernel<<<median_items(pb.W, pb.H), 256, 0, s>>>(pb);
    n++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (ev) cudaEventRecord(ev[5], s);
  if (launches) *launches = n;
  return cudaSuccess;
}

cudaError_t copy_agg_u16(const Problem& pb, bool wide, uint16_t* dst, cudaStream_t s) {
  const int64_t nde = (int64_t)pb.W * pb.H * pb.D;
  if (!wide) return cudaMemcpyAsync(dst, pb.agg, (size_t)nde * 2, cudaMemcpyDeviceToDevice, s);
  agg_to_u16_kernel<<<1216, 256, 0, s>>>(reinterpret_cast<const uint32_t*>(pb.agg), dst, nde);
  return cudaGetLastError();
}

// Independent chains of packed u16x2 min and add: 16 chains per thread, 4 instructions per chain
// and iteration (2 mins, 2 adds). The result is stored so the chains are not optimised away.
__global__ void __launch_bounds__(256) int_probe_kernel(uint32_t* sink, int iters, uint32_t seed) {
  uint32_t a[16];
#pragma unroll
  for (int k = 0; k < 16; k++) a[k] = seed * (threadIdx.x + 7 * k + 1);
  const uint32_t p1 = 0x00030003u, p2 = 0x7F007F00u;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 16; k++) {
      a[k] = vmin2(a[k], p2) + p1;
      a[k] = vmin2(a[k], p2 ^ (uint32_t)i) + p1;
    }
  }
  uint32_t r = 0;
#pragma unroll
  for (int k = 0; k < 16; k++) r ^= a[k];
  if (r == 0x12345678u) sink[blockIdx.x] = r;
}

cudaError_t probe_int_peak(int iters, cudaStream_t s, double* lane_ops_per_s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, int_probe_kernel, 256, 0);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  uint32_t* sink = nullptr;
  cudaError_t e = cudaMallocAsync(&sink, grid * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int_probe_kernel<<<grid, 256, 0, s>>>(sink, iters / 8 + 1, 3u);  // warm-up
  cudaEventRecord(e0, s);
  int_probe_kernel<<<grid, 256, 0, s>>>(sink, iters, 5u);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, s);
  if (e != cudaSuccess) return e;
  const double instr = (double)grid * 256.0 * (double)iters * 16.0 * 4.0;
  *lane_ops_per_s = instr * 2.0 / (ms * 1e-3);
  return cudaStreamSynchronize(s);
}

}  // namespace r2t
