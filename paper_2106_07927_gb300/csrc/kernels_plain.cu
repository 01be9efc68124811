// Plain single-pair launches of the SGM stages (one kernel per stage, all on the caller's stream).
#include <nvtx3/nvToolsExt.h>

#include <algorithm>

#include "aggregate.cuh"
#include "census_cost.cuh"
#include "launch.h"
#include "post.cuh"

namespace r2t {

__global__ void __launch_bounds__(256) census_kernel(Problem pb, Method mt) {
  __shared__ CensusSmem sm;
  census_tile_dispatch(pb, mt, blockIdx.x, sm);
}

__global__ void __launch_bounds__(256) cost_kernel(Problem pb, Method mt) {
  __shared__ CostSmem sm;
  cost_tile_dispatch(pb, mt, blockIdx.x, sm);
}

template <bool WIDE>
__global__ void __launch_bounds__(256) wta_dr_staged_kernel(Problem pb, int T) {
  extern __shared__ __align__(16) uint8_t wsm[];
  wta_dr_staged<WIDE>(pb, blockIdx.x, wsm, T);
}

template <bool SUB, bool WIDE>
__global__ void __launch_bounds__(256) lr_median_kernel(Problem pb, Method mt) {
  __shared__ MedianSmemT<SUB> sm;
  lr_median_tile<SUB, WIDE>(pb, mt, blockIdx.x, sm);
}

// Debug map of the sub-pixel D^L (before the left-right check).
template <bool WIDE>
__global__ void subpixel_map_kernel(Problem pb, float* out) {
  const int64_t n = (int64_t)pb.W * pb.H;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = refine_subpixel<WIDE>(pb, i, pb.dl[i]);
}

cudaError_t copy_subpixel(const Problem& pb, bool wide, float* dst, cudaStream_t s) {
  if (wide)
    subpixel_map_kernel<true><<<608, 256, 0, s>>>(pb, dst);
  else
    subpixel_map_kernel<false><<<608, 256, 0, s>>>(pb, dst);
  return cudaGetLastError();
}

// Debug copy of the aggregated volume, sums saturated to uint16.
template <bool WIDE>
__global__ void agg_copy_kernel(const void* src, uint16_t* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t v = WIDE ? min(reinterpret_cast<const uint32_t*>(src)[i], 65535u)
                            : reinterpret_cast<const uint16_t*>(src)[i];
    dst[i] = (uint16_t)v;
  }
}

Tuning default_tuning(int D) {
  Tuning t;
  t.agg_dpl = long_dpl_default(D);
  t.agg_warps = 2;  // two warps per block (measured best with one row direction per lane group)
  t.wta_chunk = 128;  // staged WTA tiles of 128 pixels: measured faster than 64 or 256 (D = 128)
  t.shear_dpl = shear_dpl_default(D);
  t.shear_cpl = shear_cpl_default(D);
  t.row_split = 1;  // one row direction per lane group (measured 2 % faster at D = 128)
  t.cost_mode = 0;  // population counts: measured faster than the tensor-core kernel
  t.row_cost = 0;   // the row kernel reads the cost volume
  return t;
}

bool tuning_valid(const Tuning& t, int D) {
  if (t.agg_dpl != 2 && t.agg_dpl != 4 && t.agg_dpl != 8) return false;
  if (D % t.agg_dpl != 0) return false;
  if ((D + t.agg_dpl - 1) / t.agg_dpl > 32) return false;
  if (t.agg_warps < 1 || t.agg_warps > 16) return false;
  if (t.wta_chunk != 64 && t.wta_chunk != 128 && t.wta_chunk != 256) return false;
  if (t.shear_dpl != 8 && t.shear_dpl != 16 && t.shear_dpl != 32) return false;
  if (t.shear_cpl != 1 && t.shear_cpl != 2) return false;
  if (D % t.shear_dpl != 0) return false;
  if (t.row_split != 0 && t.row_split != 1) return false;
  if (t.cost_mode != 0 && t.cost_mode != 1) return false;
  if (t.row_cost != 0 && t.row_cost != 1) return false;
  return true;
}

bool rows_recompute_ok(const Problem& pb, const Method& mt, const Tuning& tn) {
  return tn.row_cost == 1 && tn.row_split == 1 && !(mt.flags & 8) && pb.D == 32 * tn.agg_dpl;
}

cudaError_t fork_create(Fork* f) {
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  cudaError_t e = cudaStreamCreateWithPriority(&f->aux, cudaStreamNonBlocking, hi);
  // Timing-enabled events: measured with steps queued back to back, fork/join events created
  // with cudaEventDisableTiming left about one step in five at 0.73 ms instead of 0.39 ms (the
  // two aggregation kernels stopped overlapping); with timing enabled every step overlapped.
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->fork, cudaEventDefault);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->join, cudaEventDefault);
  return e;
}

void fork_destroy(Fork* f) {
  if (f->aux) cudaStreamDestroy(f->aux);
  if (f->fork) cudaEventDestroy(f->fork);
  if (f->join) cudaEventDestroy(f->join);
  f->aux = nullptr;
  f->fork = f->join = nullptr;
}

static cudaError_t launch_aggregate(const Problem& pb, const Method& mt, const Tuning& tn,
                                    cudaStream_t s, const Fork* fork) {
  cudaStream_t ls = s;
  if (fork) {
    cudaEventRecord(fork->fork, s);
    cudaStreamWaitEvent(fork->aux, fork->fork, 0);
    ls = fork->aux;
  }
  cudaError_t e = mt.wide ? launch_rows<true>(pb, mt, tn, ls) : launch_rows<false>(pb, mt, tn, ls);
  if (e != cudaSuccess) return e;
  e = mt.wide ? launch_shear<true>(pb, mt, tn, s) : launch_shear<false>(pb, mt, tn, s);
  if (e != cudaSuccess) return e;
  if (fork) {
    cudaEventRecord(fork->join, fork->aux);
    cudaStreamWaitEvent(s, fork->join, 0);
  }
  return cudaGetLastError();
}

// Census + cost (or the NCC cost), aggregation and WTA (with the right-disparity keys) of the
// pair pb.left / pb.right into pb.dl; adds its launches to *n. ev: NULL, or 3 events recorded
// after each of the 3 stages.
static cudaError_t run_pass(const Problem& pb, const Method& mt, const Tuning& tn, cudaStream_t s,
                            cudaEvent_t* ev, const Fork* fork, int* n) {
  cudaError_t e;
  nvtxRangePushA("res2tac census + cost");
  if (mt.flags & 8) {
    e = launch_ncc_cost(pb, mt, s);
    nvtxRangePop();
    if (e != cudaSuccess) return e;
    *n += 3;
  } else {
    census_kernel<<<2 * census_items(pb.W, pb.H), 256, 0, s>>>(pb, mt);
    if (tn.cost_mode == 1 && cost_mma_ok(pb, mt)) {
      if ((e = launch_cost_mma(pb, mt, s)) != cudaSuccess) return e;
    } else {
      cost_kernel<<<cost_items(pb.W, pb.H), 256, 0, s>>>(pb, mt);
    }
    nvtxRangePop();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    *n += 2;
  }
  if (ev) cudaEventRecord(ev[0], s);
  nvtxRangePushA("res2tac aggregation");
  e = launch_aggregate(pb, mt, tn, s, fork);
  nvtxRangePop();
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[1], s);
  nvtxRangePushA("res2tac wta + right-disparity keys");
  // pixels per block of 256 threads, capped so that the staged sums take at most 64 KB
  const int T = wta_staged_px(pb.D, mt.wide != 0, tn.wta_chunk);
  const size_t smem = wta_staged_smem_bytes(pb.D, mt.wide != 0, T);
  const int nw = wta_items(pb.W, pb.H, T);
  if (mt.wide) {
    cudaFuncSetAttribute(wta_dr_staged_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    wta_dr_staged_kernel<true><<<nw, 256, smem, s>>>(pb, T);
  } else {
    cudaFuncSetAttribute(wta_dr_staged_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    wta_dr_staged_kernel<false><<<nw, 256, smem, s>>>(pb, T);
  }
  nvtxRangePop();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[2], s);
  *n += 3;
  return cudaSuccess;
}

// The swapped, horizontally flipped pair of the exact consistency check (Sec. 3.2.3): the new
// reference is the right image mirrored, the new matching image the left one mirrored.
__global__ void flip_pair_kernel(Problem pb) {
  const int W = pb.W;
  const int64_t n = (int64_t)W * pb.H;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / W;
    const int x = (int)(i - y * W);
    const int64_t src = y * pb.in_pitch + (W - 1 - x);
    pb.flip[i] = pb.right[src];
    pb.flip[n + i] = pb.left[src];
  }
}

cudaError_t run_pipeline(const Problem& pb, const Method& mt, const Tuning& tn, cudaStream_t s,
                         int* launches, cudaEvent_t* ev, const Fork* fork) {
  const bool exact = (mt.flags & 4) != 0;
  if (exact && (!pb.flip || !pb.dp)) return cudaErrorInvalidValue;
  int n = 0;
  cudaError_t e;
  if (ev) cudaEventRecord(ev[0], s);
  if (exact) {
    // D^R from scratch: the whole matching of the swapped, flipped pair; its D^L read mirrored
    // is D^R of the original pair
    const int64_t npx = (int64_t)pb.W * pb.H;
    const int grid = (int)std::min<int64_t>((npx + 255) / 256, 1216);
    flip_pair_kernel<<<grid, 256, 0, s>>>(pb);
    n++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    Problem pf = pb;
    pf.left = pb.flip;
    pf.right = pb.flip + npx;
    pf.in_pitch = pb.W;
    pf.dl = pb.dp;
    if ((e = run_pass(pf, mt, tn, s, ev ? ev + 1 : nullptr, fork, &n)) != cudaSuccess) return e;
  }
  if ((e = run_pass(pb, mt, tn, s, ev ? ev + (exact ? 4 : 1) : nullptr, fork, &n)) !=
      cudaSuccess)
    return e;
  const int nm = median_items(pb.W, pb.H);
  nvtxRangePushA("res2tac lr check + median");
  if (pb.disp_f == nullptr)  // uint16 map
    lr_median_kernel<false, false><<<nm, 256, 0, s>>>(pb, mt);
  else if (mt.wide)          // sub-pixel float map
    lr_median_kernel<true, true><<<nm, 256, 0, s>>>(pb, mt);
  else
    lr_median_kernel<true, false><<<nm, 256, 0, s>>>(pb, mt);
  nvtxRangePop();
  n++;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[exact ? 7 : 4], s);
  if (launches) *launches = n;
  return cudaSuccess;
}

cudaError_t copy_agg_u16(const Problem& pb, bool wide, uint16_t* dst, cudaStream_t s) {
  const int64_t n = (int64_t)pb.W * pb.H * pb.D;
  if (wide)
    agg_copy_kernel<true><<<1216, 256, 0, s>>>(pb.agg, dst, n);
  else
    agg_copy_kernel<false><<<1216, 256, 0, s>>>(pb.agg, dst, n);
  return cudaGetLastError();
}

cudaError_t copy_cost(const Problem& pb, uint8_t* dst, cudaStream_t s) {
  return cudaMemcpyAsync(dst, pb.cost, (size_t)pb.W * pb.H * pb.D, cudaMemcpyDeviceToDevice, s);
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

// Independent chains of 32-bit POPC (each fed by an XOR and an integer multiply-add), 16 per
// thread: the rate at which the cost could be recomputed from census descriptors.
__global__ void __launch_bounds__(256) popc_probe_kernel(uint32_t* sink, int iters, uint32_t seed) {
  uint32_t a[16];
#pragma unroll
  for (int k = 0; k < 16; k++) a[k] = seed * (threadIdx.x + 7 * k + 1);
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 16; k++) a[k] = __popc(a[k] ^ (uint32_t)i) + a[k] * 3u;
  }
  uint32_t r = 0;
#pragma unroll
  for (int k = 0; k < 16; k++) r ^= a[k];
  if (r == 0x12345678u) sink[blockIdx.x] = r;
}

cudaError_t probe_popc_rate(int iters, cudaStream_t s, double* popc_per_s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, popc_probe_kernel, 256, 0);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  uint32_t* sink = nullptr;
  cudaError_t e = cudaMallocAsync(&sink, grid * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  popc_probe_kernel<<<grid, 256, 0, s>>>(sink, iters / 8 + 1, 3u);  // warm-up
  cudaEventRecord(e0, s);
  popc_probe_kernel<<<grid, 256, 0, s>>>(sink, iters, 5u);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, s);
  if (e != cudaSuccess) return e;
  *popc_per_s = (double)grid * 256.0 * (double)iters * 16.0 / (ms * 1e-3);
  return cudaStreamSynchronize(s);
}

// Reduction-throughput probe: every warp stages 1 KB of 32-bit ones in shared memory once, then
// adds it into the buffer's 1 KB runs with TMA bulk reductions (4 per group, at most two groups
// reading shared memory at a time), the way the sheared aggregation kernel adds its runs into S.
__global__ void __launch_bounds__(256) red_probe_kernel(uint8_t* buf, int64_t runs, int passes) {
  __shared__ __align__(16) uint32_t stage[8][256];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int i = lane; i < 256; i += 32) stage[wib][i] = 1u;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) {
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    const uint32_t src = (uint32_t)__cvta_generic_to_shared(stage[wib]);
    int k = 0;
    for (int p = 0; p < passes; p++) {
      for (int64_t r = w; r < runs; r += nw) {
        asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u32 [%0], [%1], 1024;"
                     ::"l"(buf + r * 1024), "r"(src) : "memory");
        if (++k == 4) {
          k = 0;
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        }
      }
    }
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  __syncwarp();
}

cudaError_t probe_red_peak(int64_t bytes, int passes, cudaStream_t s, double* bytes_per_s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t runs = bytes / 1024;
  uint8_t* buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, runs * 1024, s);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(buf, 0, runs * 1024, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = sms * 4;
  red_probe_kernel<<<grid, 256, 0, s>>>(buf, runs, 1);  // warm-up
  cudaEventRecord(e0, s);
  red_probe_kernel<<<grid, 256, 0, s>>>(buf, runs, passes);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(buf, s);
  if (e != cudaSuccess) return e;
  *bytes_per_s = (double)runs * 1024.0 * passes / (ms * 1e-3);
  return cudaStreamSynchronize(s);
}

}  // namespace r2t
