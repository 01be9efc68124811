// The two aggregation kernels (row paths, sheared-column paths), their plain launchers and their
// persistent batch variants, as templates over WIDE (uint32 sums). Each agg_*.cu unit
// instantiates one family for one WIDE value, so the build compiles them in parallel.
#pragma once
#include "aggregate.cuh"
#include "batch_dev.cuh"
#include "launch.h"

namespace r2t {

// ------------------------------------------------------------------------------- plain launches
template <int DPL, int LPL, bool WIDE, bool FULL, bool SPLIT>
__global__ void __launch_bounds__(512) agg_row_kernel(Problem pb, Method mt) {
  const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  agg_rows<DPL, LPL, WIDE, FULL, SPLIT>(pb, mt, warp * (32 / LPL), 0x7FFFFFFF);
}

// The row kernel with the costs recomputed from the descriptor map (one direction per warp).
template <int DPL, bool WIDE, bool FULL>
__global__ void __launch_bounds__(512) agg_row_rc_kernel(Problem pb, Method mt) {
  const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  agg_rows_recompute<DPL, 32, WIDE, FULL>(pb, mt, warp, 0x7FFFFFFF);
}

template <int DPL, int WD, int CPL, bool WIDE, bool FULL>
__global__ void __launch_bounds__(256) agg_shear_kernel(Problem pb, Method mt, int items) {
  extern __shared__ __align__(16) uint8_t shm[];
  const int wib = threadIdx.x >> 5;
  const int item = blockIdx.x * (blockDim.x >> 5) + wib;
  if (item >= items) return;  // whole warp
  uint8_t* base = shm + wib * shear_smem_bytes(DPL, WIDE, CPL);
  agg_shear<DPL, WD, CPL, WIDE, FULL>(pb, mt, item, base, base + shear_ring_bytes(DPL, CPL));
}

template <int DPL, int LPL, bool WIDE, bool SPLIT>
static cudaError_t launch_rows_t(const Problem& pb, const Method& mt, int warps, cudaStream_t s) {
  const int nu = row_units(pb.H, SPLIT);
  const int nwarp = (nu + 32 / LPL - 1) / (32 / LPL);
  const int grid = (nwarp + warps - 1) / warps;
  if (pb.D == DPL * LPL)
    agg_row_kernel<DPL, LPL, WIDE, true, SPLIT><<<grid, warps * 32, 0, s>>>(pb, mt);
  else
    agg_row_kernel<DPL, LPL, WIDE, false, SPLIT><<<grid, warps * 32, 0, s>>>(pb, mt);
  return cudaGetLastError();
}

template <bool WIDE, bool SPLIT>
static cudaError_t launch_rows_s(const Problem& pb, const Method& mt, const Tuning& tn,
                                 cudaStream_t s) {
  switch (tn.agg_dpl * 100 + long_lanes(pb.D, tn.agg_dpl)) {
    case 208: return launch_rows_t<2, 8, WIDE, SPLIT>(pb, mt, tn.agg_warps, s);
    case 216: return launch_rows_t<2, 16, WIDE, SPLIT>(pb, mt, tn.agg_warps, s);
    case 232: return launch_rows_t<2, 32, WIDE, SPLIT>(pb, mt, tn.agg_warps, s);
    case 408: return launch_rows_t<4, 8, WIDE, SPLIT>(pb, mt, tn.agg_warps, s);
    case 416: return launch_rows_t<4, 16, WIDE, SPLIT>(pb, mt, tn.agg_warps, s);
    case 432: return launch_rows_t<4, 32, WIDE, SPLIT>(pb, mt, tn.agg_warps, s);
    case 808: return launch_rows_t<8, 8, WIDE, SPLIT>(pb, mt, tn.agg_warps, s);
    case 816: return launch_rows_t<8, 16, WIDE, SPLIT>(pb, mt, tn.agg_warps, s);
    case 832: return launch_rows_t<8, 32, WIDE, SPLIT>(pb, mt, tn.agg_warps, s);
    default: return cudaErrorInvalidValue;
  }
}

// Recomputed costs (tuning row_cost 1): one row direction per warp of 32 lanes (D = 32 dpl),
// census cost only (the NCC cost has no descriptor map).
template <int DPL, bool WIDE>
static cudaError_t launch_rows_rc(const Problem& pb, const Method& mt, int warps, cudaStream_t s) {
  const int nu = row_units(pb.H, true);
  const int grid = (nu + warps - 1) / warps;
  agg_row_rc_kernel<DPL, WIDE, true><<<grid, warps * 32, 0, s>>>(pb, mt);
  return cudaGetLastError();
}

template <bool WIDE>
cudaError_t launch_rows(const Problem& pb, const Method& mt, const Tuning& tn,
                               cudaStream_t s) {
  if (rows_recompute_ok(pb, mt, tn)) {
    switch (tn.agg_dpl) {
      case 2: return launch_rows_rc<2, WIDE>(pb, mt, tn.agg_warps, s);
      case 4: return launch_rows_rc<4, WIDE>(pb, mt, tn.agg_warps, s);
      default: return launch_rows_rc<8, WIDE>(pb, mt, tn.agg_warps, s);
    }
  }
  return tn.row_split ? launch_rows_s<WIDE, true>(pb, mt, tn, s)
                      : launch_rows_s<WIDE, false>(pb, mt, tn, s);
}

template <int DPL, int WD, int CPL, bool WIDE>
static cudaError_t launch_shear_t(const Problem& pb, const Method& mt, int warps, cudaStream_t s) {
  const int items = shear_items(pb.W, pb.D, DPL, mt.num_paths, CPL);
  if (warps > 8) warps = 8;  // blocks of at most 256 threads (the kernel's launch bound)
  while (warps > 1 && warps * shear_smem_bytes(DPL, WIDE, CPL) > (200 << 10)) warps--;
  const int grid = (items + warps - 1) / warps;
  const size_t smem = (size_t)warps * shear_smem_bytes(DPL, WIDE, CPL);
  if (pb.D == DPL * WD) {
    cudaFuncSetAttribute(agg_shear_kernel<DPL, WD, CPL, WIDE, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    agg_shear_kernel<DPL, WD, CPL, WIDE, true><<<grid, warps * 32, smem, s>>>(pb, mt, items);
  } else {
    cudaFuncSetAttribute(agg_shear_kernel<DPL, WD, CPL, WIDE, false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    agg_shear_kernel<DPL, WD, CPL, WIDE, false><<<grid, warps * 32, smem, s>>>(pb, mt, items);
  }
  return cudaGetLastError();
}

template <int CPL, bool WIDE>
static cudaError_t launch_shear_c(const Problem& pb, const Method& mt, const Tuning& tn,
                                  cudaStream_t s) {
  switch (tn.shear_dpl * 100 + shear_width(pb.D, tn.shear_dpl)) {
    case 802: return launch_shear_t<8, 2, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 804: return launch_shear_t<8, 4, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 808: return launch_shear_t<8, 8, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 816: return launch_shear_t<8, 16, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 832: return launch_shear_t<8, 32, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 1601: return launch_shear_t<16, 1, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 1602: return launch_shear_t<16, 2, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 1604: return launch_shear_t<16, 4, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 1608: return launch_shear_t<16, 8, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 1616: return launch_shear_t<16, 16, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 3201: return launch_shear_t<32, 1, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 3202: return launch_shear_t<32, 2, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 3204: return launch_shear_t<32, 4, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    case 3208: return launch_shear_t<32, 8, CPL, WIDE>(pb, mt, tn.agg_warps, s);
    default: return cudaErrorInvalidValue;
  }
}

template <bool WIDE>
cudaError_t launch_shear(const Problem& pb, const Method& mt, const Tuning& tn, cudaStream_t s) {
  return tn.shear_cpl == 2 ? launch_shear_c<2, WIDE>(pb, mt, tn, s)
                           : launch_shear_c<1, WIDE>(pb, mt, tn, s);
}

// ------------------------------------------------------------------------------- batch kernels
template <int DPL, int LPL, bool WIDE>
__device__ __forceinline__ void rows_full(const Problem& pb, const Method& mt, int unit0,
                                          int unit_end) {
  // one row direction per lane group (units 0 .. 2H - 1), as the single-pair default
  if (pb.D == DPL * LPL)
    agg_rows<DPL, LPL, WIDE, true, true>(pb, mt, unit0, unit_end);
  else
    agg_rows<DPL, LPL, WIDE, false, true>(pb, mt, unit0, unit_end);
}

template <bool WIDE>
__device__ __forceinline__ void rows_dispatch(const Problem& pb, const Method& mt, int unit0,
                                              int unit_end, int dpl) {
  switch (dpl * 100 + long_lanes(pb.D, dpl)) {
    case 208: rows_full<2, 8, WIDE>(pb, mt, unit0, unit_end); break;
    case 216: rows_full<2, 16, WIDE>(pb, mt, unit0, unit_end); break;
    case 232: rows_full<2, 32, WIDE>(pb, mt, unit0, unit_end); break;
    case 408: rows_full<4, 8, WIDE>(pb, mt, unit0, unit_end); break;
    case 416: rows_full<4, 16, WIDE>(pb, mt, unit0, unit_end); break;
    case 432: rows_full<4, 32, WIDE>(pb, mt, unit0, unit_end); break;
    case 808: rows_full<8, 8, WIDE>(pb, mt, unit0, unit_end); break;
    case 816: rows_full<8, 16, WIDE>(pb, mt, unit0, unit_end); break;
    case 832: rows_full<8, 32, WIDE>(pb, mt, unit0, unit_end); break;
    default: break;
  }
}

template <int DPL, int WD, int CPL, bool WIDE>
__device__ __forceinline__ void shear_full(const Problem& pb, const Method& mt, int item,
                                           uint8_t* base) {
  if (pb.D == DPL * WD)
    agg_shear<DPL, WD, CPL, WIDE, true>(pb, mt, item, base, base + shear_ring_bytes(DPL, CPL));
  else
    agg_shear<DPL, WD, CPL, WIDE, false>(pb, mt, item, base, base + shear_ring_bytes(DPL, CPL));
}

// The sheared-column setting (dpl, cpl) of a batch bucket (batch_shear_ok). base: this warp's
// shear_smem_bytes of that setting.
template <bool WIDE>
__device__ __forceinline__ void shear_dispatch(const Problem& pb, const Method& mt, int item,
                                               uint8_t* base, int dpl, int cpl) {
  switch (dpl * 1000 + cpl * 100 + shear_width(pb.D, dpl)) {
    case 16101: shear_full<16, 1, 1, WIDE>(pb, mt, item, base); break;
    case 16102: shear_full<16, 2, 1, WIDE>(pb, mt, item, base); break;
    case 16104: shear_full<16, 4, 1, WIDE>(pb, mt, item, base); break;
    case 16108: shear_full<16, 8, 1, WIDE>(pb, mt, item, base); break;
    case 16116: shear_full<16, 16, 1, WIDE>(pb, mt, item, base); break;
    case 16201: shear_full<16, 1, 2, WIDE>(pb, mt, item, base); break;
    case 16202: shear_full<16, 2, 2, WIDE>(pb, mt, item, base); break;
    case 16204: shear_full<16, 4, 2, WIDE>(pb, mt, item, base); break;
    case 16208: shear_full<16, 8, 2, WIDE>(pb, mt, item, base); break;
    case 16216: shear_full<16, 16, 2, WIDE>(pb, mt, item, base); break;
    default: break;
  }
}

// Persistent aggregation kernels of one group of a batch: warps claim row units / sheared items
// from the group's queue; the segment of an item is found among the group's pairs.
template <bool WIDE>
__global__ void __launch_bounds__(256) batch_row_kernel(const BatchHeader* hd, const GroupDesc* gd,
                                                        const Problem* probs, const AggSeg* segs,
                                                        const int* seg_prefix, Method mt,
                                                        unsigned* counters, int warp_smem) {
  const int p0 = gd->p0, np = gd->np, lo = gd->lo[kStRows], hi = gd->hi[kStRows];
  for (;;) {
    const int item = lo + claim_warp(&counters[kStRows]);
    if (item >= hi) break;
    const int si = p0 + find_slot(seg_prefix + p0, np, item);
    const AggSeg sg = segs[si];
    const Problem pb = probs[sg.pair];
    rows_dispatch<WIDE>(pb, mt, sg.begin + (item - seg_prefix[si]) * sg.group, sg.end,
                        hd->tune[tune_bucket(pb.W, pb.H, pb.D)].row_dpl);
  }
}

// warp_smem: shared memory of one warp, at least shear_smem_bytes(dpl, WIDE, cpl) of every
// bucket setting the batch uses.
template <bool WIDE>
__global__ void __launch_bounds__(256) batch_shear_kernel(const BatchHeader* hd,
                                                          const GroupDesc* gd,
                                                          const Problem* probs, const AggSeg* segs,
                                                          const int* seg_prefix, Method mt,
                                                          unsigned* counters, int warp_smem) {
  extern __shared__ __align__(16) uint8_t shm[];
  uint8_t* base = shm + (threadIdx.x >> 5) * warp_smem;
  const int p0 = gd->p0, np = gd->np, lo = gd->lo[kStShear], hi = gd->hi[kStShear];
  for (;;) {
    const int item = lo + claim_warp(&counters[kStShear]);
    if (item >= hi) break;
    const int si = p0 + find_slot(seg_prefix + p0, np, item);
    const AggSeg sg = segs[si];
    const Problem pb = probs[sg.pair];
    const BatchTune tn = hd->tune[tune_bucket(pb.W, pb.H, pb.D)];
    shear_dispatch<WIDE>(pb, mt, sg.begin + (item - seg_prefix[si]) * sg.group, base,
                         tn.shear_dpl, tn.shear_cpl);
  }
}

template <bool WIDE>
const void* batch_row_kernel_fn() {
  return reinterpret_cast<const void*>(batch_row_kernel<WIDE>);
}
template <bool WIDE>
const void* batch_shear_kernel_fn() {
  return reinterpret_cast<const void*>(batch_shear_kernel<WIDE>);
}

}  // namespace r2t
