// Host-side launchers of the SGM kernels (C++ linkage, internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace r2t {

struct Tuning {
  int agg_dpl;    // disparities per lane of the row aggregation kernel (2, 4 or 8)
  int agg_warps;  // warps per aggregation block
  int wta_chunk;  // pixels per block of the WTA / right-disparity stage
  int shear_dpl;  // disparities per lane of the sheared-column kernel (16 or 32)
  int shear_cpl;  // chains per lane of the sheared-column kernel (1 or 2)
  int row_split;  // 1: one row direction per lane group, 0: both directions in one group
  int cost_mode;  // 0: population-count cost kernel, 1: tensor-core cost kernel (cost_mma_ok)
  int row_cost;   // 0: the row kernel reads the cost volume, 1: recomputes (rows_recompute_ok)
};

// A second stream and two events that let the two aggregation kernels run concurrently: the
// row kernel goes to `aux` (forked from and joined back to the caller's stream).
struct Fork {
  cudaStream_t aux;
  cudaEvent_t fork, join;
};
cudaError_t fork_create(Fork* f);
void fork_destroy(Fork* f);

// Default configuration for a disparity count D.
Tuning default_tuning(int D);
// True when the configuration can run a pair with D disparities.
bool tuning_valid(const Tuning& t, int D);

// Aggregation kernels on one stream (one launch each; defined in the agg_*.cu units): the row
// paths and the sheared-column paths.
template <bool WIDE>
cudaError_t launch_rows(const Problem& pb, const Method& mt, const Tuning& tn, cudaStream_t s);
template <bool WIDE>
cudaError_t launch_shear(const Problem& pb, const Method& mt, const Tuning& tn, cudaStream_t s);
// Persistent batch variants of the two kernels, as handles for cudaLaunchKernel. Parameters:
// (const BatchHeader*, const GroupDesc*, const Problem*, const AggSeg* segs,
// const int* seg_prefix, Method, unsigned* counters, int warp_smem); 256 threads; the sheared
// one takes 8 warp_smem bytes of dynamic shared memory (warp_smem: the largest shear_smem_bytes
// of the batch's settings).
template <bool WIDE>
const void* batch_row_kernel_fn();
template <bool WIDE>
const void* batch_shear_kernel_fn();

// Plain single-pair pipeline: 6 kernel launches on stream s (census of both images; cost +
// clearing of the aggregated volume; two aggregation kernels; WTA + right-disparity keys; LR
// check + median). With the exact check (mt.flags & 4; pb.flip and pb.dp set) first a flip kernel
// and the first five launches again on the swapped, flipped pair: 12 launches. The NCC cost
// (mt.flags & 8) takes 3 launches instead of 2 per pass.
// Returns the number of launches through *launches.
// ev: NULL, or events recorded around the stages: 5 (before the cost stage, after each of the
// four), with the exact check 8 (before the flip; after the cost, aggregation and WTA of each
// pass; after the LR check + median).
// fork: NULL runs the two aggregation kernels one after the other on s.
cudaError_t run_pipeline(const Problem& pb, const Method& mt, const Tuning& tn, cudaStream_t s,
                         int* launches, cudaEvent_t* ev = nullptr, const Fork* fork = nullptr);

// Cost volume of the 9 x 7 census on the tensor cores (tcgen05), with the clearing of the
// aggregated sums; the descriptor map pb.ct must be filled. cost_mma_ok: the shapes it covers
// (9 x 7 census, D = 64 or 128).
bool cost_mma_ok(const Problem& pb, const Method& mt);
// The row kernel recomputes its costs (tn.row_cost 1) when it runs one direction per warp with 32
// lanes of tn.agg_dpl disparities (D = 32 agg_dpl, one row direction per lane group) on the
// census cost; otherwise it reads the cost volume.
bool rows_recompute_ok(const Problem& pb, const Method& mt, const Tuning& tn);
cudaError_t launch_cost_mma(const Problem& pb, const Method& mt, cudaStream_t s);

// NCC matching cost (mt.flags & 8, patch mt.cw x mt.cw, pb.nst set): patch statistics
// of both images, then the cost volume with the clearing of the aggregated sums; 3 launches.
cudaError_t launch_ncc_cost(const Problem& pb, const Method& mt, cudaStream_t s);

// One image to rectify: raw rw x rh (raw_pitch bytes per row) through float maps of W x H
// (map_pitch bytes per row) into out (out_pitch bytes per row).
struct RectifyJob {
  const uint8_t* raw;
  int64_t raw_pitch;
  int rw, rh;
  const float* mapx;
  const float* mapy;
  int64_t map_pitch;
  uint8_t* out;
  int64_t out_pitch;
  int W, H;
};
// Rectifies n (1 or 2) images in one launch.
cudaError_t launch_rectify(const RectifyJob* jobs, int n, cudaStream_t s);

// Sets the calling thread's res2tac_last_error message; returns code.
int report_error(int code, const char* msg);

// Packed-u16 integer throughput probe: lane operations per second.
cudaError_t probe_int_peak(int iters, cudaStream_t s, double* lane_ops_per_s);

// POPC-throughput probe: 32-bit population counts per second on every SM.
cudaError_t probe_popc_rate(int iters, cudaStream_t s, double* popc_per_s);

// Reduction-throughput probe: bytes per second that TMA bulk add-reductions achieve into a buffer
// of `bytes` bytes, `passes` passes.
cudaError_t probe_red_peak(int64_t bytes, int passes, cudaStream_t s, double* bytes_per_s);

// Copies the aggregated volume as saturated uint16 / the cost volume, both in natural order.
cudaError_t copy_agg_u16(const Problem& pb, bool wide, uint16_t* dst, cudaStream_t s);
cudaError_t copy_cost(const Problem& pb, uint8_t* dst, cudaStream_t s);
// Writes the sub-pixel D^L map of the last sub-pixel run (float [H][W]).
cudaError_t copy_subpixel(const Problem& pb, bool wide, float* dst, cudaStream_t s);

}  // namespace r2t
