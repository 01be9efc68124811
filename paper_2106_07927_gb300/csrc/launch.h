// Host-side launchers of the SGM kernels (C++ linkage, internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace r2t {

struct Tuning {
  int agg_dpl;    // disparities per lane (2, 4 or 8)
  int agg_warps;  // warps per aggregation block
  int wta_chunk;  // pixels per chunk of the row walk
};

// Default configuration for a disparity count D.
Tuning default_tuning(int D);
// True when the configuration can run a pair with D disparities.
bool tuning_valid(const Tuning& t, int D);

// Plain single-pair pipeline: 4 or 5 kernel launches on stream s (census, cost + clearing of
// the aggregated volume, aggregation, WTA / right disparity / LR check, median). Returns the
// number of launches through *launches.
// ev: NULL, or 6 events recorded around the stages (before census, after each of the five
// stages; the median slot is recorded even when the median is skipped).
cudaError_t run_pipeline(const Problem& pb, const Method& mt, const Tuning& tn, cudaStream_t s,
                         int* launches, cudaEvent_t* ev = nullptr);

// Sets the calling thread's res2tac_last_error message; returns code.
int report_error(int code, const char* msg);

// Packed-u16 integer throughput probe: lane operations per second.
cudaError_t probe_int_peak(int iters, cudaStream_t s, double* lane_ops_per_s);

// Converts the aggregated volume to saturated uint16 (identity copy when not wide).
cudaError_t copy_agg_u16(const Problem& pb, bool wide, uint16_t* dst, cudaStream_t s);

}  // namespace r2t
