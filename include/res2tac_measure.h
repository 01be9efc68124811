/*
 * res2tac_measure.h - measurement and diagnostic aids of the GB300 SGM stereo library
 * (libres2tac.so).
 *
 * Not part of the method and not needed to compute disparities: these entry points measure the
 * GPU the library runs on (the integer and reduction rates that bound the path aggregation), for
 * the benchmark's roofline, and report the range checks of the debug build. Same conventions as res2tac.h: plain C, return 0 or a negative
 * RES2TAC_E* code, asynchronous work on the given stream unless stated.
 */
#ifndef RES2TAC_MEASURE_H_
#define RES2TAC_MEASURE_H_

#include "res2tac.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Integer-throughput probe (measurement aid, not part of the method): runs independent chains
 * of packed u16x2 min and add instructions on every SM for about `iters` iterations on stream s
 * and returns the sustained rate in 16-bit lane operations per second (one packed instruction
 * counts two) through *lane_ops_per_s. Synchronises s. */
int res2tac_probe_int_peak(int iters, res2tac_stream_t s, double* lane_ops_per_s);

/* Reduction-throughput probe (measurement aid, not part of the method): allocates a device buffer
 * of `bytes` bytes (>= 1024) on stream s, adds 32-bit ones into all of it `passes` times with TMA
 * bulk add-reductions of 1 KB (the way the column / diagonal aggregation adds its runs into the
 * aggregated volume), frees it, and returns the sustained rate in bytes reduced per second through
 * *bytes_per_s. Synchronises s. RES2TAC_ENOMEM if the buffer does not fit. */
int res2tac_probe_red_peak(int64_t bytes, int32_t passes, res2tac_stream_t s, double* bytes_per_s);

/* POPC-throughput probe (measurement aid): independent chains of 32-bit population counts on
 * every SM for about `iters` iterations on stream s; returns the sustained rate in POPC per second
 * through *popc_per_s (the bound on recomputing the census cost inside the aggregation, which
 * needs two per disparity estimate and path). Synchronises s. */
int res2tac_probe_popc_rate(int iters, res2tac_stream_t s, double* popc_per_s);

/* Range checks of the debug build. libres2tac_check.so is the same library compiled with
 * RES2TAC_CHECK_BOUNDS: before each global access of the path-aggregation and WTA kernels it
 * tests that the bytes lie inside their buffer (the cost volume, the aggregated volume, D^L),
 * and on a failure records the first failing site and byte offset in the context and skips the
 * access; nothing traps. Sites: 1 row-path cost load, 2 row-path add into the aggregated volume,
 * 3 column / diagonal cost copy, 4 and 5 column / diagonal bulk add (before / after a run wraps
 * around the image edge), 6 WTA copy of the aggregated volume, 7 WTA store of D^L.
 * res2tac_bounds_status reads the record of the context's single-pair calls (synchronous):
 * *checked = 1 in the debug build, 0 otherwise; *site = 0 when no check failed since
 * res2tac_create. Any output pointer may be NULL. */
int res2tac_bounds_status(res2tac_t h, int32_t* checked, int32_t* site, int64_t* offset);

#ifdef __cplusplus
}
#endif

#endif /* RES2TAC_MEASURE_H_ */
