/*
 * res2tac_measure.h - measurement aids of the GB300 SGM stereo library (libres2tac.so).
 *
 * Not part of the method and not needed to compute disparities: these entry points measure the
 * GPU the library runs on (the integer and reduction rates that bound the path aggregation), for
 * the benchmark's roofline. Same conventions as res2tac.h: plain C, return 0 or a negative
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

#ifdef __cplusplus
}
#endif

#endif /* RES2TAC_MEASURE_H_ */
