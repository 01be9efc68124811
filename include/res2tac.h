/*
 * res2tac.h: C ABI of the GB300 SGM stereo library (census transform, Hamming matching cost,
 * semi-global path aggregation, winner-takes-all, approximate left-right consistency check and
 * 3x3 median) after Ruf et al., "ReS2tAC: UAV-borne real-time SGM stereo optimized for embedded
 * ARM and CUDA devices", Sensors 2021.
 *
 * Every compute call runs all of its work in CUDA kernels for sm_103a on the caller's stream.
 * No call falls back to the CPU. Types are plain C: image and output buffers are raw pointers
 * (device memory unless a function says "host"), sizes are int32/int64, streams are passed as
 * an opaque pointer that must be a cudaStream_t of the current device (NULL = legacy default).
 *
 * Data layout. Images are 8-bit grayscale, row-major with a pitch in bytes. The left image is
 * the reference (Sec. 2.1.1). Disparity maps are uint16, row-major with a pitch in bytes, and
 * hold d in [0, D-1] or RES2TAC_INVALID. Cost and aggregated volumes are [y][x][d] with the D
 * disparities of one pixel contiguous (Sec. 2.2.1), d = 0 .. D-1.
 *
 * Errors. Functions return RES2TAC_OK (0) or a negative code; nothing is thrown across the
 * ABI. res2tac_last_error() returns a message for the last failure on the calling thread.
 * A context is not thread-safe: use one context per host thread / stream.
 */
#ifndef RES2TAC_H_
#define RES2TAC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RES2TAC_OK 0
#define RES2TAC_EINVAL (-1)   /* bad parameter, shape, pitch or NULL pointer */
#define RES2TAC_ENOMEM (-2)   /* device memory for the scratch could not be allocated */
#define RES2TAC_ECUDA (-3)    /* a CUDA runtime call or launch failed (message kept) */
#define RES2TAC_ETIMEOUT (-4) /* reserved: a bounded device-side wait gave up (none exists today) */

/* flags */
#define RES2TAC_LR_CHECK 1 /* approximate left-right consistency check, Eq. (LR_check) */
#define RES2TAC_MEDIAN 2   /* 3x3 median over the valid pixels, Sec. 2.1.3 */
/* exact consistency check (Sec. 3.2.3, "exact-cc" in Tab. throughput): D^R for the check is the
 * full matching of the swapped, horizontally flipped pair (census, cost, aggregation and WTA
 * again, read back mirrored) instead of the approximation of Eq. (right_disparity); about twice
 * the work. Single pairs only: res2tac_compute_batch rejects it. */
#define RES2TAC_EXACT_CC 4
/* NCC matching cost (Sec. 2.1.1, Sec. 2.2.1 "Inverted and truncated version of the normalized
 * cross-correlation") instead of the census: s = 1 - max(0, Phi) with Phi the zero-mean NCC of
 * the census_w x census_h patches (5 x 5 or 9 x 9; zero margin outside the image), on the same
 * 8-bit cost scale: cost = 255 - k, k = round(255 max(0, Phi)) with ties to even, where for
 * N = n^2 the integers cov = N sum ab - sum a sum b, vA = N sum a^2 - (sum a)^2 (vB likewise) give
 * Phi = cov / sqrt(vA vB), and Phi = 0 when vA or vB is 0 (a constant patch: cost 255). k is exact
 * (settled on integers wherever an fp32 estimate could round either way). 255 where x - d < 0.
 * Single pairs only: res2tac_compute_batch rejects it. */
#define RES2TAC_NCC 8

#define RES2TAC_INVALID 0xFFFF /* disparity of a pixel rejected by the left-right check */

typedef struct res2tac_ctx* res2tac_t;
typedef void* res2tac_stream_t; /* a cudaStream_t */

/* Problem statement as the paper gives it.
 *   width, height  image size W x H, 1 .. 16384 each.
 *   max_disp       D, the number of disparities searched, d in [0, D-1] (the range Gamma of
 *                  Sec. 2.1.1 with d_min = 0); 16 <= D <= 256, D % 16 == 0 (Sec. 3.1.2 caps D
 *                  at 256).
 *   census_w/_h    census window: 5 x 5 (24-bit descriptor) or 9 x 7 (62-bit), width first
 *                  (Sec. 2.2.1); with RES2TAC_NCC the NCC patch, 5 x 5 or 9 x 9.
 *   p1, p2         SGM penalties of Eq. (sgm_path), 0 <= p1 <= p2 <= 16384.
 *   num_paths      4 (LR, RL, TB, BT) or 8 (plus the four diagonals), Sec. 3.2.
 *   flags          RES2TAC_LR_CHECK | RES2TAC_MEDIAN | RES2TAC_EXACT_CC | RES2TAC_NCC (0 =
 *                  census cost, winner-takes-all only; RES2TAC_EXACT_CC changes D^R, so it
 *                  matters with RES2TAC_LR_CHECK).
 *   lr_threshold   largest accepted |D^L - D^R| of the left-right check (the paper uses 1). */
typedef struct res2tac_params {
  int32_t width, height;
  int32_t max_disp;
  int32_t census_w, census_h;
  int32_t p1, p2;
  int32_t num_paths;
  int32_t flags;
  int32_t lr_threshold;
} res2tac_params;

/* One stereo pair of a batch. Pointers are device memory owned by the caller. width, height
 * and max_disp override the context's values for this pair (same limits as res2tac_params);
 * the census window, penalties, path count, flags and threshold come from the context. */
typedef struct res2tac_pair {
  const uint8_t* left;
  const uint8_t* right;
  int64_t in_pitch; /* bytes, >= width */
  uint16_t* disp;
  int64_t out_pitch; /* bytes, >= 2 * width, even */
  int32_t width, height, max_disp;
  int32_t reserved; /* set to 0 */
} res2tac_pair;

/* Kernel configuration of a context. Every valid setting gives bit-identical results; only the
 * speed differs; 0 in a field selects its automatic value.
 * agg_dpl: disparities per lane of the row-path kernel (LR, RL): 2, 4 or 8 with
 *   D / agg_dpl <= 32.
 * agg_warps: warps per block of both aggregation kernels (1..16).
 * wta_chunk: pixels per block of the winner-takes-all / right-disparity kernel (64, 128 or
 *   256; one warp per pixel at a time).
 * shear_dpl: disparities per lane of the column / diagonal path kernel: 8, 16 or 32, with
 *   D % shear_dpl == 0.
 * row_mode: 1 = both directions of a row in one lane group, 2 = one direction per group.
 * shear_cpl: chains per lane of the column / diagonal path kernel (1 or 2).
 * cost_mode: kernel of the Hamming cost of the 9 x 7 census, Eq. (image_matching): 1 = population
 *   counts on the CUDA cores, 2 = the same integers as a dot product over the descriptor bits on
 *   the tensor cores (tcgen05, fp8 operands, exact fp32 accumulation; D = 64 or 128 only, other
 *   shapes and the 5 x 5 census use the population-count kernel). Its blocks take all of their
 *   SM's tensor memory, so they wait for tensor-core kernels of other libraries running
 *   concurrently on other streams.
 * row_cost: costs of the row-path kernel: 1 = read from the cost volume, 2 = recomputed from the
 *   census descriptors inside the walk (popcount of the XOR per step; census cost with
 *   row_mode 2 and D = 32 agg_dpl only, other settings read the volume).
 * Automatic values: agg_dpl 2 for D <= 64, 4 for D <= 128, else 8; agg_warps 2; wta_chunk 128;
 * shear_dpl 16; row_mode 2; shear_cpl 2 at D = 128, else 1; cost_mode 1 (measured faster);
 * row_cost 1. */
typedef struct res2tac_tuning {
  int32_t agg_dpl;
  int32_t agg_warps;
  int32_t wta_chunk;
  int32_t shear_dpl;
  int32_t row_mode;
  int32_t shear_cpl;
  int32_t cost_mode;
  int32_t row_cost;
} res2tac_tuning;

/* Validates *p, allocates the context's device scratch for a W x H x D pair on the current
 * device, and returns the handle in *out. The scratch (cost volume, aggregated
 * volume, intermediate maps, host staging) is owned by the context until res2tac_destroy.
 * Returns RES2TAC_EINVAL for invalid parameters, RES2TAC_ENOMEM if the scratch does not fit. */
int res2tac_create(const res2tac_params* p, res2tac_t* out);

/* Runs the whole pipeline of Sec. 2.1 on one rectified pair, asynchronously on stream s:
 * census (Sec. 2.2.1) -> Hamming cost, Eq. (image_matching) -> SGM aggregation over num_paths
 * paths, Eqs. (sgm_path), (sgm_path_aggr) -> WTA, Eq. (wta) -> approximate D^R,
 * Eq. (right_disparity) and left-right check, Eq. (LR_check) -> 3x3 median.
 * left/right: device images of the context's W x H, in_pitch bytes per row. disp: device
 * output, out_pitch bytes per row. The caller synchronises s before reading disp.
 * Intermediates stay in the context until the next call (see res2tac_debug_outputs). */
int res2tac_compute(res2tac_t h, const uint8_t* left, const uint8_t* right, int64_t in_pitch,
                    uint16_t* disp, int64_t out_pitch, res2tac_stream_t s);

/* Same pipeline on HOST buffers, end to end as the paper times it (upload, compute, download;
 * Sec. 3.3): left/right (host, in_pitch bytes per row) in, the map into disp (host, out_pitch
 * bytes per row), s synchronised before returning. When all three buffers are pinned host memory
 * the GPU can address (cudaHostAlloc / cudaHostRegister; on a Grace system they are reached over
 * NVLink-C2C), the kernels read the images and write the map in place; otherwise the images are
 * copied into the context's device staging and the map copied back. */
int res2tac_compute_host(res2tac_t h, const uint8_t* left, const uint8_t* right,
                         int64_t in_pitch, uint16_t* disp, int64_t out_pitch,
                         res2tac_stream_t s);

/* Pipeline with sub-pixel refinement (Sec. 2.1.3, "Subpixel disparity refinement"), the
 * configuration the paper labels "fine". Same stages as res2tac_compute; in addition each kept
 * pixel's parabola through the aggregated costs S(p, d-1), S(p, d), S(p, d+1) at the winning
 * d = D^L(p) moves d to the parabola's minimum (computed in the left-right / median stage),
 *   D^L_sub(p) = d + (S(d-1) - S(d+1)) / (2 (S(d-1) - 2 S(d) + S(d+1)))   for 1 <= d <= D-2,
 *   D^L_sub(p) = d                                                         for d = 0, D-1,
 * in fp32 with correctly rounded division and addition (S saturated at 65535 as in the uint16
 * volume). The left-right check compares the integer D^L with D^R as res2tac_compute does and
 * keeps D^L_sub; the 3x3 median then runs on the float values. disp: device float map,
 * out_pitch bytes per row (a multiple of 4, >= 4 * width), 4-byte aligned; a pixel rejected by
 * the check holds +infinity (the float counterpart of RES2TAC_INVALID, which sorts last in the
 * median exactly as 0xFFFF does). Asynchronous on s. */
int res2tac_compute_subpixel(res2tac_t h, const uint8_t* left, const uint8_t* right,
                             int64_t in_pitch, float* disp, int64_t out_pitch,
                             res2tac_stream_t s);

/* Writes the sub-pixel D^L map [H][W] (every pixel, before the left-right check and the median)
 * of the last compute call on this context into dl_sub (device, 4 B per pixel), from the D^L
 * and aggregated volume that call left in the context. Asynchronous on s. */
int res2tac_debug_subpixel(res2tac_t h, float* dl_sub, res2tac_stream_t s);

/* Rectification (Sec. 2.1.1: the pair is resampled through two maps from the camera calibration
 * so that epipolar lines lie on image rows; the paper computes the maps with OpenCV). Writes the
 * width x height image out (device, out_pitch bytes per row) from the raw image raw (device,
 * raw_w x raw_h, raw_pitch bytes per row) through the float maps mapx / mapy (device, width x
 * height, map_pitch bytes per row, a multiple of 4; 4-byte aligned), which give for each output
 * pixel its source coordinate (x right, y down, pixel centres at integers) in the raw image.
 * Each coordinate is put on a 1/32-pixel grid, X = rint(32 mapx) (ties to even; exact in
 * float), and the output is the bilinear interpolation with integer weights summing to 1024:
 *   (I(x0,y0)(32-fx)(32-fy) + I(x0+1,y0) fx(32-fy) + I(x0,y0+1)(32-fx) fy + I(x0+1,y0+1) fx fy
 *    + 512) >> 10,  x0 = floor(X / 32), fx = X - 32 x0 (y likewise),
 * where raw pixels outside the image read 0, and a coordinate that is not finite or has
 * |32 m| >= 2^24 gives 0. Sizes 1 .. 65536. Needs no context. Asynchronous on s. */
int res2tac_rectify(const uint8_t* raw, int64_t raw_pitch, int32_t raw_w, int32_t raw_h,
                    const float* mapx, const float* mapy, int64_t map_pitch, uint8_t* out,
                    int64_t out_pitch, int32_t width, int32_t height, res2tac_stream_t s);

/* Keeps the rectification maps of both cameras in the context (device copies of the W x H maps
 * mapx_l, mapy_l, mapx_r, mapy_r, map_pitch bytes per row, for raw images of raw_w x raw_h) for
 * res2tac_compute_raw. The first call allocates 16 B per pixel (not during stream capture); later
 * calls overwrite. The copies run on s: the caller's maps must stay valid until s has done them. */
int res2tac_set_rectification(res2tac_t h, const float* mapx_l, const float* mapy_l,
                              const float* mapx_r, const float* mapy_r, int64_t map_pitch,
                              int32_t raw_w, int32_t raw_h, res2tac_stream_t s);

/* res2tac_compute on a raw pair (device, raw_w x raw_h as set by res2tac_set_rectification,
 * raw_pitch bytes per row): rectifies both images into the context's staging (one launch) and
 * runs the pipeline on them. RES2TAC_EINVAL without maps. Asynchronous on s. */
int res2tac_compute_raw(res2tac_t h, const uint8_t* raw_left, const uint8_t* raw_right,
                        int64_t raw_pitch, uint16_t* disp, int64_t out_pitch,
                        res2tac_stream_t s);

/* Runs n independent pairs of uneven sizes as one batch on stream s (the paper processes one
 * pair at a time, Sec. 2.2; batching is this library's addition). The pairs are sorted by memory
 * footprint and cut into groups of at most 96 MB of cost and aggregated volumes (a larger pair is
 * a group of its own); each group runs the six stages as persistent kernels fed by device work
 * queues over its pairs, and groups rotate over four stream slots so consecutive groups
 * overlap. The whole batch is one CUDA graph, captured once per group count and replayed while
 * the capacities last (res2tac_last_launch_count: 6 per group). The context grows its batch
 * scratch when a larger batch arrives: that call allocates and must not be made during stream
 * capture. pairs: host array of n descriptors with device pointers. Results are bit-identical to
 * res2tac_compute on each pair alone. No block of the engine ever waits for another (work is
 * claimed with one atomic increment), so there is no device-side wait that could time out:
 * RES2TAC_ETIMEOUT is reserved and not returned. RES2TAC_EINVAL for an invalid pair, or for
 * RES2TAC_EXACT_CC / RES2TAC_NCC contexts (single pairs only). */
int res2tac_compute_batch(res2tac_t h, const res2tac_pair* pairs, int32_t n, res2tac_stream_t s);

/* Copies the intermediates of the last res2tac_compute on this context into caller buffers
 * (device pointers; any may be NULL): cost [H][W][D] uint8 (Eq. image_matching, 255 where
 * x - d < 0), agg [H][W][D] uint16 (S-bar of Eq. sgm_path_aggr, saturated at 65535),
 * dl / dr [H][W] uint16 (Eq. wta; Eq. right_disparity, or the exact D^R with
 * RES2TAC_EXACT_CC), mask [H][W] uint8 (1 where the
 * left-right check kept the pixel, all 1 without RES2TAC_LR_CHECK). Asynchronous on s. */
int res2tac_debug_outputs(res2tac_t h, uint8_t* cost, uint16_t* agg, uint16_t* dl, uint16_t* dr,
                          uint8_t* mask, res2tac_stream_t s);

/* Device bytes res2tac_create allocates for *p (0 if *p is invalid); for admission control. */
size_t res2tac_workspace_bytes(const res2tac_params* p);

/* Device bytes a batch of n pairs needs on top of the context (0 if a pair is invalid). */
size_t res2tac_batch_workspace_bytes(const res2tac_params* p, const res2tac_pair* pairs,
                                     int32_t n);

/* Pre-allocates the context's batch engine for batches of at most max_pairs pairs whose
 * res2tac_batch_workspace_bytes is at most scratch_bytes, so that such batches allocate nothing
 * (a serving loop reserves once, then admits work by its own memory accounting). Grow-only;
 * synchronises the device when it grows. RES2TAC_ENOMEM if the memory is not available. */
int res2tac_batch_reserve(res2tac_t h, size_t scratch_bytes, int32_t max_pairs);

/* Reads / sets the kernel configuration (RES2TAC_EINVAL for a setting the context's D cannot
 * use). res2tac_autotune times every valid setting on the given device pair (left, right,
 * in_pitch as for res2tac_compute, output into disp), then the fastest one with the other cost
 * kernel where the shape has two, keeps the fastest in the context and returns it in *best; it
 * synchronises s. */
int res2tac_get_tuning(res2tac_t h, res2tac_tuning* t);
int res2tac_set_tuning(res2tac_t h, const res2tac_tuning* t);
int res2tac_autotune(res2tac_t h, const uint8_t* left, const uint8_t* right, int64_t in_pitch,
                     uint16_t* disp, int64_t out_pitch, res2tac_stream_t s,
                     res2tac_tuning* best);

/* Kernel settings of the batch engine for one bucket of pairs (not in the paper: batching is
 * this library's addition). A pair's bucket is its D together with its size class (large = 1
 * when width * height >= 2^18 pixels, else 0); every pair of a bucket runs with the bucket's
 * settings, which change the schedule only, never the results (bit-identical maps).
 *   row_dpl    disparities per lane of the row paths (LR, RL): 2, 4 or 8, D / row_dpl <= 32
 *   shear_dpl, shear_cpl  disparities and chains per lane of the column and diagonal paths:
 *              (16, 1) or (16, 2)
 *   wta_px     pixels per WTA / right-disparity tile: 64, 128 or 256 (fewer when the tile's sums
 *              would exceed 64 KB)
 * Defaults: row_dpl 2 / 4 / 8 for D <= 64 / <= 128 / larger, (16, 1), 128. */
typedef struct res2tac_batch_tuning {
  int32_t max_disp, large;
  int32_t row_dpl, shear_dpl, shear_cpl, wta_px;
} res2tac_batch_tuning;

/* Sets the batch settings of n buckets (each entry names its bucket by max_disp and large).
 * RES2TAC_EINVAL (nothing changed) if an entry is invalid for its D. Applies from the next
 * res2tac_compute_batch; the first change that needs more shared memory than the captured graph
 * recaptures it there. */
int res2tac_set_batch_tuning(res2tac_t h, const res2tac_batch_tuning* t, int32_t n);

/* Reads the batch settings of the bucket named by t->max_disp and t->large into *t. */
int res2tac_get_batch_tuning(res2tac_t h, res2tac_batch_tuning* t);

/* Autotuner of the batch engine: for the buckets the n pairs fall into (largest total work
 * first; each starts from the defaults) it times the whole batch (res2tac_compute_batch on stream s, median of 3 runs after one
 * warm-up) for each candidate of one setting at a time - row_dpl, then (shear_dpl, shear_cpl),
 * then wta_px - keeping the fastest, and leaves the chosen table in the context. It writes up to
 * cap entries of the buckets it tuned into table (count into *count) and the batch times before
 * and after into *ms_default and *ms_tuned (any of these may be NULL). The pairs' maps are
 * written as by res2tac_compute_batch. Synchronises s; allocates the batch scratch as
 * res2tac_compute_batch does. */
int res2tac_autotune_batch(res2tac_t h, const res2tac_pair* pairs, int32_t n, res2tac_stream_t s,
                           res2tac_batch_tuning* table, int32_t cap, int32_t* count,
                           float* ms_default, float* ms_tuned);

/* Number of kernel launches the last res2tac_compute / res2tac_compute_batch issued. */
int res2tac_last_launch_count(res2tac_t h);

/* Per-stage timing. With profiling enabled, res2tac_compute records a CUDA event on the caller's
 * stream before and after each stage. res2tac_stage_times waits for the last call and writes up
 * to n durations in milliseconds: [0] census + cost (+ clearing of the aggregated volume),
 * [1] path aggregation, [2] WTA + right-disparity keys, [3] LR check + median. With
 * RES2TAC_EXACT_CC, [0] .. [2] add up both passes (and [0] the flip of the pair). */
int res2tac_set_profiling(res2tac_t h, int enable);
int res2tac_stage_times(res2tac_t h, float* ms, int n);

/* No-allocation variant of res2tac_compute. The paper has no counterpart: it is an addition for
 * callers that must not allocate device memory while they run, for example an onboard stereo loop
 * that is only allowed to allocate at start-up, a plugin whose host framework owns every byte of
 * device memory, or a latency-critical loop that cannot take the device-wide synchronisation a
 * cudaMalloc / cudaFree may cause. It needs no context and calls no cudaMalloc, cudaFree or
 * other allocating routine.
 * It runs the same pipeline as res2tac_compute on stream s, for the problem *p, with left /
 * right / disp and the pitches as in res2tac_compute. Its scratch (cost volume, aggregated
 * volume, intermediate maps) is one fixed device array of
 * RES2TAC_STATIC_SCRATCH_BYTES compiled into the library; every GPU that loads the library holds
 * that array until the process exits.
 * Size limit: a problem whose scratch does not fit the array (3 B per W*H*D plus 25 B per pixel,
 * 5 B per W*H*D when num_paths * (255 + p2) > 65535, 4 B more per pixel with RES2TAC_EXACT_CC,
 * 24 B more per pixel and 2 KB with RES2TAC_NCC)
 * is rejected with RES2TAC_ENOMEM and a
 * message giving both sizes. 640 x 480 with D = 64 fits with 16-bit sums
 * (num_paths * (255 + p2) <= 65535: about 67 MB) but not with 32-bit ones (about 106 MB).
 * Set-up: the first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * Sharing: every call in the process uses the same array, which keeps the contents of the last
 * call; each call clears what must start at zero (the aggregated volume) itself. Calls that
 * overlap on the GPU (on other streams, or from other host threads) race on the array, so the
 * caller must serialise them. */
#define RES2TAC_STATIC_SCRATCH_BYTES ((size_t)80 << 20)
int res2tac_compute_static(const res2tac_params* p, const uint8_t* left, const uint8_t* right,
                           int64_t in_pitch, uint16_t* disp, int64_t out_pitch,
                           res2tac_stream_t s);

/* Frees the context and its scratch. NULL-safe. The caller makes sure no work on the context
 * is still running. */
void res2tac_destroy(res2tac_t h);

const char* res2tac_strerror(int code);
const char* res2tac_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RES2TAC_H_ */
