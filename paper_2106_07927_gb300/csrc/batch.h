// Batch engine: many pairs of uneven W, H, D in persistent kernels fed by device work queues.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "batch_dev.cuh"
#include "common.cuh"

namespace r2t {

struct BatchEngine;

// Device bytes of the descriptor tables for n pairs (upper bound, excluding per-pair scratch).
size_t batch_fixed_bytes(int n);

// Creates or grows the engine so it holds scratch_bytes of per-pair scratch and n pairs.
// Returns 0, -2 when device memory is short, -3 on another CUDA error.
int batch_reserve(BatchEngine** e, size_t scratch_bytes, int n);

// Base of the per-pair scratch (valid after batch_reserve).
char* batch_scratch(BatchEngine* e);

// Runs the batch on stream s: uploads the descriptors, clears the queue counters and replays
// the captured graph (capturing it first when the capacities changed). Returns 0 or -3.
int batch_run(BatchEngine* e, const Problem* probs, int n, const Method& mt, cudaStream_t s,
              int* launches);

// Kernel settings per bucket of pairs (tune_bucket: D / 16 and the size class): the defaults,
// their validity, and the engine's table (set returns -1 for an invalid setting).
BatchTune batch_default_tune(int bucket);
bool batch_tune_valid(int bucket, const BatchTune& t);
int batch_set_tune(BatchEngine* e, int bucket, const BatchTune& t);
BatchTune batch_get_tune(BatchEngine* e, int bucket);

const char* batch_error(BatchEngine* e);
void batch_destroy(BatchEngine* e);

}  // namespace r2t
