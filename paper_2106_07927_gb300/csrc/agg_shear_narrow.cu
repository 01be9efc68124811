// Sheared-column aggregation kernels with uint16 sums, plain launches (the persistent batch
// variant is its own unit, agg_shear_batch_narrow.cu, so the two compile in parallel).
#include "agg_units.cuh"

namespace r2t {
template cudaError_t launch_shear<false>(const Problem&, const Method&, const Tuning&, cudaStream_t);
}  // namespace r2t
