// Sheared-column aggregation kernels with uint32 sums, plain and batch variants.
#include "agg_units.cuh"

namespace r2t {
template cudaError_t launch_shear<true>(const Problem&, const Method&, const Tuning&, cudaStream_t);
template const void* batch_shear_kernel_fn<true>();
}  // namespace r2t
