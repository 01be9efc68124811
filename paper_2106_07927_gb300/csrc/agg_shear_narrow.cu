// Sheared-column aggregation kernels with uint16 sums, plain and batch variants.
#include "agg_units.cuh"

namespace r2t {
template cudaError_t launch_shear<false>(const Problem&, const Method&, const Tuning&, cudaStream_t);
template const void* batch_shear_kernel_fn<false>();
}  // namespace r2t
