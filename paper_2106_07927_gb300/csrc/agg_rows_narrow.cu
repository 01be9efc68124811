// Row-path aggregation kernels (LR, RL) with uint16 sums, plain and batch variants.
#include "agg_units.cuh"

namespace r2t {
template cudaError_t launch_rows<false>(const Problem&, const Method&, const Tuning&, cudaStream_t);
template const void* batch_row_kernel_fn<false>();
}  // namespace r2t
