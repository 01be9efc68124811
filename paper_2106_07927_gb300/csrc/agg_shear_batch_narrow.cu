// Persistent batch variant of the sheared-column aggregation kernel with uint16 sums.
#include "agg_units.cuh"

namespace r2t {
template const void* batch_shear_kernel_fn<false>();
}  // namespace r2t
