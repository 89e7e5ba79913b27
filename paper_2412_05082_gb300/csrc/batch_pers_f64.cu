// Instantiation unit: the batched form's persistent V-cycle kernel in FP64.
#include "batch_dev.cuh"

namespace bh {
namespace bdev {
const void* vcycle_persistent_kernel_f64() { return vcycle_persistent_kernel_table<double>(); }
}  // namespace bdev
}  // namespace bh
