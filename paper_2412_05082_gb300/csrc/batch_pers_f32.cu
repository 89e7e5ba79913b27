// Instantiation unit: the batched form's persistent V-cycle kernel in FP32 (the FP32 V-cycle with FP64 defects).
#include "batch_dev.cuh"

namespace bh {
namespace bdev {
const void* vcycle_persistent_kernel_f32() { return vcycle_persistent_kernel_table<float>(); }
}  // namespace bdev
}  // namespace bh
