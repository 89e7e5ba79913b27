// Instantiation unit: the batched form's per-degree colored-MVS kernels in FP32.
#include "batch_dev.cuh"

namespace bh {
namespace bdev {
const void* mvs2_batch_kernel_f32(int k) { return mvs2_batch_kernel_table<float>(k); }
}  // namespace bdev
}  // namespace bh
