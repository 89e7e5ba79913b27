// Instantiation unit: the compensated defect's kernels for degrees 2, 3, 4.
#include "defect_ff.cuh"

namespace bh {
BH_FF_INSTANTIATE(2)
BH_FF_INSTANTIATE(3)
BH_FF_INSTANTIATE(4)
}  // namespace bh
