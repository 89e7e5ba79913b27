// Instantiation unit: the compensated defect's kernels for degree 5.
#include "defect_ff.cuh"

namespace bh {
BH_FF_INSTANTIATE(5)
}  // namespace bh
