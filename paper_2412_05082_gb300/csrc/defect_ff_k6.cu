// Instantiation unit: the compensated defect's kernels for degree 6.
#include "defect_ff.cuh"

namespace bh {
BH_FF_INSTANTIATE(6)
}  // namespace bh
