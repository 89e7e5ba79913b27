// Instantiation unit: the compensated defect's kernels for degree 7.
#include "defect_ff.cuh"

namespace bh {
BH_FF_INSTANTIATE(7)
}  // namespace bh
