// FP32 instantiation of the kernels and launchers (mixed-precision V-cycle).
#include "ops_impl.cuh"
namespace bh {
template struct Ops<float>;
}
