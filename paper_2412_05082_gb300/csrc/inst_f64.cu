// FP64 instantiation of the kernels and launchers.
#include "ops_impl.cuh"
namespace bh {
template struct Ops<double>;
}
