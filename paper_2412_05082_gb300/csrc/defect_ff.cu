// Dispatch of the compensated defect by degree (defect_ff.cuh; kernels in
// defect_ff_k*.cu).
#include "defect_ff.cuh"

namespace bh {

BH_FF_EXTERN(2)
BH_FF_EXTERN(3)
BH_FF_EXTERN(4)
BH_FF_EXTERN(5)
BH_FF_EXTERN(6)
BH_FF_EXTERN(7)

cudaError_t defect_ff(const void* tab32, const LevelGeom& g, const float* x, const double* b,
                      double* r, double scale, void* scratch, cudaStream_t st) {
#define BH_CALL(KK) return defect_ff_k<KK>(tab32, g, x, b, r, scale, scratch, st)
  BH_K_DISPATCH(g.k, BH_CALL)
#undef BH_CALL
  return cudaErrorInvalidValue;
}

const void* ff_device_tables(const void* tab32, int k) {
  switch (k) {
    case 2: return ff_dev_k<2>(tab32);
    case 3: return ff_dev_k<3>(tab32);
    case 4: return ff_dev_k<4>(tab32);
    case 5: return ff_dev_k<5>(tab32);
    case 6: return ff_dev_k<6>(tab32);
    case 7: return ff_dev_k<7>(tab32);
  }
  return nullptr;
}

const void* ff_list_kernel(int k, int kind) {
  switch (k) {
    case 2: return ff_list_kernel_k<2>(kind);
    case 3: return ff_list_kernel_k<3>(kind);
    case 4: return ff_list_kernel_k<4>(kind);
    case 5: return ff_list_kernel_k<5>(kind);
    case 6: return ff_list_kernel_k<6>(kind);
    case 7: return ff_list_kernel_k<7>(kind);
  }
  return nullptr;
}

}  // namespace bh
