// Host launchers of the compensated defect (ffsweep.cuh): the sweeps of
// apply() with double-float intermediates, from the FP32 tables' hi + lo parts.
// Instantiated per degree in defect_ff_k*.cu (one translation unit each,
// compiled in parallel); dispatched in defect_ff.cu.
#pragma once
#include "ops_impl.cuh"

namespace bh {

template <int K, int KIND>
inline cudaError_t launch_ff(const FfTab<K>& tab, const FfSweepArgs& a, cudaStream_t st) {
  const int block = kFfBlock;
  ff_sweep_kernel<K, KIND><<<grid_for(ff_sweep_threads(KIND, a.lines, a.N), block), block, 0, st>>>(
      tab, a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <int K>
cudaError_t defect_ff_k(const void* tabp, const LevelGeom& g, const float* x,
                               const double* b, double* r, double scale, void* scratch,
                               cudaStream_t st) {
  const auto* h = static_cast<const HostTables<float, K>*>(tabp);
  if (!h->ff) return cudaErrorInvalidValue;
  const FfTab<K>& tab = *h->ff;
  FfSweepArgs a{};
  a.d = g.d;
  a.N = g.N;
  a.n = g.n;
  a.lines = g.nd / g.n;
  a.scale = scale;
  a.b = b;
  a.r = r;
  float2* s[6];
  for (int i = 0; i < 6; ++i) s[i] = static_cast<float2*>(scratch) + (int64_t)i * g.nd;
  a.axis = 0;
  a.stride = 1;
  a.x = x;
  for (int i = 0; i < 3; ++i) a.out[i] = s[i];
  cudaError_t e = launch_ff<K, 0>(tab, a, st);
  if (e != cudaSuccess) return e;
  a.axis = 1;
  a.stride = g.n;
  for (int i = 0; i < 3; ++i) a.in[i] = s[i];
  if (g.d == 2) return launch_ff<K, 2>(tab, a, st);
  for (int i = 0; i < 3; ++i) a.out[i] = s[3 + i];
  if ((e = launch_ff<K, 1>(tab, a, st)) != cudaSuccess) return e;
  a.axis = 2;
  a.stride = (int64_t)g.n * g.n;
  for (int i = 0; i < 3; ++i) a.in[i] = s[3 + i];
  return launch_ff<K, 3>(tab, a, st);
}

template <int K>
const void* ff_dev_k(const void* tabp) {
  return static_cast<const HostTables<float, K>*>(tabp)->dev_ff;
}

// the batched form's per-degree list kernels (kind 0: split of x, 2: residual)
template <int K>
const void* ff_list_kernel_k(int kind) {
  return kind == 0 ? (const void*)ff_sweep_list_kernel<K, 0> : (const void*)ff_sweep_list_kernel<K, 2>;
}

#define BH_FF_EXTERN(KK)                                                                          \
  extern template cudaError_t defect_ff_k<KK>(const void*, const LevelGeom&, const float*,         \
                                              const double*, double*, double, void*, cudaStream_t); \
  extern template const void* ff_list_kernel_k<KK>(int);
#define BH_FF_INSTANTIATE(KK)                                                                    \
  template cudaError_t defect_ff_k<KK>(const void*, const LevelGeom&, const float*,               \
                                       const double*, double*, double, void*, cudaStream_t);      \
  template const void* ff_list_kernel_k<KK>(int);

}  // namespace bh
