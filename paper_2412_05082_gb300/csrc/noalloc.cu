// bh_apply_A_noalloc: y = A_l x without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// operator: a plugin running inside a host framework that owns every device
// allocation and forbids its plugins to allocate while executing, or a
// latency-critical loop that cannot afford cudaMalloc's implicit device
// synchronization.  This entry point serves them.  It needs no context and no
// heap: the kernel-parameter tables are built by the heap-free 1D core into
// static host storage (once per degree and penalty, then reused), and the
// sweep intermediates (three arrays of n^d values in 2D, six in 3D) live in
// the file-scope device array below, which every GPU that loads the library
// holds (64 MiB) until the process exits.
//
// Sharing rules: every call uses the same array.  Calls whose kernels could
// overlap on the GPU (two streams, or two host threads) race on it; callers
// must serialize them.  The array keeps the last call's contents; nothing in
// it has to start at zero, because each call writes every scratch value it
// later reads (the x-split pass writes all three arrays before the next pass
// reads them).
//
// Set-up: the first call on a device looks up the device address of the array
// with cudaGetSymbolAddress while that device is current (the host-side name
// of the array is only a stand-in, not a device address) and keeps it for the
// later calls on that device.  Make that first call before any stream capture.
// A cudaDeviceReset of that device invalidates the kept address, and the
// library does not notice it: do not reset a device between calls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "biharm.h"
#include "kernels.cuh"
#include "line1d.h"

namespace bh {
void set_last_error(const std::string& msg);  // api.cu
}

namespace {

using namespace bh;

constexpr int64_t kScratchValues = 8 * 1024 * 1024;  // 8 Mi doubles = 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[kScratchValues];

double* g_scratch_dev[kMaxDevices] = {};  // device address per device ordinal
std::mutex g_scratch_mutex;

bh_status err(bh_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

// ---- host tables without heap allocation (cells of size 1) ------------------
// Built by the heap-free 1D core (line1d.h) into static host storage, and
// cached per degree for the last penalty gamma: both are guarded by
// g_scratch_mutex, so a call reuses the table of the previous call with the
// same (degree, gamma) and only a change of gamma rebuilds it.
constexpr int kLineNodes = line1d::kMaxLineNodes;
double g_line[6][kLineNodes * kLineNodes];  // M, L, B of the 7-cell and the 2-cell line
double g_class[3][(3 * kMaxK + 1) * (4 * kMaxK + 1)];

template <int K>
struct CachedTab {
  double gamma = 0.0;  // 0: not built yet
  OpTab<double, K> tab;
};
template <int K>
CachedTab<K> g_tab;

// The operator's row-class tables for (K, gamma); g_scratch_mutex held.
template <int K>
const OpTab<double, K>& optab(double gamma) {
  CachedTab<K>& c = g_tab<K>;
  if (c.gamma != gamma) {
    const int n7 = 7 * K + 1, n2 = 2 * K + 1, bw = 4 * K + 1;
    line1d::line_matrices(K, gamma, 7, g_line[0], g_line[1], g_line[2], n7);
    line1d::line_matrices(K, gamma, 2, g_line[3], g_line[4], g_line[5], n2);
    line1d::class_tables(K, g_line[0], g_line[1], g_line[2], n7, g_line[3], g_line[4], g_line[5],
                         n2, g_class[0], g_class[1], g_class[2]);
    for (int cl = 0; cl < 3 * K + 1; ++cl)
      for (int t = 0; t < bw; ++t) {
        c.tab.M[cl][t] = g_class[0][cl * bw + t];
        c.tab.L[cl][t] = g_class[1][cl * bw + t];
        c.tab.B[cl][t] = g_class[2][cl * bw + t];
      }
    c.gamma = gamma;
  }
  return c.tab;
}

template <int K, int KIND>
cudaError_t sweep(const OpTab<double, K>& tab, const SweepArgs<double>& a, cudaStream_t st) {
  const int block = 128;
  const unsigned grid = (unsigned)((sweep_launch_threads(KIND, a.lines, a.N) + block - 1) / block);
  sweep_kernel<double, K, KIND><<<grid, block, 0, st>>>(tab, a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

// the sweeps of y = A_l x; g_scratch_mutex held (the cached table)
template <int K>
cudaError_t apply_static(int d, int N, double gamma, const double* x, double* y, double* scr,
                         cudaStream_t st) {
  const OpTab<double, K>& tab = optab<K>(gamma);
  const int n = K * N - 1;
  const int64_t nd = d == 2 ? (int64_t)n * n : (int64_t)n * n * n;
  SweepArgs<double> a{};
  a.d = d;
  a.N = N;
  a.n = n;
  a.lines = nd / n;
  a.scale = std::pow((double)N, 4 - d);  // A_l = h^(d-4) A_ref
  a.mode = kStore;
  double* s[6];
  for (int i = 0; i < 6; ++i) s[i] = scr + i * nd;
  a.axis = 0;
  a.stride = 1;
  a.in[0] = x;
  a.out[0] = s[0];
  a.out[1] = s[1];
  a.out[2] = s[2];
  cudaError_t e = sweep<K, 0>(tab, a, st);
  if (e != cudaSuccess) return e;
  a.in[0] = s[0];
  a.in[1] = s[1];
  a.in[2] = s[2];
  a.axis = 1;
  a.stride = n;
  if (d == 2) {
    a.out[0] = y;
    return sweep<K, 2>(tab, a, st);
  }
  a.out[0] = s[3];
  a.out[1] = s[4];
  a.out[2] = s[5];
  e = sweep<K, 1>(tab, a, st);
  if (e != cudaSuccess) return e;
  a.in[0] = s[3];
  a.in[1] = s[4];
  a.in[2] = s[5];
  a.out[0] = y;
  a.axis = 2;
  a.stride = (int64_t)n * n;
  return sweep<K, 3>(tab, a, st);
}

}  // namespace

extern "C" bh_status bh_apply_A_noalloc(int dim, int degree, int level, double gamma,
                                        const double* x_dev, double* y_dev, void* stream) {
  if (dim != 2 && dim != 3) return err(BH_EINVAL, "bh_apply_A_noalloc: dim must be 2 or 3");
  if (degree < 2 || degree > kMaxK)
    return err(BH_EINVAL, "bh_apply_A_noalloc: degree must be in 2..7");
  if (level < 1 || level > 14) return err(BH_EINVAL, "bh_apply_A_noalloc: level must be in 1..14");
  if (!x_dev || !y_dev || x_dev == y_dev)
    return err(BH_EINVAL, "bh_apply_A_noalloc: null or aliased vectors");
  const int N = 1 << level, n = degree * N - 1;
  const int64_t nd = dim == 2 ? (int64_t)n * n : (int64_t)n * n * n;
  const int64_t need = (dim == 2 ? 3 : 6) * nd;
  if (need > kScratchValues) {
    static thread_local char msg[256];
    std::snprintf(msg, sizeof(msg),
                  "bh_apply_A_noalloc: %lld unknowns need %lld scratch values, above the "
                  "static maximum of %lld (at most %lld unknowns in %dD)",
                  (long long)nd, (long long)need, (long long)kScratchValues,
                  (long long)(kScratchValues / (dim == 2 ? 3 : 6)), dim);
    return err(BH_EINVAL, msg);
  }
  if (!(gamma > 0.0)) gamma = degree * (degree + 1.0);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return err(BH_ECUDA, "bh_apply_A_noalloc: no usable current CUDA device");
  }
  // one lock for the device address, the cached host table and the launches
  // (the launch copies the table into its kernel parameters)
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_dev[dev]) {  // once per device, with that device current
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return err(BH_ECUDA, "bh_apply_A_noalloc: cudaGetSymbolAddress of the scratch array failed");
    }
    g_scratch_dev[dev] = static_cast<double*>(p);
  }
  double* scr = g_scratch_dev[dev];
  const cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaErrorInvalidValue;
  switch (degree) {
    case 2: e = apply_static<2>(dim, N, gamma, x_dev, y_dev, scr, st); break;
    case 3: e = apply_static<3>(dim, N, gamma, x_dev, y_dev, scr, st); break;
    case 4: e = apply_static<4>(dim, N, gamma, x_dev, y_dev, scr, st); break;
    case 5: e = apply_static<5>(dim, N, gamma, x_dev, y_dev, scr, st); break;
    case 6: e = apply_static<6>(dim, N, gamma, x_dev, y_dev, scr, st); break;
    case 7: e = apply_static<7>(dim, N, gamma, x_dev, y_dev, scr, st); break;
  }
  if (e != cudaSuccess) {
    set_last_error(std::string("bh_apply_A_noalloc: ") + cudaGetErrorString(e));
    return BH_ECUDA;
  }
  return BH_OK;
}
