// bh_apply_A_noalloc: y = A_l x without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// operator: a plugin running inside a host framework that owns every device
// allocation and forbids its plugins to allocate while executing, or a
// latency-critical loop that cannot afford cudaMalloc's implicit device
// synchronization.  This entry point serves them.  It needs no context: the
// kernel-parameter tables are built on the host stack for every call, and the
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
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "biharm.h"
#include "kernels.cuh"

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
constexpr int kMaxNodes = 7 * kMaxK + 1;

void legendre(int n, double x, double& pn, double& pm) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { pn = 1.0; pm = 0.0; return; }
  for (int m = 1; m < n; ++m) {
    const double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
    p0 = p1;
    p1 = p2;
  }
  pn = p1;
  pm = p0;
}

void gll(int k, double* z) {  // Gauss-Lobatto-Legendre points on [0, 1]
  z[0] = -1.0;
  z[k] = 1.0;
  for (int j = 1; j < k; ++j) {
    double t = -std::cos(M_PI * j / k);
    for (int it = 0; it < 100; ++it) {
      double pn, pm;
      legendre(k, t, pn, pm);
      const double d1 = k * (t * pn - pm) / (t * t - 1.0);
      const double d2 = (2.0 * t * d1 - k * (k + 1.0) * pn) / (1.0 - t * t);
      const double dt = d1 / d2;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    z[j] = t;
  }
  for (int j = 0; j <= k; ++j) z[j] = 0.5 * (z[j] + 1.0);
  z[0] = 0.0;
  z[k] = 1.0;
}

void gauss(int q, double* x, double* w) {  // Gauss-Legendre on [0, 1]
  for (int j = 0; j < q; ++j) {
    double t = std::cos(M_PI * (j + 0.75) / (q + 0.5)), d1 = 1.0, pn, pm;
    for (int it = 0; it < 100; ++it) {
      legendre(q, t, pn, pm);
      d1 = q * (t * pn - pm) / (t * t - 1.0);
      const double dt = pn / d1;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    legendre(q, t, pn, pm);
    d1 = q * (t * pn - pm) / (t * t - 1.0);
    x[j] = 0.5 * (t + 1.0);
    w[j] = 1.0 / ((1.0 - t * t) * d1 * d1);
  }
}

double lag(const double* z, int n, int i, double x, int deriv) {  // Lagrange basis derivative
  auto fac = [&](int j) { return (x - z[j]) / (z[i] - z[j]); };
  double s = 0.0;
  if (deriv == 0) {
    s = 1.0;
    for (int j = 0; j < n; ++j)
      if (j != i) s *= fac(j);
  } else if (deriv == 1) {
    for (int m = 0; m < n; ++m) {
      if (m == i) continue;
      double p = 1.0 / (z[i] - z[m]);
      for (int j = 0; j < n; ++j)
        if (j != i && j != m) p *= fac(j);
      s += p;
    }
  } else {
    for (int m = 0; m < n; ++m) {
      if (m == i) continue;
      for (int l = 0; l < n; ++l) {
        if (l == i || l == m) continue;
        double p = 1.0 / ((z[i] - z[m]) * (z[i] - z[l]));
        for (int j = 0; j < n; ++j)
          if (j != i && j != m && j != l) p *= fac(j);
        s += p;
      }
    }
  }
  return s;
}

// Global 1D M, L, B on a line of `cells` unit cells (Eq. (matrix1d) plus the
// face points of Eq. (ev)), nodes 0..k*cells, leading dimension kMaxNodes.
void line_1d(int k, double gamma, int cells, double (*M)[kMaxNodes], double (*L)[kMaxNodes],
             double (*B)[kMaxNodes]) {
  double z[kMaxK + 1], x[kMaxK + 2], w[kMaxK + 2];
  gll(k, z);
  gauss(k + 2, x, w);
  const int c1 = k + 1, n = k * cells + 1;
  double cM[kMaxK + 1][kMaxK + 1] = {}, cL[kMaxK + 1][kMaxK + 1] = {}, cB[kMaxK + 1][kMaxK + 1] = {};
  for (int q = 0; q < k + 2; ++q)
    for (int i = 0; i < c1; ++i)
      for (int j = 0; j < c1; ++j) {
        cM[i][j] += w[q] * lag(z, c1, i, x[q], 0) * lag(z, c1, j, x[q], 0);
        cL[i][j] += w[q] * lag(z, c1, i, x[q], 1) * lag(z, c1, j, x[q], 1);
        cB[i][j] += w[q] * lag(z, c1, i, x[q], 2) * lag(z, c1, j, x[q], 2);
      }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) M[i][j] = L[i][j] = B[i][j] = 0.0;
  for (int c = 0; c < cells; ++c)
    for (int i = 0; i < c1; ++i)
      for (int j = 0; j < c1; ++j) {
        M[k * c + i][k * c + j] += cM[i][j];
        L[k * c + i][k * c + j] += cL[i][j];
        B[k * c + i][k * c + j] += cB[i][j];
      }
  for (int f = 0; f <= cells; ++f) {  // jump = sum of outward derivatives, mean = half sum
    int ids[2 * kMaxK + 2], cnt = 0;
    double J[2 * kMaxK + 2], Mu[2 * kMaxK + 2];
    const bool interior = f > 0 && f < cells;
    if (f > 0)
      for (int i = 0; i < c1; ++i, ++cnt) {
        ids[cnt] = k * (f - 1) + i;
        J[cnt] = lag(z, c1, i, 1.0, 1);
        Mu[cnt] = lag(z, c1, i, 1.0, 2) * (interior ? 0.5 : 1.0);
      }
    if (f < cells)
      for (int i = 0; i < c1; ++i, ++cnt) {
        ids[cnt] = k * f + i;
        J[cnt] = -lag(z, c1, i, 0.0, 1);
        Mu[cnt] = lag(z, c1, i, 0.0, 2) * (interior ? 0.5 : 1.0);
      }
    for (int a = 0; a < cnt; ++a)
      for (int b = 0; b < cnt; ++b)
        B[ids[a]][ids[b]] += gamma * J[a] * J[b] - J[a] * Mu[b] - Mu[a] * J[b];
  }
}

// band row t = -2k..2k of row g of a line of `cells` cells; ghost columns zero
template <int K>
void class_row(double (*P)[kMaxNodes], int cells, int g, double* row) {
  for (int t = -2 * K; t <= 2 * K; ++t) {
    const int col = g + t;
    row[t + 2 * K] = (col >= 1 && col <= K * cells - 1) ? P[g][col] : 0.0;
  }
}

template <int K>
void build_optab(double gamma, OpTab<double, K>& tab) {
  static_assert(7 * K + 1 <= kMaxNodes, "line too long");
  double M[kMaxNodes][kMaxNodes], L[kMaxNodes][kMaxNodes], B[kMaxNodes][kMaxNodes];
  line_1d(K, gamma, 7, M, L, B);  // canonical rows 3K..4K-1, left 1..K, right 6K..7K-1
  for (int q = 0; q < K; ++q) {
    class_row<K>(M, 7, 3 * K + q, tab.M[q]);
    class_row<K>(L, 7, 3 * K + q, tab.L[q]);
    class_row<K>(B, 7, 3 * K + q, tab.B[q]);
  }
  for (int g = 1; g <= K; ++g) {
    class_row<K>(M, 7, g, tab.M[K + g - 1]);
    class_row<K>(L, 7, g, tab.L[K + g - 1]);
    class_row<K>(B, 7, g, tab.B[K + g - 1]);
  }
  for (int g = 6 * K; g <= 7 * K - 1; ++g) {
    class_row<K>(M, 7, g, tab.M[2 * K + g - 6 * K]);
    class_row<K>(L, 7, g, tab.L[2 * K + g - 6 * K]);
    class_row<K>(B, 7, g, tab.B[2 * K + g - 6 * K]);
  }
  line_1d(K, gamma, 2, M, L, B);  // N = 2: the middle vertex touches both faces
  class_row<K>(M, 2, K, tab.M[3 * K]);
  class_row<K>(L, 2, K, tab.L[3 * K]);
  class_row<K>(B, 2, K, tab.B[3 * K]);
}

template <int K, int KIND>
cudaError_t sweep(const OpTab<double, K>& tab, const SweepArgs<double>& a, cudaStream_t st) {
  const int block = 128;
  const unsigned grid = (unsigned)((a.lines * a.N + block - 1) / block);
  sweep_kernel<double, K, KIND><<<grid, block, 0, st>>>(tab, a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

template <int K>
cudaError_t apply_static(int d, int N, double gamma, const double* x, double* y, double* scr,
                         cudaStream_t st) {
  OpTab<double, K> tab;
  build_optab<K>(gamma, tab);
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
  double* scr;
  {
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
    scr = g_scratch_dev[dev];
  }
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
