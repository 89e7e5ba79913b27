// Vector kernels of the FP64 GMRES driver and the precision conversions.
#include <cuda_runtime.h>

#include "ops.h"

namespace bh {

std::atomic<long long> g_kernel_launches{0};

namespace {

inline unsigned grid1d(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;  // grid-stride beyond 32 waves of 152 SMs
  return (unsigned)(g < 1 ? 1 : g);
}

inline cudaError_t launched() {
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

// block partial sums of x . y over a grid-stride range (fixed grid => fixed order)
__global__ void __launch_bounds__(256) dot_partial_kernel(const double* __restrict__ x,
                                                          const double* __restrict__ y, int64_t n,
                                                          double* partials) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    partials[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) dot_final_kernel(const double* partials, int m,
                                                        double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += partials[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    *out = t;
  }
}

__global__ void axpy_kernel(double* y, double a, const double* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

__global__ void axpy_dev_kernel(double* y, const double* a, double sign,
                                const double* __restrict__ x, int64_t n) {
  const double c = sign * *a;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(c, x[i], y[i]);
}

__global__ void xpay_kernel(double* y, double a, const double* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fma(a, y[i], x[i]);
}

__global__ void scale_kernel(double* y, double a, const double* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

__global__ void sub_kernel(double* r, const double* __restrict__ b, const double* __restrict__ y,
                           int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - y[i];
}

__global__ void d2f_kernel(float* y, const double* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void f2d_kernel(double* y, const float* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

__global__ void rhs_kernel(int d, int n, int nterms, const double* __restrict__ coef,
                           const double* __restrict__ F, double* b, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int c[3] = {(int)(i % n), (int)((i / n) % n), d == 3 ? (int)(i / ((int64_t)n * n)) : 0};
    double s = 0.0;
    for (int t = 0; t < nterms; ++t) {
      double p = coef[t];
      for (int a = 0; a < d; ++a) p *= F[((int64_t)t * d + a) * n + c[a]];
      s += p;
    }
    b[i] = s;
  }
}

}  // namespace

cudaError_t vec_dot(const double* x, const double* y, int64_t n, double* partials, double* out,
                    cudaStream_t st) {
  dot_partial_kernel<<<kDotBlocks, 256, 0, st>>>(x, y, n, partials);
  cudaError_t e = launched();
  if (e != cudaSuccess) return e;
  dot_final_kernel<<<1, 256, 0, st>>>(partials, kDotBlocks, out);
  return launched();
}

cudaError_t vec_axpy(double* y, double a, const double* x, int64_t n, cudaStream_t st) {
  axpy_kernel<<<grid1d(n, 256), 256, 0, st>>>(y, a, x, n);
  return launched();
}

cudaError_t vec_axpy_dev(double* y, const double* a, double sign, const double* x, int64_t n,
                         cudaStream_t st) {
  axpy_dev_kernel<<<grid1d(n, 256), 256, 0, st>>>(y, a, sign, x, n);
  return launched();
}

cudaError_t vec_xpay(double* y, double a, const double* x, int64_t n, cudaStream_t st) {
  xpay_kernel<<<grid1d(n, 256), 256, 0, st>>>(y, a, x, n);
  return launched();
}

cudaError_t vec_scale(double* y, double a, const double* x, int64_t n, cudaStream_t st) {
  scale_kernel<<<grid1d(n, 256), 256, 0, st>>>(y, a, x, n);
  return launched();
}

cudaError_t vec_sub(double* r, const double* b, const double* y, int64_t n, cudaStream_t st) {
  sub_kernel<<<grid1d(n, 256), 256, 0, st>>>(r, b, y, n);
  return launched();
}

cudaError_t vec_d2f(float* y, const double* x, int64_t n, cudaStream_t st) {
  d2f_kernel<<<grid1d(n, 256), 256, 0, st>>>(y, x, n);
  return launched();
}

cudaError_t vec_f2d(double* y, const float* x, int64_t n, cudaStream_t st) {
  f2d_kernel<<<grid1d(n, 256), 256, 0, st>>>(y, x, n);
  return launched();
}

cudaError_t rhs_separable(int d, int n, int nterms, const double* coef, const double* F,
                          double* b, cudaStream_t st) {
  int64_t total = 1;
  for (int a = 0; a < d; ++a) total *= n;
  rhs_kernel<<<grid1d(total, 256), 256, 0, st>>>(d, n, nterms, coef, F, b, total);
  return launched();
}

}  // namespace bh
