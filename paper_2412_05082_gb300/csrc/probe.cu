// FP64 FMA throughput probe: the denominator against which the FP64 kernels
// of this library can be read.  Every thread runs ILP independent chains of
// dependent fused multiply-adds on registers (no memory traffic inside the
// timed loop); the rate is timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include <string>

#include "biharm.h"
#include "ops.h"

namespace bh {
void set_last_error(const std::string& msg);  // api.cu
}

namespace {

constexpr int kIlp = 4, kUnroll = 16;

__global__ void __launch_bounds__(128) fma_chains(double* out, double a, double c, int iters) {
  double s[kIlp];
#pragma unroll
  for (int i = 0; i < kIlp; ++i) s[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kIlp; ++i) s[i] = fma(s[i], a, c);
  }
  double acc = 0.0;
#pragma unroll
  for (int i = 0; i < kIlp; ++i) acc += s[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;  // keeps the chains alive
}

bh_status perr(bh_status s, const std::string& m) {
  bh::set_last_error(m);
  return s;
}

}  // namespace

extern "C" bh_status bh_fp64_fma_rate(void* stream, double* tflops) {
  if (!tflops) return perr(BH_EINVAL, "null output");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return perr(BH_ECUDA, "no CUDA device available");
  }
  const int blocks = 4 * sms, threads = 128, iters = 400;
  cudaStream_t st = (cudaStream_t)stream;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bh_status status = BH_OK;
  float ms = 0.f;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) {
    cudaGetLastError();
    return perr(BH_ENOMEM, "probe buffer");
  }
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    status = perr(BH_ECUDA, "event creation failed");
  } else {
    fma_chains<<<blocks, threads, 0, st>>>(out, 0.999999, 1e-7, iters);  // warm-up
    cudaEventRecord(e0, st);
    fma_chains<<<blocks, threads, 0, st>>>(out, 0.999999, 1e-7, iters);
    cudaEventRecord(e1, st);
    bh::g_kernel_launches.fetch_add(2);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        !(ms > 0.f))
      status = perr(BH_ECUDA, std::string("probe: ") + cudaGetErrorString(cudaGetLastError()));
  }
  if (status == BH_OK) {
    const double fmas = (double)blocks * threads * iters * kUnroll * kIlp;
    *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return status;
}
