// FP64 throughput probes: the denominators against which the FP64 kernels of
// this library can be read.  Every thread runs ILP independent chains of
// dependent fused multiply-adds (or FP64 tensor-core MMAs) on registers, no
// memory traffic inside the timed loop; the rate is timed with CUDA events on
// the caller's stream.
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

// the same with the FP64 tensor-core instruction: D = A B + C on 8x8x4 tiles
// (mma.sync, 512 flops per warp instruction), ILP independent accumulators
__global__ void __launch_bounds__(128) mma_chains(double* out, double a, double b, int iters) {
  double c[kIlp][2];
#pragma unroll
  for (int i = 0; i < kIlp; ++i) c[i][0] = c[i][1] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r)
#pragma unroll
      for (int i = 0; i < kIlp; ++i)
        asm volatile(
            "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
            : "+d"(c[i][0]), "+d"(c[i][1])
            : "d"(a), "d"(b));
  }
  double acc = 0.0;
#pragma unroll
  for (int i = 0; i < kIlp; ++i) acc += c[i][0] + c[i][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

bh_status perr(bh_status s, const std::string& m) {
  bh::set_last_error(m);
  return s;
}

// time `kernel` over 4 blocks of 128 threads per SM; flops_per_thread_iter:
// flops one thread contributes per loop iteration
template <typename Kernel>
bh_status rate(Kernel kernel, double a, double b, double flops_per_thread_iter, void* stream,
               double* tflops) {
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
    kernel<<<blocks, threads, 0, st>>>(out, a, b, iters);  // warm-up
    cudaEventRecord(e0, st);
    kernel<<<blocks, threads, 0, st>>>(out, a, b, iters);
    cudaEventRecord(e1, st);
    bh::g_kernel_launches.fetch_add(2);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        !(ms > 0.f))
      status = perr(BH_ECUDA, std::string("probe: ") + cudaGetErrorString(cudaGetLastError()));
  }
  if (status == BH_OK)
    *tflops = (double)blocks * threads * iters * flops_per_thread_iter / (ms * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return status;
}

}  // namespace

extern "C" bh_status bh_fp64_fma_rate(void* stream, double* tflops) {
  // 2 flops per FMA, kUnroll x kIlp FMAs per thread and iteration
  return rate(fma_chains, 0.999999, 1e-7, 2.0 * kUnroll * kIlp, stream, tflops);
}

extern "C" bh_status bh_fp64_mma_rate(void* stream, double* tflops) {
  // 512 flops per warp-wide 8x8x4 MMA = 16 per thread, kUnroll x kIlp per iteration
  return rate(mma_chains, 0.999999, 1e-7, 16.0 * kUnroll * kIlp, stream, tflops);
}
