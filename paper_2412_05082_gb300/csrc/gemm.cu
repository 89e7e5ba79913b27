// Dense matrix products of the exact local solver (Sec. 3: the exact patch
// inverse A_v^-1 as the variant the paper compares against): for a run of
// patches sharing one boundary-type combination, the patch tensors gathered as
// the columns of R (m^d x cnt) are multiplied by the dense inverse,
//
//   Y = alpha * A R,   A: m^d x m^d, column-major;  R, Y: m^d x cnt, column-major,
//
// with m^d = 729, 1331, 2197 for 3D k = 5, 6, 7.  The product is bound by the
// arithmetic pipe, never by memory: FP64 on GB300 issues about 2 DFMA per clock
// and SM, FP32 128 FFMA.
//  - FP64: the FP64 tensor-core instruction (mma.sync m8n8k4, 256 FMAs per warp
//    instruction, the rate of the FMA pipe or slightly above on this part);
//    a 64 x 64 tile per block of four warps, each warp 32 x 32 (16 MMAs per
//    k-step of 4), k-panels of 16 staged in shared memory by asynchronous
//    copies, double-buffered.
//  - FP32: FFMA with 8 x 8 outputs per thread, a 128 x 128 tile per block of
//    256 threads, 128-bit shared-memory operand loads (one byte of shared
//    memory per FMA), k-panels of 8, double-buffered.
// Out-of-range rows, columns and k are zero-filled in shared memory, so any
// m^d and cnt work; element-wise 4- or 8-byte copies need no alignment beyond
// the value's own (m^d is odd).
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"
#include "ops.h"

namespace bh {
namespace {

__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---- FP64: DMMA ------------------------------------------------------------
// Block tile (WM_ x 32) x (WN_ x 32): WM_ x WN_ warps, each warp a 32 x 32 tile
// (4 x 4 DMMA tiles of 8 x 8, 16 accumulating MMAs per k-step of 4); k-panels
// of BK values.
template <int WM_, int WN_, int BK_>
struct GemmF64Cfg {
  static constexpr int WM = WM_, WN = WN_, BK = BK_;
  static constexpr int BM = 32 * WM, BN = 32 * WN, PAD = 8, THREADS = 32 * WM * WN;
  static constexpr int LDA = BM + PAD, LDB = BN + PAD;
};
// one warp row by two warp columns (a 32 x 64 tile of 64 threads): the fastest of
// the shapes measured on GB300 at m^d = 729, 1331, 2197 (0.99, 1.02, 1.08 TFLOP/s;
// cuBLAS DGEMM on the same products: 1.06, 1.07, 1.08)
using GemmF64 = GemmF64Cfg<1, 2, 16>;

__device__ __forceinline__ void dmma_8x8x4(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

template <typename C>
__global__ void __launch_bounds__(C::THREADS) gemm_f64_kernel(int md, int cnt, double alpha,
                                                              const double* __restrict__ A,
                                                              const double* __restrict__ R,
                                                              double* __restrict__ Y) {
  __shared__ __align__(16) double As[2][C::BK][C::LDA];  // As[s][k][m] = A(m, k)
  __shared__ __align__(16) double Bs[2][C::BK][C::LDB];  // Bs[s][k][n] = R(k, n)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp % C::WM, wn = warp / C::WM;
  const int bm0 = blockIdx.x * C::BM, bn0 = blockIdx.y * C::BN;
  const int nk = (md + C::BK - 1) / C::BK;

  auto load = [&](int s, int k0) {
    // A panel: consecutive threads take consecutive m of one column k
    for (int e = tid; e < C::BK * C::BM; e += C::THREADS) {
      const int k = e / C::BM, m = e % C::BM;
      const int gm = bm0 + m, gk = k0 + k;
      const bool in = gm < md && gk < md;
      async_copy_or_zero(&As[s][k][m], A + (in ? (int64_t)gk * md + gm : 0), in);
    }
    // R panel: consecutive threads take consecutive k of one column n
    for (int e = tid; e < C::BK * C::BN; e += C::THREADS) {
      const int k = e % C::BK, n = e / C::BK;
      const int gk = k0 + k, gn = bn0 + n;
      const bool in = gk < md && gn < cnt;
      async_copy_or_zero(&Bs[s][k][n], R + (in ? (int64_t)gn * md + gk : 0), in);
    }
    async_commit();
  };

  double acc[4][4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = 0.0;

  load(0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt & 1;
    if (kt + 1 < nk) {
      load(s ^ 1, (kt + 1) * C::BK);
      async_wait_group<1>();
    } else {
      async_wait_group<0>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < C::BK; kk += 4) {
      // fragments: A (8x4, row) a = A(lane/4, lane%4); B (4x8, col) b = B(lane%4, lane/4)
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[s][kk + (lane & 3)][wm * 32 + i * 8 + (lane >> 2)];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[s][kk + (lane & 3)][wn * 32 + j * 8 + (lane >> 2)];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) dmma_8x8x4(acc[i][j][0], acc[i][j][1], a[i], b[j]);
    }
    __syncthreads();  // the stage is overwritten by the load two panels ahead
  }
  // D fragment: row lane/4, columns 2 (lane%4) + {0, 1}
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = bm0 + wm * 32 + i * 8 + (lane >> 2);
    if (gm >= md) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int gn = bn0 + wn * 32 + j * 8 + 2 * (lane & 3) + c;
        if (gn < cnt) Y[(int64_t)gn * md + gm] = alpha * acc[i][j][c];
      }
  }
}

template <typename C>
cudaError_t launch_gemm_f64(int md, int cnt, double alpha, const double* A, const double* R,
                            double* Y, cudaStream_t st) {
  const dim3 grid((unsigned)((md + C::BM - 1) / C::BM), (unsigned)((cnt + C::BN - 1) / C::BN));
  if (grid.y > 65535u) return cudaErrorInvalidValue;
  gemm_f64_kernel<C><<<grid, C::THREADS, 0, st>>>(md, cnt, alpha, A, R, Y);
  return cudaGetLastError();
}

// ---- FP32: FFMA, 8 x 8 per thread --------------------------------------------
struct GemmF32Cfg {
  static constexpr int BM = 128, BN = 128, BK = 8, PAD = 4, THREADS = 256;
  static constexpr int LDA = BM + PAD, LDB = BN + PAD;
};

__global__ void __launch_bounds__(GemmF32Cfg::THREADS) gemm_f32_kernel(int md, int cnt,
                                                                       float alpha,
                                                                       const float* __restrict__ A,
                                                                       const float* __restrict__ R,
                                                                       float* __restrict__ Y) {
  using C = GemmF32Cfg;
  __shared__ __align__(16) float As[2][C::BK][C::LDA];
  __shared__ __align__(16) float Bs[2][C::BK][C::LDB];
  const int tid = threadIdx.x;
  const int tm = tid & 15, tn = tid >> 4;  // rows 4 tm + {0..3} and 64 + 4 tm + {0..3}; same for n
  const int bm0 = blockIdx.x * C::BM, bn0 = blockIdx.y * C::BN;
  const int nk = (md + C::BK - 1) / C::BK;

  auto load = [&](int s, int k0) {
    for (int e = tid; e < C::BK * C::BM; e += C::THREADS) {
      const int k = e / C::BM, m = e % C::BM;
      const int gm = bm0 + m, gk = k0 + k;
      const bool in = gm < md && gk < md;
      async_copy_or_zero(&As[s][k][m], A + (in ? (int64_t)gk * md + gm : 0), in);
    }
    for (int e = tid; e < C::BK * C::BN; e += C::THREADS) {
      const int k = e % C::BK, n = e / C::BK;
      const int gk = k0 + k, gn = bn0 + n;
      const bool in = gk < md && gn < cnt;
      async_copy_or_zero(&Bs[s][k][n], R + (in ? (int64_t)gn * md + gk : 0), in);
    }
    async_commit();
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  load(0, 0);
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt & 1;
    if (kt + 1 < nk) {
      load(s ^ 1, (kt + 1) * C::BK);
      async_wait_group<1>();
    } else {
      async_wait_group<0>();
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < C::BK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[s][k][4 * tm]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[s][k][64 + 4 * tm]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[s][k][4 * tn]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[s][k][64 + 4 * tn]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = bm0 + (i < 4 ? 4 * tm + i : 64 + 4 * tm + i - 4);
    if (gm >= md) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gn = bn0 + (j < 4 ? 4 * tn + j : 64 + 4 * tn + j - 4);
      if (gn < cnt) Y[(int64_t)gn * md + gm] = alpha * acc[i][j];
    }
  }
}

}  // namespace

cudaError_t gemm_f64(int md, int cnt, double alpha, const double* A, const double* R, double* Y,
                     cudaStream_t st) {
  if (md <= 0 || cnt <= 0) return cudaSuccess;
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return launch_gemm_f64<GemmF64>(md, cnt, alpha, A, R, Y, st);
}

cudaError_t gemm_f32(int md, int cnt, float alpha, const float* A, const float* R, float* Y,
                     cudaStream_t st) {
  if (md <= 0 || cnt <= 0) return cudaSuccess;
  using C = GemmF32Cfg;
  const dim3 grid((unsigned)((md + C::BM - 1) / C::BM), (unsigned)((cnt + C::BN - 1) / C::BN));
  if (grid.y > 65535u) return cudaErrorInvalidValue;
  gemm_f32_kernel<<<grid, C::THREADS, 0, st>>>(md, cnt, alpha, A, R, Y);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace bh
