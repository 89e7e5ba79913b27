// Dense matrix products of the exact local solver (Sec. 3: the exact patch
// inverse A_v^-1 as the variant the paper compares against): for a run of
// patches sharing one boundary-type combination, the patch tensors gathered as
// the columns of R (m^d x cnt) are multiplied by the dense inverse,
//
//   Y = alpha * A R,   A: m^d x m^d symmetric;  R, Y: m^d x cnt, column-major,
//
// with m^d = 729, 1331, 2197 for 3D k = 5, 6, 7.
//
// FP64: emulated on the FP16 tensor cores by splitting the operands into
// integer slices (an error-free splitting of the Ozaki type).  Every row of A
// and every column of R is scaled by a power of two into (-1, 1) and split into
// kSlices slices of kSliceBits bits: x = 2^e sum_i x_i 2^(-6 (i+1)), x_i an
// integer with |x_i| <= 63, exact in FP16.  A slice product sum_k a_i r_j is an
// integer below K 63^2 < 2^24 for K <= 4,227, so the tensor cores' FP32
// accumulation over the whole inner dimension is exact; the products of the
// slice pairs (i, j) with i + j < kSlices are scaled by 2^(-6 (i + j + 2)) and
// summed in FP64.  The dropped pairs and the split's remainder are below
// 2^(-6 kSlices) relative to the row and column maxima: 2^-54 for 9 slices,
// the FP64 significand.  The bound is relative to the maxima, so fewer slices
// fail where a row of the inverse spans a wide range (8 slices: 2.5e-10 on one
// exact step of the single 3D k = 7 patch of level 1, against 1e-10 asked).
// FP16 mma.sync runs at 600 TFLOP/s on GB300 against 1.1 for the FP64 tensor
// instruction (measured), so the 45 slice products of the emulation still beat
// the FP64 product several times over.
//
// FP32 (the mixed forms): FFMA with 8 x 8 outputs per thread, a 128 x 128 tile
// per block of 256 threads, 128-bit shared-memory operand loads, k-panels of 8,
// double-buffered.
#include <cuda_runtime.h>

#include <cuda_fp16.h>

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

// ---- FP64 by FP16 slices ----------------------------------------------------
// One warp per column n of X (rows x cols, column-major, leading dimension
// rows): F[n] = e with max_k |X(k, n)| < 2^e, slices Xs[i][n][k] (leading
// dimension ldk >= rows, a multiple of 8; zero for k in [rows, ldk)).
__global__ void __launch_bounds__(256) slice_cols_kernel(const double* __restrict__ X, int rows,
                                                         int cols, int ldk, __half* __restrict__ Xs,
                                                         int* __restrict__ F) {
  const int col = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (col >= cols) return;
  const double* x = X + (int64_t)col * rows;
  double mx = 0.0;
  for (int k = lane; k < rows; k += 32) mx = fmax(mx, fabs(x[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int e = mx > 0.0 ? ilogb(mx) + 1 : 0;
  if (lane == 0) F[col] = e;
  const int64_t plane = (int64_t)cols * ldk;
  for (int k = lane; k < ldk; k += 32) {
    double t = k < rows ? ldexp(x[k], -e) : 0.0;  // |t| < 1, exact
#pragma unroll
    for (int i = 0; i < kSlices; ++i) {
      t *= (double)(1 << kSliceBits);  // exact
      const double q = trunc(t);       // |q| <= 63
      t -= q;                          // exact
      Xs[i * plane + (int64_t)col * ldk + k] = __float2half_rn((float)q);
    }
  }
}

struct SlicedCfg {
  static constexpr int BM = 128, BN = 64, BK = 32, PADK = 8, THREADS = 256;
  static constexpr int LD = BK + PADK;  // halves per shared-memory row (80 bytes)
  static constexpr int PAIRS = kSlices * (kSlices + 1) / 2;
};

__device__ __forceinline__ void async_copy16(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}

__device__ __forceinline__ void hmma_16x8x16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Y = alpha A R from the slices: As[i][m][k] and Ea[m] of the rows of A, Rs[j][n][k] and
// Fr[n] of the columns of R (leading dimension ldk).  A block computes a 128 x 64
// tile with 8 warps of 32 x 32 (2 x 4 MMA tiles of 16 x 8); the (pair, k-panel)
// sequence is one stream of 16-byte asynchronous copies, double-buffered.
__global__ void __launch_bounds__(SlicedCfg::THREADS, 2) gemm_sliced_kernel(
    int md, int cnt, int ldk, double alpha, const __half* __restrict__ As,
    const int* __restrict__ Ea, const __half* __restrict__ Rs, const int* __restrict__ Fr,
    double* __restrict__ Y) {
  using C = SlicedCfg;
  __shared__ __align__(16) __half sA[2][C::BM][C::LD];
  __shared__ __align__(16) __half sB[2][C::BN][C::LD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 3, wn = warp >> 2;  // 4 x 2 warps
  const int g = lane >> 2, t = lane & 3;
  const int bm0 = blockIdx.x * C::BM, bn0 = blockIdx.y * C::BN;
  const int nk = (md + C::BK - 1) / C::BK;
  const int64_t aplane = (int64_t)md * ldk, rplane = (int64_t)cnt * ldk;
  // slice pairs (i, j), i + j < kSlices, the level i + j ascending
  int pi[C::PAIRS], pj[C::PAIRS];
  {
    int q = 0;
#pragma unroll
    for (int l = 0; l < kSlices; ++l)
#pragma unroll
      for (int i = 0; i <= l; ++i) {
        pi[q] = i;
        pj[q] = l - i;
        ++q;
      }
  }
  const int total = C::PAIRS * nk;
  auto load = [&](int st, int idx) {
    const int pr = idx / nk, kt = idx - pr * nk;
    const __half* Ai = As + pi[pr] * aplane;
    const __half* Rj = Rs + pj[pr] * rplane;
    const int k0 = kt * C::BK;
    for (int e = tid; e < C::BM * (C::BK / 8); e += C::THREADS) {
      const int m = e >> 2, c = e & 3, gm = bm0 + m, gk = k0 + 8 * c;
      const bool in = gm < md && gk < ldk;
      async_copy16(&sA[st][m][8 * c], Ai + (in ? (int64_t)gm * ldk + gk : 0), in);
    }
    for (int e = tid; e < C::BN * (C::BK / 8); e += C::THREADS) {
      const int n = e >> 2, c = e & 3, gn = bn0 + n, gk = k0 + 8 * c;
      const bool in = gn < cnt && gk < ldk;
      async_copy16(&sB[st][n][8 * c], Rj + (in ? (int64_t)gn * ldk + gk : 0), in);
    }
    async_commit();
  };
  float acc32[2][4][4];
  double acc64[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        acc32[a][b][c] = 0.f;
        acc64[a][b][c] = 0.0;
      }
  load(0, 0);
  for (int idx = 0; idx < total; ++idx) {
    const int st = idx & 1;
    if (idx + 1 < total) {
      load(st ^ 1, idx + 1);
      async_wait_group<1>();
    } else {
      async_wait_group<0>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < C::BK; kk += 16) {
      // fragments of m16n8k16: A (row) rows g, g + 8 and columns 2t, 2t + 1 (+ 8);
      // B (col) rows 2t, 2t + 1 (+ 8) and column g
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int r0 = wm * 32 + a * 16 + g;
        af[a][0] = *reinterpret_cast<const uint32_t*>(&sA[st][r0][kk + 2 * t]);
        af[a][1] = *reinterpret_cast<const uint32_t*>(&sA[st][r0 + 8][kk + 2 * t]);
        af[a][2] = *reinterpret_cast<const uint32_t*>(&sA[st][r0][kk + 2 * t + 8]);
        af[a][3] = *reinterpret_cast<const uint32_t*>(&sA[st][r0 + 8][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c0 = wn * 32 + b * 8 + g;
        bf[b][0] = *reinterpret_cast<const uint32_t*>(&sB[st][c0][kk + 2 * t]);
        bf[b][1] = *reinterpret_cast<const uint32_t*>(&sB[st][c0][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) hmma_16x8x16(acc32[a][b], af[a], bf[b]);
    }
    __syncthreads();  // the stage is overwritten by the copy two panels ahead
    const int pr = idx / nk, kt = idx - pr * nk;
    if (kt == nk - 1) {  // the pair's product is complete, an exact integer
      const double sc = ldexp(1.0, -kSliceBits * (pi[pr] + pj[pr] + 2));
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            acc64[a][b][c] = fma((double)acc32[a][b][c], sc, acc64[a][b][c]);
            acc32[a][b][c] = 0.f;
          }
    }
  }
  // D fragment c: row g (+ 8 for c >= 2), column 2t + (c & 1)
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int gm = bm0 + wm * 32 + a * 16 + g + (c >= 2 ? 8 : 0);
        const int gn = bn0 + wn * 32 + b * 8 + 2 * t + (c & 1);
        if (gm < md && gn < cnt)
          Y[(int64_t)gn * md + gm] = alpha * ldexp(acc64[a][b][c], Ea[gm] + Fr[gn]);
      }
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

int slice_ld(int rows) { return (rows + 7) / 8 * 8; }

cudaError_t slice_cols(const double* X, int rows, int cols, uint16_t* Xs, int* F,
                       cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const int64_t threads = (int64_t)cols * 32;
  slice_cols_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      X, rows, cols, slice_ld(rows), reinterpret_cast<__half*>(Xs), F);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t gemm_f64_sliced(int md, int cnt, double alpha, const uint16_t* As, const int* Ea,
                            const uint16_t* Rs, const int* Fr, double* Y, cudaStream_t st) {
  if (md <= 0 || cnt <= 0) return cudaSuccess;
  // the FP32 accumulation of a slice product is exact while md 63^2 < 2^24
  if (md * 63 * 63 >= (1 << 24)) return cudaErrorInvalidValue;
  using C = SlicedCfg;
  const dim3 grid((unsigned)((md + C::BM - 1) / C::BM), (unsigned)((cnt + C::BN - 1) / C::BN));
  if (grid.y > 65535u) return cudaErrorInvalidValue;
  gemm_sliced_kernel<<<grid, C::THREADS, 0, st>>>(md, cnt, slice_ld(md), alpha,
                                                  reinterpret_cast<const __half*>(As), Ea,
                                                  reinterpret_cast<const __half*>(Rs), Fr, Y);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
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
