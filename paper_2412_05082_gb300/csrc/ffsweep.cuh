// Compensated defect of the FP32 V-cycle: r = b - scale * A_ref x for an FP32
// iterate x, evaluated in double-float arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats.  Every coefficient c of
// the 1D class tables is stored as c_hi = fl32(c) and c_lo = fl32(c - c_hi)
// (24 + 24 significant bits).  A product c x with x in FP32 is split exactly
// into p + e by an FMA (TwoProduct); c_lo x is added to e; the hi parts are
// summed with TwoSum (Knuth), which yields the exact rounding error of every
// addition.  The only roundings left are those of the low-order terms, so the
// defect carries an error of about (number of terms) 2^-48 of sum |terms|
// instead of 2^-24 for FP32 arithmetic.  The sum factorization, the row classes
// and the thread layout are those of the FP64 sweeps (kernels.cuh); the
// intermediates T_P = P_x x (and the 3D U_P) are stored as float2 (hi, lo),
// the same 8 bytes per value as FP64.  The final subtraction from the FP64
// right-hand side b is done in FP64 (two FMAs per node).
//
// On GB300 the FP64 pipe issues 1/64 of the FP32 rate, so the 10-12 FP32
// operations per band term cost far less issue time than one DFMA.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "kernels.cuh"

namespace bh {

template <int K>
struct FfTab {  // class tables of M, L, B as hi + lo FP32 parts
  OpTab<float, K> hi;
  OpTab<float, K> lo;
};

struct FfSweepArgs {
  const float* x;      // KIND 0: the FP32 iterate
  const float2* in[3];  // KIND 1..3: double-float intermediates
  float2* out[3];      // KIND 0, 1: double-float intermediates
  const double* b;     // KIND 2, 3: right-hand side
  double* r;           // KIND 2, 3: defect b - scale * A_ref x
  int d, axis, N, n;
  int64_t lines;       // n^(d-1)
  int64_t stride;      // n^axis
  double scale;
};

struct FfAcc {  // running sum of the hi parts and the accumulated low-order terms
  float s, c;
};

// s + e = a + b exactly (TwoSum); the intrinsics keep the compiler from
// contracting or reordering the operations
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += (ch + cl) x
__device__ __forceinline__ void ff_acc(FfAcc& acc, float ch, float cl, float x) {
  const float p = __fmul_rn(ch, x);
  float e = __fmaf_rn(ch, x, -p);  // ch x - p, exact
  e = __fmaf_rn(cl, x, e);
  float s, t;
  ff_two_sum(acc.s, p, s, t);
  acc.s = s;
  acc.c = __fadd_rn(acc.c, __fadd_rn(t, e));
}

// acc += (ch + cl) (xh + xl)
__device__ __forceinline__ void ff_acc(FfAcc& acc, float ch, float cl, float2 x) {
  const float p = __fmul_rn(ch, x.x);
  float e = __fmaf_rn(ch, x.x, -p);
  e = __fmaf_rn(ch, x.y, e);
  e = __fmaf_rn(cl, x.x, e);
  float s, t;
  ff_two_sum(acc.s, p, s, t);
  acc.s = s;
  acc.c = __fadd_rn(acc.c, __fadd_rn(t, e));
}

// the accumulated value as a normalized pair (FastTwoSum, |s| >= |c|)
__device__ __forceinline__ float2 ff_value(const FfAcc& a) {
  const float s = __fadd_rn(a.s, a.c);
  return make_float2(s, __fsub_rn(a.c, __fsub_rn(s, a.s)));
}

// window of double-float values: node c K - 2K + j, j in [LO, HI), hi parts in
// wh[j], lo parts in wl[j], zero outside 1..n
template <int K, int LO, int HI>
__device__ __forceinline__ void ff_load_window(const float2* __restrict__ p, int64_t base,
                                               int64_t stride, int c, int n, float* wh,
                                               float* wl) {
#pragma unroll
  for (int j = LO; j < HI; ++j) {
    const int g = c * K - 2 * K + j;
    float2 v = make_float2(0.f, 0.f);
    if (g >= 1 && g <= n) v = __ldg(p + base + (int64_t)(g - 1) * stride);
    wh[j] = v.x;
    wl[j] = v.y;
  }
}

// compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1 (the
// unrolled band loops exceed the compiler's unroll budget for k >= 4, which
// would leave the windows in local memory)
template <int B, int E, typename F>
__device__ __forceinline__ void ff_static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    ff_static_for<B + 1, E>(f);
  }
}

// acc[q] += C (P w)[q], q = 0..K-1, P given by its class tables (C = 1 or 2:
// exact scalings of both coefficient parts); FF: a double-float window (wh, wl), else an FP32 one (wh)
template <int K, int OP, int C, bool CANON, bool FF>
__device__ __forceinline__ void ff_band(const float (&th)[3 * K + 1][4 * K + 1],
                                        const float (&tl)[3 * K + 1][4 * K + 1],
                                        const int* cls, const float* wh, const float* wl,
                                        FfAcc* acc) {
  ff_static_for<0, K>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    const int c = CANON ? q : cls[q];
    ff_static_for<band_lo(OP, q, K), band_hi(OP, q, K) + 1>([&](auto tc) {
      constexpr int t = decltype(tc)::value;
      const float ch = (float)C * th[c][t + 2 * K], cl = (float)C * tl[c][t + 2 * K];
      if constexpr (FF)
        ff_acc(acc[q], ch, cl, make_float2(wh[q + t + 2 * K], wl[q + t + 2 * K]));
      else
        ff_acc(acc[q], ch, cl, wh[q + t + 2 * K]);
    });
  });
}

// KIND 0: split  out0 = M x, out1 = L x, out2 = B x   (x FP32)
// KIND 1: mix3d  out0 = M in2 + B in0 + 2 L in1, out1 = M in0, out2 = 2 (L in0 + M in1)
// KIND 2: r = b - scale (B in0 + 2 L in1 + M in2)      (2D final sweep)
// KIND 3: r = b - scale (M in0 + B in1 + L in2)        (3D final sweep)
// KIND 0 reads the FP32 x window from the block's staged copy: xw[j] is the
// value at node c K - 2K + j of the line, zero outside 1..n (ff_split_tile)
template <int K, int KIND, bool CANON>
__device__ __forceinline__ void ff_sweep_cell(const FfTab<K>& tab, const FfSweepArgs& a,
                                              int64_t base, int c, const int* cls,
                                              const float* xw = nullptr) {
  constexpr int W = 4 * K + 1, WML = 3 * K + 1;
  const OpTab<float, K>& hi = tab.hi;
  const OpTab<float, K>& lo = tab.lo;
  if (KIND == 0 || KIND == 1) {
    FfAcc u0[K], u1[K], u2[K];
#pragma unroll
    for (int q = 0; q < K; ++q) u0[q] = u1[q] = u2[q] = FfAcc{0.f, 0.f};
    if (KIND == 0) {
      float w[W];
#pragma unroll
      for (int j = 0; j < W; ++j) w[j] = xw[j];
      ff_band<K, 0, 1, CANON, false>(hi.M, lo.M, cls, w, nullptr, u0);
      ff_band<K, 1, 1, CANON, false>(hi.L, lo.L, cls, w, nullptr, u1);
      ff_band<K, 2, 1, CANON, false>(hi.B, lo.B, cls, w, nullptr, u2);
    } else {
      float wh[W], wl[W];
      ff_load_window<K, 0, W>(a.in[0], base, a.stride, c, a.n, wh, wl);  // T_M
      ff_band<K, 2, 1, CANON, true>(hi.B, lo.B, cls, wh, wl, u0);
      ff_band<K, 0, 1, CANON, true>(hi.M, lo.M, cls, wh, wl, u1);
      ff_band<K, 1, 2, CANON, true>(hi.L, lo.L, cls, wh, wl, u2);
      ff_load_window<K, K, WML>(a.in[1], base, a.stride, c, a.n, wh, wl);  // T_L
      ff_band<K, 1, 2, CANON, true>(hi.L, lo.L, cls, wh, wl, u0);
      ff_band<K, 0, 2, CANON, true>(hi.M, lo.M, cls, wh, wl, u2);
      ff_load_window<K, K, WML>(a.in[2], base, a.stride, c, a.n, wh, wl);  // T_B
      ff_band<K, 0, 1, CANON, true>(hi.M, lo.M, cls, wh, wl, u0);
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int g = c * K + q;
      if (g < 1) continue;
      const int64_t o = base + (int64_t)(g - 1) * a.stride;
      a.out[0][o] = ff_value(u0[q]);
      a.out[1][o] = ff_value(u1[q]);
      a.out[2][o] = ff_value(u2[q]);
    }
  } else {
    FfAcc y[K];
#pragma unroll
    for (int q = 0; q < K; ++q) y[q] = FfAcc{0.f, 0.f};
    float wh[W], wl[W];
    if (KIND == 2) {
      ff_load_window<K, 0, W>(a.in[0], base, a.stride, c, a.n, wh, wl);
      ff_band<K, 2, 1, CANON, true>(hi.B, lo.B, cls, wh, wl, y);
      ff_load_window<K, K, WML>(a.in[1], base, a.stride, c, a.n, wh, wl);
      ff_band<K, 1, 2, CANON, true>(hi.L, lo.L, cls, wh, wl, y);
      ff_load_window<K, K, WML>(a.in[2], base, a.stride, c, a.n, wh, wl);
      ff_band<K, 0, 1, CANON, true>(hi.M, lo.M, cls, wh, wl, y);
    } else {
      ff_load_window<K, K, WML>(a.in[0], base, a.stride, c, a.n, wh, wl);
      ff_band<K, 0, 1, CANON, true>(hi.M, lo.M, cls, wh, wl, y);
      ff_load_window<K, 0, W>(a.in[1], base, a.stride, c, a.n, wh, wl);
      ff_band<K, 2, 1, CANON, true>(hi.B, lo.B, cls, wh, wl, y);
      ff_load_window<K, K, WML>(a.in[2], base, a.stride, c, a.n, wh, wl);
      ff_band<K, 1, 1, CANON, true>(hi.L, lo.L, cls, wh, wl, y);
    }
    const double sc = a.scale;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int g = c * K + q;
      if (g < 1) continue;
      const int64_t o = base + (int64_t)(g - 1) * a.stride;
      const float2 v = ff_value(y[q]);
      a.r[o] = fma(-sc, (double)v.y, fma(-sc, (double)v.x, a.b[o]));
    }
  }
}

// one thread of a sweep: thread index tid in [0, lines * N), the layout of
// sweep_thread
template <int K, int KIND>
__device__ __forceinline__ void ff_sweep_thread(const FfTab<K>& tab, const FfSweepArgs& a,
                                                int64_t tid) {
  static_assert(KIND != 0, "the split runs in tiles (ff_split_tile)");
  int64_t line;
  int c;
  if (a.axis == 0) {
    line = tid / a.N;
    c = (int)(tid % a.N);
  } else {
    c = (int)(tid / a.lines);
    line = tid % a.lines;
  }
  int dims[3] = {a.n, a.n, a.n};
  int64_t strides[3] = {1, (int64_t)a.n, (int64_t)a.n * a.n};
  const int64_t base = line_offset(line, a.d, a.axis, dims, strides);
  if (c >= 2 && c <= a.N - 2) {
    ff_sweep_cell<K, KIND, true>(tab, a, base, c, nullptr);
  } else {
    int cls[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int g = c * K + q;
      cls[q] = (g >= 1) ? row_class<K>(g, a.N) : 0;
    }
    ff_sweep_cell<K, KIND, false>(tab, a, base, c, cls);
  }
}

// KIND 0 runs along the contiguous axis, in the tiles of the FP64 split
// (kernels.cuh: 32 lines x 4 cells per block, a warp per cell, from a
// shared-memory copy of the tile's x)
constexpr int kFfBlock = kSplitBlock;
__host__ __device__ inline int64_t ff_sweep_threads(int kind, int64_t lines, int N) {
  return sweep_launch_threads(kind, lines, N);
}

template <int K>
__device__ __forceinline__ void ff_split_tile(const FfTab<K>& tab, const FfSweepArgs& a,
                                              int64_t blk, float* sx) {
  int64_t l;
  int c;
  const float* xw = split_stage<float, K>(a.x, a.lines, a.N, a.n, blk, sx, l, c);
  if (c < 0) return;
  const int64_t base = l * a.n;  // axis 0: line l starts at l n
  if (c >= 2 && c <= a.N - 2) {
    ff_sweep_cell<K, 0, true>(tab, a, base, c, nullptr, xw);
  } else {
    int cls[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int g = c * K + q;
      cls[q] = (g >= 1) ? row_class<K>(g, a.N) : 0;
    }
    ff_sweep_cell<K, 0, false>(tab, a, base, c, cls, xw);
  }
}

template <int K, int KIND>
__global__ void __launch_bounds__(kFfBlock) ff_sweep_kernel(const __grid_constant__ FfTab<K> tab,
                                                            const FfSweepArgs a) {
  if constexpr (KIND == 0) {
    __shared__ float sx[kSplitTileLines * SplitTile<K>::RS];
    ff_split_tile<K>(tab, a, blockIdx.x, sx);
  } else {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid < a.lines * a.N) ff_sweep_thread<K, KIND>(tab, a, tid);
  }
}

// the sweep over a (problem, range) list of problems of one degree K (the
// batched form): tabs[p] is problem p's FfTab<K> device copy, active[p] = 0
// skips problem p.  Every problem's range holds ff_sweep_threads(KIND, ...)
// threads, whole blocks, so that a block works on one problem.
template <int K, int KIND>
__global__ void __launch_bounds__(kFfBlock) ff_sweep_list_kernel(const FfSweepArgs* args,
                                                                 const int64_t* prefix,
                                                                 const int* pid, int n,
                                                                 const int* active,
                                                                 const void* const* tabs) {
  const int64_t bstart = (int64_t)blockIdx.x * blockDim.x;
  if (bstart >= prefix[n]) return;
  const int s = find_seg(prefix, n, bstart);  // the same for the whole block
  const int p = pid[s];
  if (!active[p]) return;
  const FfSweepArgs& a = args[s];
  const FfTab<K>& tab = *static_cast<const FfTab<K>*>(tabs[p]);
  const int64_t first = bstart - prefix[s];
  if constexpr (KIND == 0) {
    __shared__ float sx[kSplitTileLines * SplitTile<K>::RS];
    ff_split_tile<K>(tab, a, first / kFfBlock, sx);
  } else {
    const int64_t tid = first + threadIdx.x;
    if (tid < a.lines * a.N) ff_sweep_thread<K, KIND>(tab, a, tid);
  }
}

}  // namespace bh
