// CUDA kernels of the multigrid hot path, templated on the value type T
// (double or float) and the degree K.  Instantiated in inst_f64.cu / inst_f32.cu.
//
// Data layout: a level's unknowns are the interior support points of the
// uniform mesh with N cells per direction, n = K N - 1 per direction, stored
// lexicographically with x fastest (index i_0 + n i_1 + n^2 i_2 for the global
// node (i_0+1, i_1+1, i_2+1)).
//
// Operator: on a Cartesian mesh the C0IP matrix is the Kronecker sum of
// Eq. (c0iptensorvp) / Eq. (c0iptensorvp3D) of banded 1D matrices M, L, B.
// apply() evaluates it by sum factorization, one sweep per direction:
//   2D:  T_P = P_x x (P = M, L, B);       y = B_y T_M + 2 L_y T_L + M_y T_B
//   3D:  T_P = P_x x;  U_M = M_y T_B + B_y T_M + 2 L_y T_L,  U_B = M_y T_M,
//        U_L = 2 (L_y T_M + M_y T_L);     y = M_z U_M + B_z U_B + L_z U_L
// (the six terms of Eq. (c0iptensorvp3D) with shared intermediates).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "fdm_line.cuh"
#include "ops.h"

namespace bh {

// ---------------------------------------------------------------------------
// kernel-parameter tables at reference scale (cells of size 1)
// ---------------------------------------------------------------------------
template <typename T, int K>
struct OpTab {  // row classes x band entries t = -2K..2K
  T M[3 * K + 1][4 * K + 1];
  T L[3 * K + 1][4 * K + 1];
  T B[3 * K + 1][4 * K + 1];
};

template <typename T, int K>
struct FdmTab {  // fast diagonalization per patch type (Sec. 4.1)
  T S[4][2 * K - 1][2 * K - 1];  // S[type][row][col], column = eigenvector
  T lam[4][2 * K - 1];
};

template <typename T, int K>
struct XferTab {  // coarse basis q at fine offset r inside a coarse cell
  T P[2 * K][K + 1];
};

template <typename T, int K>
struct Tables {
  OpTab<T, K> op;
  FdmTab<T, K> fdm;
  XferTab<T, K> xfer;
};

// class of interior row g (1..KN-1) of a global 1D matrix (see setup.h)
template <int K>
__device__ __forceinline__ int row_class(int g, int N) {
  if (N == 2) return g < K ? K + g - 1 : (g == K ? 3 * K : 2 * K + (g - K));
  if (g <= K) return K + g - 1;
  if (g >= K * N - K) return 2 * K + g - (K * N - K);
  return g % K;
}

// band of row position q inside an output cell: operator 0 = M, 1 = L, 2 = B
__host__ __device__ constexpr int band_lo(int op, int q, int K) {
  return op == 2 ? (q == 0 ? -2 * K : -K - q) : (q == 0 ? -K : -q);
}
__host__ __device__ constexpr int band_hi(int op, int q, int K) {
  return op == 2 ? (q == 0 ? 2 * K : 2 * K - q) : (q == 0 ? K : K - q);
}

// first index p with prefix[p + 1] > tid (prefix[0] = 0, increasing)
__device__ __forceinline__ int find_seg(const int64_t* prefix, int n, int64_t tid) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= tid)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Coordinates of a line (all non-axis coordinates) -> offset, x fastest.
__device__ __forceinline__ int64_t line_offset(int64_t line, int d, int axis, const int* dims,
                                               const int64_t* strides) {
  int64_t off = 0;
  for (int a = 0; a < d; ++a) {
    if (a == axis) continue;
    int64_t c = line % dims[a];
    line /= dims[a];
    off += c * strides[a];
  }
  return off;
}

// ---------------------------------------------------------------------------
// sweeps along one axis
// ---------------------------------------------------------------------------
template <typename T>
struct SweepArgs {
  const T* in[3];
  T* out[3];
  const T* b;      // residual mode
  int d, axis, N, n;
  int64_t lines;   // n^(d-1)
  int64_t stride;  // n^axis
  double scale;
  int mode;
};

// window w[j] = value at node c K - 2K + j, j in [LO, HI), zero outside 1..n;
// row c K + q (q = 0..K-1) with band offset t reads w[q + t + 2K].  A sweep
// kernel reads its inputs through the read-only data path (__ldg); a kernel
// that writes them itself in an earlier phase (the persistent V-cycle) takes
// COHERENT = true and plain loads.
template <typename T, int K, int LO, int HI, bool COHERENT = false>
__device__ __forceinline__ void load_window(const T* __restrict__ p, int64_t base,
                                            int64_t stride, int c, int n, T* w) {
#pragma unroll
  for (int j = LO; j < HI; ++j) {
    const int g = c * K - 2 * K + j;
    const T* src = p + base + (int64_t)(g - 1) * stride;
    w[j] = (g >= 1 && g <= n) ? (COHERENT ? *src : __ldg(src)) : T(0);
  }
}

// acc[q] += C * (P w)[q], q = 0..K-1, P given by its class table
template <typename T, int K, int OP, bool CANON>
__device__ __forceinline__ void band_acc(const T (&tab)[3 * K + 1][4 * K + 1], const int* cls,
                                         const T* w, T* acc, T C) {
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const int c = CANON ? q : cls[q];
    T s = T(0);
#pragma unroll
    for (int t = band_lo(OP, q, K); t <= band_hi(OP, q, K); ++t)
      s = fma(tab[c][t + 2 * K], w[q + t + 2 * K], s);
    acc[q] = (C == T(1)) ? acc[q] + s : fma(C, s, acc[q]);
  }
}

// KIND 0: split  out0 = M in0, out1 = L in0, out2 = B in0
// KIND 1: mix3d  out0 = M in2 + B in0 + 2 L in1, out1 = M in0, out2 = 2 (L in0 + M in1)
//                (in0 = T_M, in1 = T_L, in2 = T_B)
// KIND 2: final2d y = B in0 + 2 L in1 + M in2  (in = T_M, T_L, T_B)
// KIND 3: final3d y = M in0 + B in1 + L in2    (in = U_M, U_B, U_L)
// KIND 0 may take its window from a staged copy: xw[j] = value at node
// c K - 2K + j of the line, zero outside 1..n (sweep_split_tile)
template <typename T, int K, int KIND, bool CANON, bool COHERENT = false>
__device__ __forceinline__ void sweep_cell(const OpTab<T, K>& tab, const SweepArgs<T>& a,
                                           int64_t base, int c, const int* cls,
                                           const T* xw = nullptr) {
  constexpr int W = 4 * K + 1;  // B band reaches node offsets -2K..2K of every row
  constexpr int WML = 3 * K + 1;  // M and L reach -K..K
  T w[W];
  if (KIND == 0) {
    T aM[K], aL[K], aB[K];
#pragma unroll
    for (int q = 0; q < K; ++q) aM[q] = aL[q] = aB[q] = T(0);
    if (xw) {
#pragma unroll
      for (int j = 0; j < W; ++j) w[j] = xw[j];
    } else {
      load_window<T, K, 0, W, COHERENT>(a.in[0], base, a.stride, c, a.n, w);
    }
    band_acc<T, K, 0, CANON>(tab.M, cls, w, aM, T(1));
    band_acc<T, K, 1, CANON>(tab.L, cls, w, aL, T(1));
    band_acc<T, K, 2, CANON>(tab.B, cls, w, aB, T(1));
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int g = c * K + q;
      if (g < 1) continue;
      const int64_t o = base + (int64_t)(g - 1) * a.stride;
      a.out[0][o] = aM[q];
      a.out[1][o] = aL[q];
      a.out[2][o] = aB[q];
    }
  } else if (KIND == 1) {
    T u0[K], u1[K], u2[K];
#pragma unroll
    for (int q = 0; q < K; ++q) u0[q] = u1[q] = u2[q] = T(0);
    load_window<T, K, 0, W, COHERENT>(a.in[0], base, a.stride, c, a.n, w);  // T_M
    band_acc<T, K, 2, CANON>(tab.B, cls, w, u0, T(1));
    band_acc<T, K, 0, CANON>(tab.M, cls, w, u1, T(1));
    band_acc<T, K, 1, CANON>(tab.L, cls, w, u2, T(2));
    load_window<T, K, K, WML, COHERENT>(a.in[1], base, a.stride, c, a.n, w);  // T_L
    band_acc<T, K, 1, CANON>(tab.L, cls, w, u0, T(2));
    band_acc<T, K, 0, CANON>(tab.M, cls, w, u2, T(2));
    load_window<T, K, K, WML, COHERENT>(a.in[2], base, a.stride, c, a.n, w);  // T_B
    band_acc<T, K, 0, CANON>(tab.M, cls, w, u0, T(1));
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int g = c * K + q;
      if (g < 1) continue;
      const int64_t o = base + (int64_t)(g - 1) * a.stride;
      a.out[0][o] = u0[q];
      a.out[1][o] = u1[q];
      a.out[2][o] = u2[q];
    }
  } else {
    T y[K];
#pragma unroll
    for (int q = 0; q < K; ++q) y[q] = T(0);
    if (KIND == 2) {
      load_window<T, K, 0, W, COHERENT>(a.in[0], base, a.stride, c, a.n, w);
      band_acc<T, K, 2, CANON>(tab.B, cls, w, y, T(1));
      load_window<T, K, K, WML, COHERENT>(a.in[1], base, a.stride, c, a.n, w);
      band_acc<T, K, 1, CANON>(tab.L, cls, w, y, T(2));
      load_window<T, K, K, WML, COHERENT>(a.in[2], base, a.stride, c, a.n, w);
      band_acc<T, K, 0, CANON>(tab.M, cls, w, y, T(1));
    } else {
      load_window<T, K, K, WML, COHERENT>(a.in[0], base, a.stride, c, a.n, w);
      band_acc<T, K, 0, CANON>(tab.M, cls, w, y, T(1));
      load_window<T, K, 0, W, COHERENT>(a.in[1], base, a.stride, c, a.n, w);
      band_acc<T, K, 2, CANON>(tab.B, cls, w, y, T(1));
      load_window<T, K, K, WML, COHERENT>(a.in[2], base, a.stride, c, a.n, w);
      band_acc<T, K, 1, CANON>(tab.L, cls, w, y, T(1));
    }
    const T sc = (T)a.scale;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int g = c * K + q;
      if (g < 1) continue;
      const int64_t o = base + (int64_t)(g - 1) * a.stride;
      a.out[0][o] = (a.mode == kResidual) ? a.b[o] - sc * y[q] : sc * y[q];
    }
  }
}

// one thread of a sweep: thread index tid in [0, lines * N)
template <typename T, int K, int KIND, bool COHERENT = false>
__device__ __forceinline__ void sweep_thread(const OpTab<T, K>& tab, const SweepArgs<T>& a,
                                             int64_t tid) {
  int64_t line;
  int c;
  if (a.axis == 0) {  // consecutive threads: consecutive cells of one line
    line = tid / a.N;
    c = (int)(tid % a.N);
  } else {            // consecutive threads: consecutive x of one cell layer
    c = (int)(tid / a.lines);
    line = tid % a.lines;
  }
  int dims[3] = {a.n, a.n, a.n};
  int64_t strides[3] = {1, (int64_t)a.n, (int64_t)a.n * a.n};
  const int64_t base = line_offset(line, a.d, a.axis, dims, strides);
  if (c >= 2 && c <= a.N - 2) {
    sweep_cell<T, K, KIND, true, COHERENT>(tab, a, base, c, nullptr);
  } else {
    int cls[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int g = c * K + q;
      cls[q] = (g >= 1) ? row_class<K>(g, a.N) : 0;
    }
    sweep_cell<T, K, KIND, false, COHERENT>(tab, a, base, c, cls);
  }
}

// The split along the contiguous axis (KIND 0, axis 0) in tiles: one thread
// per cell along a line would put different cells (boundary and interior row
// classes, two code paths) in one warp and read x k values apart.  A block of
// 128 threads takes 32 lines x 4 consecutive cells instead, warp w the cell
// c0 + w of all 32 lines (lane = line), so that its row classes and branch
// are uniform; it first copies the tile's x values (per line the nodes of the
// four cells' windows, c0 K - 2K .. (c0 + 3) K + 2K, zero outside 1..n) into
// shared memory with loads along the lines.
constexpr int kSplitBlock = 128, kSplitTileLines = 32;
constexpr int kSplitTileCells = kSplitBlock / kSplitTileLines;
__host__ __device__ inline int64_t split_blocks(int64_t lines, int N) {
  return (lines + kSplitTileLines - 1) / kSplitTileLines *
         ((N + kSplitTileCells - 1) / kSplitTileCells);
}
// threads of one sweep launch: the split (KIND 0) in tiles, the other sweeps
// one thread per cell, in whole blocks of 128
__host__ __device__ inline int64_t sweep_launch_threads(int kind, int64_t lines, int N) {
  return kind == 0 ? split_blocks(lines, N) * kSplitBlock
                   : (lines * N + kSplitBlock - 1) / kSplitBlock * kSplitBlock;
}
template <int K>
struct SplitTile {
  static constexpr int R = 7 * K + 1;  // staged nodes per line
  static constexpr int RS = R | 1;     // row stride: odd, so the lanes' rows fall in distinct banks
};

// the tile's staged x (V: the value type) for block blk of a split; returns
// for the calling thread its line l, cell c and the window pointer, c = -1
// for a thread without a cell
template <typename V, int K>
__device__ __forceinline__ const V* split_stage(const V* x, int64_t lines, int N, int n,
                                                int64_t blk, V* sx, int64_t& l, int& c) {
  using S = SplitTile<K>;
  const int tc = (N + kSplitTileCells - 1) / kSplitTileCells;
  const int64_t lt = blk / tc;
  const int c0 = (int)(blk - lt * tc) * kSplitTileCells;
  const int64_t l0 = lt * kSplitTileLines;
  const int g0 = c0 * K - 2 * K;  // node of staged column 0
  for (int e = threadIdx.x; e < kSplitTileLines * S::R; e += blockDim.x) {
    const int r = e / S::R, col = e - r * S::R;
    const int64_t lr = l0 + r;
    const int g = g0 + col;
    sx[r * S::RS + col] = (lr < lines && g >= 1 && g <= n) ? __ldg(x + lr * n + (g - 1)) : V(0);
  }
  __syncthreads();
  const int lane = threadIdx.x % kSplitTileLines, w = threadIdx.x / kSplitTileLines;
  c = c0 + w;
  l = l0 + lane;
  if (c >= N || l >= lines) c = -1;
  return sx + lane * S::RS + w * K;
}

template <typename T, int K>
__device__ __forceinline__ void sweep_split_tile(const OpTab<T, K>& tab, const SweepArgs<T>& a,
                                                 int64_t blk, T* sx) {
  int64_t l;
  int c;
  const T* xw = split_stage<T, K>(a.in[0], a.lines, a.N, a.n, blk, sx, l, c);
  if (c < 0) return;
  const int64_t base = l * a.n;  // axis 0: line l starts at l n
  if (c >= 2 && c <= a.N - 2) {
    sweep_cell<T, K, 0, true>(tab, a, base, c, nullptr, xw);
  } else {
    int cls[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int g = c * K + q;
      cls[q] = (g >= 1) ? row_class<K>(g, a.N) : 0;
    }
    sweep_cell<T, K, 0, false>(tab, a, base, c, cls, xw);
  }
}

template <typename T, int K, int KIND>
__global__ void __launch_bounds__(128) sweep_kernel(const __grid_constant__ OpTab<T, K> tab,
                                                    const SweepArgs<T> a) {
  if constexpr (KIND == 0) {
    __shared__ T sx[kSplitTileLines * SplitTile<K>::RS];
    sweep_split_tile<T, K>(tab, a, blockIdx.x, sx);
  } else {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= a.lines * a.N) return;
    sweep_thread<T, K, KIND>(tab, a, tid);
  }
}

// ---------------------------------------------------------------------------
// vertex-patch kernels
// ---------------------------------------------------------------------------
// Asynchronous global -> shared copy of one value (cp.async, no register
// staging, so all of a thread's window loads are in flight together); when
// `valid` is false no byte is read and the value is filled with zero.  The
// caller waits with async_copy_wait before the barrier that publishes it.
template <typename T>
__device__ __forceinline__ void async_copy_or_zero(T* dst, const T* src, bool valid) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte values");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const unsigned bytes = valid ? (unsigned)sizeof(T) : 0u;
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src),
               "n"(sizeof(T)), "r"(bytes)
               : "memory");
}

// Asynchronous global -> shared copy of 16 bytes through L2 (cp.async.cg); both
// addresses must be 16-byte aligned.
__device__ __forceinline__ void async_copy_chunk16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void async_copy_wait() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <typename T>
struct PatchArgs {
  const T* r;
  T* x;
  const int* verts;   // vertex ids sum_a (v_a - 1) (N-1)^a
  int count;
  int N, n;
  double scale;
  const T* dinv;      // FDM: 1 / (sum_a lambda_a) per type combo slot x m^d
  const T* ainv;      // exact: m^d x m^d per type combo slot
};

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

template <typename T, int D, int K>
struct PatchCfg {
  static constexpr int M = 2 * K - 1;
  static constexpr int MD = ipow(M, D);
  static constexpr int BUF = 32768 / (2 * MD * (int)sizeof(T));
  static constexpr int PB = BUF < 1 ? 1 : (BUF > 64 ? 64 : BUF);  // patches per block
};

template <int D>
__device__ __forceinline__ void patch_geom(int vid, int N, int n, int K, int* type, int64_t& base,
                                           int& combo) {
  int64_t b = 0, stride = 1;
  combo = 0;
  int mul = 1;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const int v = vid % (N - 1) + 1;
    vid /= (N - 1);
    const int t = (N == 2) ? 3 : (v == 1 ? 1 : (v == N - 1 ? 2 : 0));
    type[a] = t;
    combo += t * mul;
    mul *= 4;
    b += (int64_t)(K * (v - 1)) * stride;  // first patch node K(v-1)+1 -> index K(v-1)
    stride *= n;
  }
  base = b;
}

template <int D, int M>
__device__ __forceinline__ void local_coords(int l, int* c) {
#pragma unroll
  for (int a = 0; a < D; ++a) {
    c[a] = l % M;
    l /= M;
  }
}

// x += scale * R_v^T (S (x) S) D^-1 (S (x) S)^T R_v r   for the patches in verts
template <typename T, int D, int K, bool ATOMIC>
__global__ void __launch_bounds__(256) patch_fdm_kernel(const __grid_constant__ FdmTab<T, K> tab,
                                                        const PatchArgs<T> a) {
  using C = PatchCfg<T, D, K>;
  constexpr int M = C::M, MD = C::MD, PB = C::PB;
  __shared__ T sS[4][M][M];
  __shared__ T bufA[PB * MD];
  __shared__ T bufB[PB * MD];
  __shared__ int sType[PB][D];
  __shared__ int sCombo[PB];
  __shared__ int64_t sBase[PB];

  const int first = blockIdx.x * PB;
  const int np = min(PB, a.count - first);
  if (np <= 0) return;
  for (int e = threadIdx.x; e < 4 * M * M; e += blockDim.x)
    (&sS[0][0][0])[e] = (&tab.S[0][0][0])[e];
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    int64_t base;
    patch_geom<D>(a.verts[first + p], a.N, a.n, K, sType[p], base, sCombo[p]);
    sBase[p] = base;
  }
  __syncthreads();
  const int64_t n = a.n, n2 = n * n;
  const int tot = np * MD;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int p = e / MD, l = e % MD;
    int c[3] = {0, 0, 0};
    local_coords<D, M>(l, c);
    const int64_t gi = sBase[p] + c[0] + c[1] * n + (D == 3 ? c[2] * n2 : 0);
    async_copy_or_zero(bufA + e, a.r + gi, true);
  }
  async_copy_wait();
  __syncthreads();
  T* in = bufA;
  T* out = bufB;
  // S^T along every axis (the last one divides by the eigenvalue sums), then S
  // along every axis; one half-line per item, folded for interior axes
  constexpr int NL = MD / M;  // lines per axis and patch
#pragma unroll
  for (int pass = 0; pass < 2 * D; ++pass) {
    const int ax = pass < D ? pass : pass - D;
    const int st = ipow(M, ax);
    for (int e = threadIdx.x; e < 2 * np * NL; e += blockDim.x) {
      const int q_ = e / (NL), q = e - q_ * (NL);  // item (half, patch, q)
      const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
      const int l0 = (q / st) * st * M + q % st;  // first element of line q
      const int t = sType[p][ax];
      const T* S = &sS[t][0][0];
      const T* src = in + p * MD + l0;
      T* dst = out + p * MD + l0;
      if (pass == D - 1)
        fdm_line<T, K, true, kFdmScaled>(half, S, t == 0, src, st, dst, st,
                                         a.dinv + (int64_t)sCombo[p] * MD + l0, st, T(0));
      else if (pass < D)
        fdm_line<T, K, true, kFdmStore>(half, S, t == 0, src, st, dst, st, nullptr, 0, T(0));
      else
        fdm_line<T, K, false, kFdmStore>(half, S, t == 0, src, st, dst, st, nullptr, 0, T(0));
    }
    __syncthreads();
    T* tmp = in;
    in = out;
    out = tmp;
  }
  const T sc = (T)a.scale;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int p = e / MD, l = e % MD;
    int c[3] = {0, 0, 0};
    local_coords<D, M>(l, c);
    const int64_t gi = sBase[p] + c[0] + c[1] * n + (D == 3 ? c[2] * n2 : 0);
    const T v = sc * in[e];
    if (ATOMIC)
      atomicAdd(a.x + gi, v);
    else
      a.x[gi] += v;
  }
}

// exact local solver: y_v = Ainv[combo] r_v, one patch per block row pass
template <typename T, int D, int K, bool ATOMIC>
__global__ void __launch_bounds__(256) patch_exact_kernel(const PatchArgs<T> a) {
  using C = PatchCfg<T, D, K>;
  constexpr int M = C::M, MD = C::MD;
  constexpr int PB = C::PB;
  __shared__ T buf[PB * MD];
  __shared__ int sType[PB][D];
  __shared__ int sCombo[PB];
  __shared__ int64_t sBase[PB];
  const int first = blockIdx.x * PB;
  const int np = min(PB, a.count - first);
  if (np <= 0) return;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    int64_t base;
    patch_geom<D>(a.verts[first + p], a.N, a.n, K, sType[p], base, sCombo[p]);
    sBase[p] = base;
  }
  __syncthreads();
  const int64_t n = a.n, n2 = n * n;
  const int tot = np * MD;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int p = e / MD, l = e % MD;
    int c[3] = {0, 0, 0};
    local_coords<D, M>(l, c);
    async_copy_or_zero(buf + e, a.r + sBase[p] + c[0] + c[1] * n + (D == 3 ? c[2] * n2 : 0), true);
  }
  async_copy_wait();
  __syncthreads();
  const T sc = (T)a.scale;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int p = e / MD, i = e % MD;
    const T* A = a.ainv + (int64_t)sCombo[p] * MD * MD;  // symmetric: read row j, column i
    const T* rv = buf + p * MD;
    T s = T(0);
    for (int j = 0; j < MD; ++j) s = fma(__ldg(A + (int64_t)j * MD + i), rv[j], s);
    int c[3] = {0, 0, 0};
    local_coords<D, M>(i, c);
    const int64_t gi = sBase[p] + c[0] + c[1] * n + (D == 3 ? c[2] * n2 : 0);
    if (ATOMIC)
      atomicAdd(a.x + gi, sc * s);
    else
      a.x[gi] += sc * s;
  }
}

// patch tensors as the columns of a matrix (column j = patch verts[j], local
// node l at row l): R[l + j MD] = r[node], and the reverse x[node] += Y[...]
template <typename T, int D, int K>
__global__ void __launch_bounds__(256) patch_gather_kernel(const T* __restrict__ r,
                                                           const int* verts, int count, int N,
                                                           int n, T* __restrict__ R) {
  using C = PatchCfg<T, D, K>;
  constexpr int M = C::M, MD = C::MD;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)count * MD) return;
  const int j = (int)(e / MD), l = (int)(e % MD);
  int type[D], combo;
  int64_t base;
  patch_geom<D>(verts[j], N, n, K, type, base, combo);
  int c[3] = {0, 0, 0};
  local_coords<D, M>(l, c);
  const int64_t nn = n;
  R[e] = r[base + c[0] + c[1] * nn + (D == 3 ? c[2] * nn * nn : 0)];
}

template <typename T, int D, int K, bool ATOMIC>
__global__ void __launch_bounds__(256) patch_scatter_kernel(const T* __restrict__ Y,
                                                            const int* verts, int count, int N,
                                                            int n, T* x) {
  using C = PatchCfg<T, D, K>;
  constexpr int M = C::M, MD = C::MD;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)count * MD) return;
  const int j = (int)(e / MD), l = (int)(e % MD);
  int type[D], combo;
  int64_t base;
  patch_geom<D>(verts[j], N, n, K, type, base, combo);
  int c[3] = {0, 0, 0};
  local_coords<D, M>(l, c);
  const int64_t nn = n;
  T* o = x + base + c[0] + c[1] * nn + (D == 3 ? c[2] * nn * nn : 0);
  if (ATOMIC)
    atomicAdd(o, Y[e]);
  else
    *o += Y[e];
}

// ---------------------------------------------------------------------------
// transfers: embedding prolongation and its transpose, one axis per pass
// ---------------------------------------------------------------------------
template <typename T>
struct XferArgs {
  const T* in;
  T* out;
  int d, axis;
  int dims_in[3], dims_out[3];
  int64_t str_in[3], str_out[3];
  int64_t lines;
  int Nc;       // coarse cells per direction
  int nc, nf;   // interior nodes per direction: coarse, fine
  bool add;     // out += (prolongation into x) instead of out =
  float* out32;  // restriction: the result also rounded to FP32 here (nullptr: not)
};

// prolongation along an axis: thread <-> (line, coarse cell C); fine nodes
// 2KC + r (r = 0..2K-1) from coarse nodes KC + q (q = 0..K).
template <typename T, int K>
__device__ __forceinline__ void prolong_thread(const XferTab<T, K>& tab, const XferArgs<T>& a,
                                               int64_t tid) {
  int64_t line;
  int C;
  if (a.axis == 0) {
    line = tid / a.Nc;
    C = (int)(tid % a.Nc);
  } else {
    C = (int)(tid / a.lines);
    line = tid % a.lines;
  }
  const int64_t bi = line_offset(line, a.d, a.axis, a.dims_in, a.str_in);
  const int64_t bo = line_offset(line, a.d, a.axis, a.dims_out, a.str_out);
  const int64_t si = a.str_in[a.axis], so = a.str_out[a.axis];
  T w[K + 1];
#pragma unroll
  for (int q = 0; q <= K; ++q) {
    const int g = K * C + q;
    w[q] = (g >= 1 && g <= a.nc) ? a.in[bi + (int64_t)(g - 1) * si] : T(0);
  }
#pragma unroll
  for (int r = 0; r < 2 * K; ++r) {
    const int g = 2 * K * C + r;
    if (g < 1) continue;
    T s = T(0);
#pragma unroll
    for (int q = 0; q <= K; ++q) s = fma(tab.P[r][q], w[q], s);
    T* o = a.out + bo + (int64_t)(g - 1) * so;
    *o = a.add ? *o + s : s;
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(128) prolong_kernel(const __grid_constant__ XferTab<T, K> tab,
                                                      const XferArgs<T> a) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < a.lines * a.Nc) prolong_thread<T, K>(tab, a, tid);
}

// restriction along an axis: thread <-> (line, coarse cell C); coarse nodes KC+q
// (q = 0..K-1) from the fine nodes 2K(C-1) .. 2KC + 2K - 1.
template <typename T, int K>
__device__ __forceinline__ void restrict_thread(const XferTab<T, K>& tab, const XferArgs<T>& a,
                                                int64_t tid) {
  int64_t line;
  int C;
  if (a.axis == 0) {
    line = tid / a.Nc;
    C = (int)(tid % a.Nc);
  } else {
    C = (int)(tid / a.lines);
    line = tid % a.lines;
  }
  const int64_t bi = line_offset(line, a.d, a.axis, a.dims_in, a.str_in);
  const int64_t bo = line_offset(line, a.d, a.axis, a.dims_out, a.str_out);
  const int64_t si = a.str_in[a.axis], so = a.str_out[a.axis];
  T w[4 * K];
#pragma unroll
  for (int j = 0; j < 4 * K; ++j) {
    const int g = 2 * K * (C - 1) + j;
    w[j] = (g >= 1 && g <= a.nf) ? a.in[bi + (int64_t)(g - 1) * si] : T(0);
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const int g = K * C + q;
    if (g < 1) continue;
    T s = T(0);
    if (q == 0) {
#pragma unroll
      for (int r = 0; r < 2 * K; ++r) s = fma(tab.P[r][K], w[r], s);
    }
#pragma unroll
    for (int r = 0; r < 2 * K; ++r) s = fma(tab.P[r][q], w[2 * K + r], s);
    a.out[bo + (int64_t)(g - 1) * so] = s;
    if (a.out32) a.out32[bo + (int64_t)(g - 1) * so] = (float)s;
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(128) restrict_kernel(const __grid_constant__ XferTab<T, K> tab,
                                                       const XferArgs<T> a) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < a.lines * a.Nc) restrict_thread<T, K>(tab, a, tid);
}

template <typename T>
__global__ void add_kernel(T* y, const T* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

// ---------------------------------------------------------------------------
// dense symmetric matrix-vector product (coarse solve), FP64 matrix
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) dense_symv_kernel(int n, const double* __restrict__ A,
                                                         const T* __restrict__ in, T* out,
                                                         double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int j = 0; j < n; ++j) s = fma(A[(int64_t)j * n + i], (double)in[j], s);
  out[i] = (T)(scale * s);
}

}  // namespace bh
