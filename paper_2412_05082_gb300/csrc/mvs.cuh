// Fused kernel of one color of the colored multiplicative vertex-patch smoother
// (Sec. 3, colored MVS) in 2D:
//
//   for every patch v of the color:  x_v += omega A~_v^-1 R_v (b - A x)
//
// Patches of one color are A-orthogonal, so each patch needs the residual only
// on its own (2k-1)^2 interior nodes, and that residual depends only on x in the
// (4k+1)^2 window of nodes k(v_a - 2) .. k(v_a + 2) -- never on the interior of
// another patch of the same color (the window's corners, which may hold such
// values, are loaded but never used).  The kernel therefore computes the local
// residual by sum factorization inside the patch (x-split of the window rows,
// y-combination on the patch nodes), applies the fast-diagonalization inverse
// (Sec. 4.1) and adds the correction in place: one launch per color instead of
// a full-grid residual plus a patch launch.
//
// Work per patch (m = 2k-1, band nonzeros of the 1D M, L, B rows):
//   x-split: T_M on the 4k+1 window rows, T_L and T_B on the 2k+1 middle rows
//   y-combine: m^2 residual values, (5k+6) FMAs each
//   FDM: 4 m^3 FMAs + m^2 scalings
// Every stage is split into single output points; a warp's points share the
// row position q inside the cell, so the band loops are uniform and unrolled.
#pragma once
#include "kernels.cuh"

namespace bh {

template <typename T, int K>
struct MvsTab {
  OpTab<T, K> op;
  FdmTab<T, K> fdm;
};

template <typename T>
struct MvsArgs {
  T* x;
  const T* b;
  const int* verts;   // patches of one color, vertex ids sum_a (v_a - 1)(N-1)^a
  int count;
  int N, n;
  int pb;             // patches per block (runtime, <= Mvs2Cfg::PB_MAX)
  double ascale;      // A_l = ascale * A_ref
  double pscale;      // omega * h^(4-d)
  const T* dinv;      // 1 / (lambda_x + lambda_y) per type combination, m^2 each
};

template <typename T, int K>
struct Mvs2Cfg {
  static constexpr int M = 2 * K - 1;   // patch nodes per direction
  static constexpr int W = 4 * K + 1;   // window nodes per direction
  static constexpr int WM = 2 * K + 1;  // rows of T_L, T_B
  static constexpr int NC = 3 * K + 1, BW = 4 * K + 1;
  // values per patch: window, T_M, T_L, T_B, two m x m buffers
  static constexpr int PER = W * W + W * M + 2 * WM * M + 2 * M * M;
  static constexpr int TABLES = 3 * NC * BW + 4 * M * M;
  static constexpr int BUDGET = 96 * 1024;  // bytes of shared memory per block
  static constexpr int FIT = (BUDGET / (int)sizeof(T) - TABLES) / PER;
  static constexpr int PB_MAX = FIT < 1 ? 1 : (FIT > 32 ? 32 : FIT);
  static size_t smem_bytes(int pb) { return sizeof(T) * (size_t)(TABLES + pb * PER) + 64; }
};

// sum_t C[t + 2K] v[t * stride] over the band of operator OP at row position Q
template <typename T, int K, int OP, int Q>
__device__ __forceinline__ T band_dot(const T* c, const T* v, int stride) {
  T s = T(0);
#pragma unroll
  for (int t = band_lo(OP, Q, K); t <= band_hi(OP, Q, K); ++t)
    s = fma(c[t + 2 * K], v[t * stride], s);
  return s;
}

template <typename T, int K, int Q>
__device__ __forceinline__ void xsplit_point(const T* sM, const T* sL, const T* sB, int cls,
                                             const T* xr, T* tm, T* tl, T* tb, bool mid) {
  constexpr int BW = 4 * K + 1;
  *tm = band_dot<T, K, 0, Q>(sM + cls * BW, xr, 1);
  if (mid) {
    *tl = band_dot<T, K, 1, Q>(sL + cls * BW, xr, 1);
    *tb = band_dot<T, K, 2, Q>(sB + cls * BW, xr, 1);
  }
}

template <typename T, int K, int Q>
__device__ __forceinline__ T ycombine_point(const T* sM, const T* sL, const T* sB, int cls,
                                            const T* cm, const T* cl, const T* cb, int stride) {
  constexpr int BW = 4 * K + 1;
  return band_dot<T, K, 2, Q>(sB + cls * BW, cm, stride) +
         T(2) * band_dot<T, K, 1, Q>(sL + cls * BW, cl, stride) +
         band_dot<T, K, 0, Q>(sM + cls * BW, cb, stride);
}

// compile-time dispatch over the row position q = 0..K-1 (uniform per warp)
#define BH_Q_SWITCH(q, CALL)                         \
  switch (q) {                                       \
    case 0: CALL(0); break;                          \
    case 1: if constexpr (K > 1) { CALL(1); } break; \
    case 2: if constexpr (K > 2) { CALL(2); } break; \
    case 3: if constexpr (K > 3) { CALL(3); } break; \
    case 4: if constexpr (K > 4) { CALL(4); } break; \
    case 5: if constexpr (K > 5) { CALL(5); } break; \
    case 6: if constexpr (K > 6) { CALL(6); } break; \
  }

template <typename T, int K>
__global__ void __launch_bounds__(256) mvs2_color_kernel(const __grid_constant__ MvsTab<T, K> tab,
                                                         const MvsArgs<T> a) {
  using C = Mvs2Cfg<T, K>;
  constexpr int M = C::M, W = C::W, WM = C::WM, NC = C::NC, BW = C::BW, MM = M * M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sM = reinterpret_cast<T*>(smem_raw);
  T* sL = sM + NC * BW;
  T* sB = sL + NC * BW;
  T* sS = sB + NC * BW;  // [4][M][M]
  const int pb = a.pb;
  T* sX = sS + 4 * MM;         // [pb][W][W]
  T* sTM = sX + pb * W * W;    // [pb][W][M]
  T* sTL = sTM + pb * W * M;   // [pb][WM][M]
  T* sTB = sTL + pb * WM * M;  // [pb][WM][M]
  T* sR = sTB + pb * WM * M;   // [pb][M][M]
  T* sF = sR + pb * MM;        // [pb][M][M]
  __shared__ int sV[32][2], sTy[32][2], sCombo[32];

  const int first = blockIdx.x * pb;
  const int np = min(pb, a.count - first);
  if (np <= 0) return;
  const int N = a.N, n = a.n;
  for (int e = threadIdx.x; e < NC * BW; e += blockDim.x) {
    sM[e] = (&tab.op.M[0][0])[e];
    sL[e] = (&tab.op.L[0][0])[e];
    sB[e] = (&tab.op.B[0][0])[e];
  }
  for (int e = threadIdx.x; e < 4 * MM; e += blockDim.x) sS[e] = (&tab.fdm.S[0][0][0])[e];
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const int vid = a.verts[first + p];
    const int v0 = vid % (N - 1) + 1, v1 = vid / (N - 1) + 1;
    const int t0 = (N == 2) ? 3 : (v0 == 1 ? 1 : (v0 == N - 1 ? 2 : 0));
    const int t1 = (N == 2) ? 3 : (v1 == 1 ? 1 : (v1 == N - 1 ? 2 : 0));
    sV[p][0] = v0;
    sV[p][1] = v1;
    sTy[p][0] = t0;
    sTy[p][1] = t1;
    sCombo[p] = t0 + 4 * t1;
  }
  __syncthreads();
  // window of x: global nodes K(v_a - 2) + w, zero outside the interior 1..n
  for (int e = threadIdx.x; e < np * W * W; e += blockDim.x) {
    const int p = e / (W * W), wy = (e / W) % W, wx = e % W;
    const int gx = K * (sV[p][0] - 2) + wx, gy = K * (sV[p][1] - 2) + wy;
    sX[e] = (gx >= 1 && gx <= n && gy >= 1 && gy <= n) ? a.x[(int64_t)(gy - 1) * n + (gx - 1)]
                                                       : T(0);
  }
  __syncthreads();
  // x-split, one point (patch column j, patch p, window row wy) per item; j outermost
  for (int e = threadIdx.x; e < M * np * W; e += blockDim.x) {
    const int wy = e % W, p = (e / W) % np, j = e / (W * np) + 1;
    const int q = j % K;
    const int gx = K * (sV[p][0] - 1) + j;
    const int cls = sTy[p][0] == 0 ? q : row_class<K>(gx, N);
    const bool mid = wy >= K && wy <= 3 * K;
    const int r = mid ? wy - K : 0;
    const T* xr = sX + (p * W + wy) * W + K + j;
    T* tm = sTM + (p * W + wy) * M + (j - 1);
    T* tl = sTL + (p * WM + r) * M + (j - 1);
    T* tb = sTB + (p * WM + r) * M + (j - 1);
#define BH_CALL(QQ) xsplit_point<T, K, QQ>(sM, sL, sB, cls, xr, tm, tl, tb, mid)
    BH_Q_SWITCH(q, BH_CALL)
#undef BH_CALL
  }
  __syncthreads();
  // y-combination and residual r = b - A x on the patch nodes; patch row i outermost
  const T asc = (T)a.ascale;
  for (int e = threadIdx.x; e < M * np * M; e += blockDim.x) {
    const int j = e % M, p = (e / M) % np, i = e / (M * np) + 1;
    const int q = i % K;
    const int gy = K * (sV[p][1] - 1) + i;
    const int cls = sTy[p][1] == 0 ? q : row_class<K>(gy, N);
    const T* cm = sTM + (p * W + K + i) * M + j;
    const T* cl = sTL + (p * WM + i) * M + j;
    const T* cb = sTB + (p * WM + i) * M + j;
    T y = T(0);
#define BH_CALL(QQ) y = ycombine_point<T, K, QQ>(sM, sL, sB, cls, cm, cl, cb, M)
    BH_Q_SWITCH(q, BH_CALL)
#undef BH_CALL
    const int gx = K * (sV[p][0] - 1) + j + 1;
    sR[(p * M + (i - 1)) * M + j] = a.b[(int64_t)(gy - 1) * n + (gx - 1)] - asc * y;
  }
  __syncthreads();
  // fast diagonalization: F = R S_x (rows), R = S_y^T F scaled (columns)
  for (int e = threadIdx.x; e < np * MM; e += blockDim.x) {
    const int p = e / MM, i = (e / M) % M, c = e % M;
    const T* S = sS + sTy[p][0] * MM;  // S[j][c]: eigenvector c, component j
    const T* r = sR + (p * M + i) * M;
    T s = T(0);
#pragma unroll
    for (int j = 0; j < M; ++j) s = fma(S[j * M + c], r[j], s);
    sF[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < np * MM; e += blockDim.x) {
    const int p = e / MM, c1 = (e / M) % M, c0 = e % M;
    const T* S = sS + sTy[p][1] * MM;
    const T* f = sF + p * MM + c0;
    T s = T(0);
#pragma unroll
    for (int i = 0; i < M; ++i) s = fma(S[i * M + c1], f[i * M], s);
    sR[e] = s * a.dinv[(int64_t)sCombo[p] * MM + c1 * M + c0];
  }
  __syncthreads();
  // back transform: F = S_y G (columns), x_v += pscale * F S_x^T (rows)
  for (int e = threadIdx.x; e < np * MM; e += blockDim.x) {
    const int p = e / MM, i = (e / M) % M, c0 = e % M;
    const T* S = sS + sTy[p][1] * MM;
    const T* g = sR + p * MM + c0;
    T s = T(0);
#pragma unroll
    for (int c1 = 0; c1 < M; ++c1) s = fma(S[i * M + c1], g[c1 * M], s);
    sF[e] = s;
  }
  __syncthreads();
  const T ps = (T)a.pscale;
  for (int e = threadIdx.x; e < np * MM; e += blockDim.x) {
    const int p = e / MM, i = (e / M) % M, j = e % M;
    const T* S = sS + sTy[p][0] * MM;
    const T* f = sF + (p * M + i) * M;
    T s = T(0);
#pragma unroll
    for (int c = 0; c < M; ++c) s = fma(S[j * M + c], f[c], s);
    const int gx = K * (sV[p][0] - 1) + j + 1, gy = K * (sV[p][1] - 1) + i + 1;
    a.x[(int64_t)(gy - 1) * n + (gx - 1)] += ps * s;
  }
}

}  // namespace bh
