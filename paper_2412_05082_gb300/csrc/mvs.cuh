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
//   FDM: 4 m^3 FMAs + m^2 scalings (tiles touching the boundary), or the
//   folded form, 2 m (4k^2 + k - 3) operations (interior tiles)
// Every stage is split into half-lines or single points so that all threads of
// a warp run the same FP64 instruction stream.
#pragma once
#include "kernels.cuh"

namespace bh {

template <typename T, int K>
struct MvsTab {
  OpTab<T, K> op;
  FdmTab<T, K> fdm;
};

// The interior (canonical) row classes 0..K-1 of M, L, B and the interior
// patch type's eigenvectors: all that the interior tiles of the fused kernel
// read (a small kernel parameter for the batched form's FP32 launches).
template <typename T, int K>
struct CanonTab {
  T M[K][4 * K + 1];
  T L[K][4 * K + 1];
  T B[K][4 * K + 1];
  T S[1][2 * K - 1][2 * K - 1];
};

// the first table when DIRECT, else the second (of another type)
template <bool DIRECT, typename A, typename B>
__device__ __forceinline__ const auto& pick_tab(const A& a, const B& b) {
  if constexpr (DIRECT)
    return a;
  else
    return b;
}

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
  const void* dtab;   // single-problem kernel: device copy of its Tables<T, K> (the tables
                      // staged in shared memory are read from it with coalesced loads)
};

template <typename T, int K>
struct Mvs2Cfg {
  static constexpr int M = 2 * K - 1;   // patch nodes per direction
  static constexpr int W = 4 * K + 1;   // window nodes per direction
  static constexpr int WM = 2 * K + 1;  // rows of T_L, T_B
  static constexpr int NC = 3 * K + 1, BW = 4 * K + 1;
  // FP32: b and x on the patch nodes are copied to shared memory together
  // with the window, so that no stage after the window copy waits on a global
  // load (the FP32 kernel is bound by load latency, the FP64 one by its pipe)
  static constexpr bool PREFETCH = sizeof(T) == 4;
  // FP32, k <= 4: window rows of tiles away from the boundary are copied as
  // 16-byte chunks; each shared-memory row starts on a 16-byte boundary and
  // holds its row at the row's own offset 0..3 (the global row start modulo 4
  // values).  For k >= 5 the padded rows would cost a resident block per SM.
  static constexpr bool VECWIN = sizeof(T) == 4 && K <= 4;
  static constexpr int CH = (W + 3 + 3) / 4;      // 16-byte chunks per window row
  static constexpr int WS = VECWIN ? 4 * CH : W;  // shared-memory row stride of the window
  static constexpr int WIN = W * WS;
  // values per patch: window, T_M, T_L, T_B (and the prefetched b and x, or
  // in the interior form b and the residual); the m x m buffers of the
  // residual and the FDM reuse space whose contents are no longer needed
  static constexpr int PER = WIN + W * M + 2 * WM * M + (PREFETCH ? 2 * M * M : 0);
  static_assert(2 * M * M <= W * W, "FDM buffers must fit in the window region");
  static_assert(M * M <= W * M, "the FDM buffer must fit in the T_M region");
  // M, L, B class tables, the four S, and the interior type's 1 / (l_x + l_y),
  // padded so that the window starts on a 16-byte boundary
  static constexpr int TABLES = (3 * NC * BW + 5 * M * M + 3) / 4 * 4;
  static constexpr int BUDGET = 110 * 1024;  // bytes of shared memory per block (2 per SM)
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

// Half-lines: the 2k-1 patch positions along an axis split into half 0 =
// positions 1..k (the k-1 nodes inside cell v-1 and the vertex) and half 1 =
// positions k+1..2k-1 (inside cell v).  A thread handles one half-line with
// its row positions q unrolled at compile time, so all threads of a warp run
// the same FP64 instruction stream (masked lanes would still occupy the FP64
// pipe).  cls(pos) is q for patches away from the boundary and the row class
// of the global node otherwise.
template <int K, int HALF>
struct Half {
  static constexpr int J0 = HALF == 0 ? 1 : K + 1;
  static constexpr int J1 = HALF == 0 ? K : 2 * K - 1;
};

// T_P[pos] = (P x)(pos) along a window row for P = M (OPS = 1) or P = L, B (OPS = 2)
template <typename T, int K, int HALF, int OPS>
__device__ __forceinline__ void xsplit_half(const T* sM, const T* sL, const T* sB, bool canon,
                                            int g0, int N, const T* xr, T* o0, T* o1) {
  constexpr int BW = 4 * K + 1;
#pragma unroll
  for (int j = Half<K, HALF>::J0; j <= Half<K, HALF>::J1; ++j) {
    const int q = j % K;
    const int cls = canon ? q : row_class<K>(g0 + j, N);
    if (OPS == 1) {
      T s = T(0);
#pragma unroll
      for (int t = band_lo(0, j % K, K); t <= band_hi(0, j % K, K); ++t)
        s = fma(sM[cls * BW + t + 2 * K], xr[j + t], s);
      o0[j - 1] = s;
    } else {
      T sl = T(0), sb = T(0);
#pragma unroll
      for (int t = band_lo(1, j % K, K); t <= band_hi(1, j % K, K); ++t)
        sl = fma(sL[cls * BW + t + 2 * K], xr[j + t], sl);
#pragma unroll
      for (int t = band_lo(2, j % K, K); t <= band_hi(2, j % K, K); ++t)
        sb = fma(sB[cls * BW + t + 2 * K], xr[j + t], sb);
      o0[j - 1] = sl;
      o1[j - 1] = sb;
    }
  }
}

// r_i = b_i - ascale (B T_M + 2 L T_L + M T_B)_i along a patch column; cm = T_M
// column at window row K (patch position 0), cl, cb = T_L, T_B columns at their
// row 0 (window row K), stride M between rows; bcol = b at patch position 0 of
// the column (stride n), rcol = residual column (stride M).
template <typename T, int K, int HALF>
__device__ __forceinline__ void ycombine_half(const T* sM, const T* sL, const T* sB, bool canon,
                                              int g0, int N, const T* cm, const T* cl,
                                              const T* cb, const T* bcol, int64_t n, T asc,
                                              T* rcol) {
  constexpr int BW = 4 * K + 1, M = 2 * K - 1;
#pragma unroll
  for (int i = Half<K, HALF>::J0; i <= Half<K, HALF>::J1; ++i) {
    const int q = i % K;
    const int cls = canon ? q : row_class<K>(g0 + i, N);
    T sb = T(0), sl = T(0), sm = T(0);
#pragma unroll
    for (int t = band_lo(2, i % K, K); t <= band_hi(2, i % K, K); ++t)
      sb = fma(sB[cls * BW + t + 2 * K], cm[(i + t) * M], sb);
#pragma unroll
    for (int t = band_lo(0, i % K, K); t <= band_hi(0, i % K, K); ++t) {
      sl = fma(sL[cls * BW + t + 2 * K], cl[(i + t) * M], sl);
      sm = fma(sM[cls * BW + t + 2 * K], cb[(i + t) * M], sm);
    }
    rcol[(i - 1) * M] = bcol[(int64_t)(i - 1) * n] - asc * (sb + T(2) * sl + sm);
  }
}

// Asynchronous copies of b and x on the m x m patch nodes of the tile's
// patches into sBv, sXv ([patch][row][column]).  Patch nodes always lie in the
// interior 1..n.  Values of x on a patch's own nodes are changed by no other
// patch of its color, so the copy stays current until the patch's update.
// WITH_X false: b only.
template <typename T, int K, bool WITH_X = true>
__device__ __forceinline__ void prefetch_patch_nodes(const MvsArgs<T>& a, int np,
                                                     const int (*sV)[2], T* sBv, T* sXv) {
  constexpr int M = 2 * K - 1, MM = M * M;
  const int64_t n = a.n;
  for (int e = threadIdx.x; e < np * MM; e += blockDim.x) {
    const int p = e / MM, i = (e / M) % M, j = e % M;
    const int64_t gi = (int64_t)(K * (sV[p][1] - 1) + i) * n + (K * (sV[p][0] - 1) + j);
    async_copy_or_zero(sBv + e, a.b + gi, true);
    if constexpr (WITH_X) async_copy_or_zero(sXv + e, a.x + gi, true);
  }
}

// Patches first .. first + np - 1 of a.verts by one thread block; tables read
// from `op` / `fdm` (kernel parameters or device memory) into shared memory.
// smem_raw: dynamic shared memory of at least Mvs2Cfg::smem_bytes(a.pb) bytes.
template <typename T, int K>
__device__ __forceinline__ void mvs2_tile(const OpTab<T, K>& op, const FdmTab<T, K>& fdm,
                                          const MvsArgs<T>& a, int first, int np,
                                          unsigned char* smem_raw) {
  using C = Mvs2Cfg<T, K>;
  constexpr int M = C::M, W = C::W, WM = C::WM, NC = C::NC, BW = C::BW, MM = M * M;
  T* sM = reinterpret_cast<T*>(smem_raw);
  T* sL = sM + NC * BW;
  T* sB = sL + NC * BW;
  T* sS = sB + NC * BW;  // [4][M][M]
  const int pb = a.pb;
  T* sX = reinterpret_cast<T*>(smem_raw) + C::TABLES;  // [pb][W][W] (in a [pb][W][WS] region)
  T* sTM = sX + pb * C::WIN;   // [pb][W][M]
  T* sTL = sTM + pb * W * M;   // [pb][WM][M]
  T* sTB = sTL + pb * WM * M;  // [pb][WM][M]
  T* sR = sX;                  // [pb][M][M], over the window after the x-split
  T* sF = sR + pb * MM;        // [pb][M][M]
  T* sBv = sTB + pb * WM * M;  // [pb][M][M] b on the patch nodes (PREFETCH)
  T* sXv = sBv + pb * MM;      // [pb][M][M] x on the patch nodes (PREFETCH)
  __shared__ int sV[32][2], sTy[32][2], sCombo[32];

  if (np <= 0) return;
  const int N = a.N, n = a.n;
  for (int e = threadIdx.x; e < NC * BW; e += blockDim.x) {
    sM[e] = (&op.M[0][0])[e];
    sL[e] = (&op.L[0][0])[e];
    sB[e] = (&op.B[0][0])[e];
  }
  for (int e = threadIdx.x; e < 4 * MM; e += blockDim.x) sS[e] = (&fdm.S[0][0][0])[e];
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
    const bool in = gx >= 1 && gx <= n && gy >= 1 && gy <= n;
    async_copy_or_zero(sX + e, a.x + (in ? (int64_t)(gy - 1) * n + (gx - 1) : 0), in);
  }
  if constexpr (C::PREFETCH) prefetch_patch_nodes<T, K>(a, np, sV, sBv, sXv);
  async_copy_wait();
  __syncthreads();
  // x-split: T_M on every window row, one half-line (half, patch, row) per item
  for (int e = threadIdx.x; e < 2 * np * W; e += blockDim.x) {
    const int q_ = e / (W), wy = e - q_ * (W);  // item (half, patch, wy)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const T* xr = sX + (p * W + wy) * W + K;  // xr[j] = window column K + j
    T* tm = sTM + (p * W + wy) * M;
    const bool canon = sTy[p][0] == 0;
    const int g0 = K * (sV[p][0] - 1);       // global node of patch position j: g0 + j
    if (half == 0)
      xsplit_half<T, K, 0, 1>(sM, sL, sB, canon, g0, N, xr, tm, nullptr);
    else
      xsplit_half<T, K, 1, 1>(sM, sL, sB, canon, g0, N, xr, tm, nullptr);
  }
  // T_L and T_B on the 2k+1 middle window rows
  for (int e = threadIdx.x; e < 2 * np * WM; e += blockDim.x) {
    const int q_ = e / (WM), r = e - q_ * (WM);  // item (half, patch, r)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const T* xr = sX + (p * W + K + r) * W + K;
    T* tl = sTL + (p * WM + r) * M;
    T* tb = sTB + (p * WM + r) * M;
    const bool canon = sTy[p][0] == 0;
    const int g0 = K * (sV[p][0] - 1);
    if (half == 0)
      xsplit_half<T, K, 0, 2>(sM, sL, sB, canon, g0, N, xr, tl, tb);
    else
      xsplit_half<T, K, 1, 2>(sM, sL, sB, canon, g0, N, xr, tl, tb);
  }
  __syncthreads();
  // y-combination and residual r = b - A x on the patch nodes, one half-column per item
  const T asc = (T)a.ascale;
  for (int e = threadIdx.x; e < 2 * np * M; e += blockDim.x) {
    const int q_ = e / (M), j = e - q_ * (M);  // item (half, patch, j)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const T* cm = sTM + (p * W + K) * M + j;
    const T* cl = sTL + (p * WM) * M + j;
    const T* cb = sTB + (p * WM) * M + j;
    const bool canon = sTy[p][1] == 0;
    const int g0 = K * (sV[p][1] - 1);
    const int gx = K * (sV[p][0] - 1) + j + 1;
    // b at patch position 1 (global row g0 + 1) of the column, and its row stride
    const T* bcol = C::PREFETCH ? sBv + p * MM + j : a.b + (int64_t)g0 * n + (gx - 1);
    const int64_t bs = C::PREFETCH ? M : n;
    T* rcol = sR + p * M * M + j;
    if (half == 0)
      ycombine_half<T, K, 0>(sM, sL, sB, canon, g0, N, cm, cl, cb, bcol, bs, asc, rcol);
    else
      ycombine_half<T, K, 1>(sM, sL, sB, canon, g0, N, cm, cl, cb, bcol, bs, asc, rcol);
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
    T* xo = a.x + (int64_t)(gy - 1) * n + (gx - 1);
    if constexpr (C::PREFETCH)
      *xo = sXv[e] + ps * s;
    else
      *xo += ps * s;
  }
}

// ---- interior tiles --------------------------------------------------------
// A tile whose patches all lie away from the boundary (2 <= v_a <= N-2) meets
// only the canonical row classes q = j mod K and the interior patch type in
// both directions.  Its coefficients are then read from shared memory at
// compile-time offsets (one broadcast load each), and every thread first
// loads the window values of its half-line into registers, so that each FP64
// FMA needs one shared-memory load instead of two.  The interior 1D
// pencil is centrosymmetric, so the FDM lines take the folded form (even and
// odd eigenvectors: 2K^2 + K - 2 operations per forward line and 2K^2 - 1 per
// backward line instead of (2K-1)^2).

// T_M along a window row: o[j - 1] = (M x)(j) for the half's positions j.  The
// window values live in registers, so each output is stored as soon as it is
// formed.
template <typename T, int K, int HALF, typename OpT>
__device__ __forceinline__ void xsplit_m_canon(const OpT& op, const T* xr, T* o) {
  constexpr int J0 = Half<K, HALF>::J0, J1 = Half<K, HALF>::J1;
  constexpr int A = HALF == 0 ? 0 : K, Z = 2 * K;  // nodes read: xr[A .. Z]
  T w[Z - A + 1];
#pragma unroll
  for (int u = 0; u <= Z - A; ++u) w[u] = xr[A + u];
#pragma unroll
  for (int j = J0; j <= J1; ++j) {
    const int q = j % K;
    T s = T(0);
#pragma unroll
    for (int t = band_lo(0, q, K); t <= band_hi(0, q, K); ++t)
      s = fma(op.M[q][t + 2 * K], w[j + t - A], s);
    o[j - 1] = s;
  }
}

// T_L and T_B along a middle window row
template <typename T, int K, int HALF, typename OpT>
__device__ __forceinline__ void xsplit_lb_canon(const OpT& op, const T* xr, T* ol,
                                                T* ob) {
  constexpr int J0 = Half<K, HALF>::J0, J1 = Half<K, HALF>::J1;
  constexpr int A = HALF == 0 ? -K : 0, Z = 3 * K;  // nodes read: xr[A .. Z]
  T w[Z - A + 1];
#pragma unroll
  for (int u = 0; u <= Z - A; ++u) w[u] = xr[A + u];
#pragma unroll
  for (int j = J0; j <= J1; ++j) {
    const int q = j % K;
    T sl = T(0), sb = T(0);
#pragma unroll
    for (int t = band_lo(1, q, K); t <= band_hi(1, q, K); ++t)
      sl = fma(op.L[q][t + 2 * K], w[j + t - A], sl);
#pragma unroll
    for (int t = band_lo(2, q, K); t <= band_hi(2, q, K); ++t)
      sb = fma(op.B[q][t + 2 * K], w[j + t - A], sb);
    ol[j - 1] = sl;
    ob[j - 1] = sb;
  }
}

// residual on a half-column: r_i = b_i - ascale (B T_M + 2 L T_L + M T_B)_i
// (pointers as in ycombine_half), accumulated operator by operator
template <typename T, int K, int HALF, typename OpT>
__device__ __forceinline__ void ycombine_canon(const OpT& op, const T* cm, const T* cl,
                                               const T* cb, const T* bcol, int64_t n, T asc,
                                               T* rcol) {
  constexpr int M = 2 * K - 1;
  constexpr int I0 = Half<K, HALF>::J0, I1 = Half<K, HALF>::J1, NI = I1 - I0 + 1;
  T acc[NI];
  {  // B on T_M: rows i + t in [A, 3K]
    constexpr int A = HALF == 0 ? -K : 0, Z = 3 * K;
    T w[Z - A + 1];
#pragma unroll
    for (int u = 0; u <= Z - A; ++u) w[u] = cm[(A + u) * M];
#pragma unroll
    for (int i = I0; i <= I1; ++i) {
      const int q = i % K;
      T s = T(0);
#pragma unroll
      for (int t = band_lo(2, q, K); t <= band_hi(2, q, K); ++t)
        s = fma(op.B[q][t + 2 * K], w[i + t - A], s);
      acc[i - I0] = s;
    }
  }
  {  // 2 L on T_L: rows i + t in [A, 2K]
    constexpr int A = HALF == 0 ? 0 : K, Z = 2 * K;
    T w[Z - A + 1];
#pragma unroll
    for (int u = 0; u <= Z - A; ++u) w[u] = cl[(A + u) * M];
#pragma unroll
    for (int i = I0; i <= I1; ++i) {
      const int q = i % K;
      T s = T(0);
#pragma unroll
      for (int t = band_lo(1, q, K); t <= band_hi(1, q, K); ++t)
        s = fma(op.L[q][t + 2 * K], w[i + t - A], s);
      acc[i - I0] = fma(T(2), s, acc[i - I0]);
    }
  }
  {  // M on T_B
    constexpr int A = HALF == 0 ? 0 : K, Z = 2 * K;
    T w[Z - A + 1];
#pragma unroll
    for (int u = 0; u <= Z - A; ++u) w[u] = cb[(A + u) * M];
#pragma unroll
    for (int i = I0; i <= I1; ++i) {
      const int q = i % K;
#pragma unroll
      for (int t = band_lo(0, q, K); t <= band_hi(0, q, K); ++t)
        acc[i - I0] = fma(op.M[q][t + 2 * K], w[i + t - A], acc[i - I0]);
    }
  }
#pragma unroll
  for (int i = I0; i <= I1; ++i)
    rcol[(i - 1) * M] = bcol[(int64_t)(i - 1) * n] - asc * acc[i - I0];
}

// Folded FDM line of the interior type: forward (S^T v)_c for the half's
// eigenvectors c (half 0: the K even ones, half 1: the K-1 odd ones);
// put(c, value) receives each output.
template <typename T, int K, int HALF, typename Put, typename FdmT>
__device__ __forceinline__ void fdm_fwd_canon(const FdmT& fdm, const T* src, int is,
                                              Put put) {
  constexpr int M = 2 * K - 1;
  if (HALF == 0) {
    T f[K];
#pragma unroll
    for (int j = 0; j < K - 1; ++j) f[j] = src[j * is] + src[(M - 1 - j) * is];
    f[K - 1] = src[(K - 1) * is];
#pragma unroll
    for (int c = 0; c < K; ++c) {
      T s = T(0);
#pragma unroll
      for (int j = 0; j < K; ++j) s = fma(fdm.S[0][j][c], f[j], s);
      put(c, s);
    }
  } else {
    T f[K - 1];
#pragma unroll
    for (int j = 0; j < K - 1; ++j) f[j] = src[j * is] - src[(M - 1 - j) * is];
#pragma unroll
    for (int c = K; c < M; ++c) {
      T s = T(0);
#pragma unroll
      for (int j = 0; j < K - 1; ++j) s = fma(fdm.S[0][j][c], f[j], s);
      put(c, s);
    }
  }
}

// backward (S g)_i for the half's position pairs (i, M-1-i): half 0 takes
// i < K/2, half 1 the rest (with the middle position K-1)
template <typename T, int K, int HALF, typename Put, typename FdmT>
__device__ __forceinline__ void fdm_bwd_canon(const FdmT& fdm, const T* src, int is,
                                              Put put) {
  constexpr int M = 2 * K - 1;
  constexpr int I0 = HALF == 0 ? 0 : K / 2, I1 = HALF == 0 ? K / 2 : K;
  T g[M];
#pragma unroll
  for (int c = 0; c < M; ++c) g[c] = src[c * is];
#pragma unroll
  for (int i = I0; i < I1; ++i) {
    T e = T(0);
#pragma unroll
    for (int c = 0; c < K; ++c) e = fma(fdm.S[0][i][c], g[c], e);
    if (i < K - 1) {
      T o = T(0);
#pragma unroll
      for (int c = K; c < M; ++c) o = fma(fdm.S[0][i][c], g[c], o);
      put(i, e + o);
      put(M - 1 - i, e - o);
    } else {
      put(i, e);
    }
  }
}

// all patches of the tile interior: same stages as mvs2_tile.  COEF_DIRECT:
// the coefficients are read from `op` and `fdm` themselves at compile-time
// offsets -- for tables that are kernel parameters, constant-bank operands of
// the FMAs, with no load instruction (FP32: 32 instead of 46 registers at
// k = 4); otherwise they are staged in shared memory first (FP64 kernels,
// whose constant operands the compiler hoists into 104-152 registers, and
// tables in device memory).
template <typename T, int K, bool COEF_DIRECT = false, typename OpT = OpTab<T, K>,
          typename FdmT = FdmTab<T, K>>
__device__ __forceinline__ void mvs2_tile_interior(const OpT& op, const FdmT& fdm,
                                                   const MvsArgs<T>& a, int first, int np,
                                                   unsigned char* smem_raw) {
  using C = Mvs2Cfg<T, K>;
  constexpr int M = C::M, W = C::W, WM = C::WM, MM = M * M;
  constexpr int WS = C::WS;
  const int pb = a.pb;
  T* sX = reinterpret_cast<T*>(smem_raw) + C::TABLES;  // [pb][W][WS]
  T* sTM = sX + pb * C::WIN;
  T* sTL = sTM + pb * W * M;
  T* sTB = sTL + pb * WM * M;
  T* sBv = sTB + pb * WM * M;  // b on the patch nodes (PREFETCH)
  // FP64: R and F over the window once the x-split has read it.  FP32: the
  // window stays intact to the update, which reads x on the patch nodes from
  // it; R takes the space after b, F that of T_M once the y-combination has
  // read it
  T* sR = C::PREFETCH ? sBv + pb * MM : sX;
  T* sF = C::PREFETCH ? sTM : sR + pb * MM;
  __shared__ int sVi[32][2];
  // index in x of window node (0, 0) (negative for patches at v_a = 2), the
  // row offset of window row 0 in shared memory, and whether the window lies in
  // the interior 1..n (then its rows are copied as 16-byte chunks)
  __shared__ long long sW0[32];
  __shared__ int sOff0[32], sDeep[32];
  const int N = a.N, n = a.n;
  // operator and eigenvector tables staged in shared memory (layout of OpTab
  // and FdmTab), read at compile-time offsets (unless COEF_DIRECT), and the
  // interior type's reciprocal eigenvalue sums
  constexpr int NOP = 3 * C::NC * C::BW;
  T* sDinv = reinterpret_cast<T*>(smem_raw) + NOP + 4 * MM;
  {
    T* sT = reinterpret_cast<T*>(smem_raw);
    if constexpr (!COEF_DIRECT) {
      for (int e = threadIdx.x; e < NOP; e += blockDim.x) sT[e] = (&op.M[0][0])[e];
      for (int e = threadIdx.x; e < 4 * MM; e += blockDim.x) sT[NOP + e] = (&fdm.S[0][0][0])[e];
    }
    for (int e = threadIdx.x; e < MM; e += blockDim.x) sDinv[e] = a.dinv[e];  // combination 0
  }
  const auto& op_s = pick_tab<COEF_DIRECT>(op, *reinterpret_cast<const OpTab<T, K>*>(smem_raw));
  const auto& fdm_s = pick_tab<COEF_DIRECT>(
      fdm, *reinterpret_cast<const FdmTab<T, K>*>(smem_raw + sizeof(T) * 3 * C::NC * C::BW));
  // offset in values of a.x from a 16-byte boundary
  const int xo = C::VECWIN ? (int)((reinterpret_cast<uintptr_t>(a.x) / sizeof(T)) & 3) : 0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const int vid = a.verts[first + p];
    const int v0 = vid % (N - 1) + 1, v1 = vid / (N - 1) + 1;
    sVi[p][0] = v0;
    sVi[p][1] = v1;
    const long long w0 = (long long)(K * (v1 - 2) - 1) * n + (K * (v0 - 2) - 1);
    sW0[p] = w0;
    sOff0[p] = (int)((xo + w0) & 3);
    sDeep[p] = (v0 >= 3 && v0 <= N - 3 && v1 >= 3 && v1 <= N - 3) ? 1 : 0;
  }
  __syncthreads();
  // window column 0 of window row wy of patch p in shared memory
  auto win_row = [&](int p, int wy) -> const T* {
    if constexpr (C::VECWIN)
      return sX + (p * W + wy) * WS + ((sOff0[p] + wy * n) & 3);
    else
      return sX + (p * W + wy) * W;
  };
  if constexpr (C::VECWIN) {
    // item (patch, row, chunk); a chunk holds shared positions 4c .. 4c + 3 of
    // the row, i.e. window columns 4c - off .. 4c + 3 - off
    constexpr int CH = C::CH;
    for (int e = threadIdx.x; e < np * W * CH; e += blockDim.x) {
      const int row = e / CH, c = e - row * CH;  // row = p W + wy
      const int p = row / W, wy = row - p * W;
      const long long s = sW0[p] + (long long)wy * n;  // index in x of window node (wy, 0)
      const int off = (sOff0[p] + wy * n) & 3;
      T* dst = sX + row * WS + 4 * c;
      if (sDeep[p]) {
        // a.x + s - off is 16-byte aligned; the chunk lies in 0 .. n^2 - 1
        // because the window lies at least k - 1 nodes inside the interior
        async_copy_chunk16(dst, a.x + (s - off + 4 * c));
      } else {
        const int gy = K * (sVi[p][1] - 2) + wy, gx0 = K * (sVi[p][0] - 2);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int wx = 4 * c + u - off;
          if (wx < 0 || wx >= W) continue;
          const int gx = gx0 + wx;
          const bool in = gx >= 1 && gx <= n && gy >= 1 && gy <= n;
          async_copy_or_zero(dst + u, a.x + (in ? s + wx : 0), in);
        }
      }
    }
  } else {
    for (int e = threadIdx.x; e < np * W * W; e += blockDim.x) {
      const int p = e / (W * W), wy = (e / W) % W, wx = e % W;
      const int gx = K * (sVi[p][0] - 2) + wx, gy = K * (sVi[p][1] - 2) + wy;
      const bool in = gx >= 1 && gx <= n && gy >= 1 && gy <= n;
      // outside the interior the (unread) source is the first value of x
      async_copy_or_zero(sX + e, a.x + (in ? (int64_t)(gy - 1) * n + (gx - 1) : 0), in);
    }
  }
  if constexpr (C::PREFETCH) prefetch_patch_nodes<T, K, false>(a, np, sVi, sBv, nullptr);
  async_copy_wait();
  __syncthreads();
  for (int e = threadIdx.x; e < 2 * np * W; e += blockDim.x) {
    const int q_ = e / (W), wy = e - q_ * (W);  // item (half, patch, wy)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const T* xr = win_row(p, wy) + K;
    T* tm = sTM + (p * W + wy) * M;
    if (half == 0)
      xsplit_m_canon<T, K, 0>(op_s, xr, tm);
    else
      xsplit_m_canon<T, K, 1>(op_s, xr, tm);
  }
  for (int e = threadIdx.x; e < 2 * np * WM; e += blockDim.x) {
    const int q_ = e / (WM), r = e - q_ * (WM);  // item (half, patch, r)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const T* xr = win_row(p, K + r) + K;
    T* tl = sTL + (p * WM + r) * M;
    T* tb = sTB + (p * WM + r) * M;
    if (half == 0)
      xsplit_lb_canon<T, K, 0>(op_s, xr, tl, tb);
    else
      xsplit_lb_canon<T, K, 1>(op_s, xr, tl, tb);
  }
  __syncthreads();
  const T asc = (T)a.ascale;
  for (int e = threadIdx.x; e < 2 * np * M; e += blockDim.x) {
    const int q_ = e / (M), j = e - q_ * (M);  // item (half, patch, j)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const T* cm = sTM + (p * W + K) * M + j;
    const T* cl = sTL + (p * WM) * M + j;
    const T* cb = sTB + (p * WM) * M + j;
    const int g0 = K * (sVi[p][1] - 1);
    const int gx = K * (sVi[p][0] - 1) + j + 1;
    const T* bcol = C::PREFETCH ? sBv + p * MM + j : a.b + (int64_t)g0 * n + (gx - 1);
    const int64_t bs = C::PREFETCH ? M : n;
    T* rcol = sR + p * MM + j;
    if (half == 0)
      ycombine_canon<T, K, 0>(op_s, cm, cl, cb, bcol, bs, asc, rcol);
    else
      ycombine_canon<T, K, 1>(op_s, cm, cl, cb, bcol, bs, asc, rcol);
  }
  __syncthreads();
  // F = R S (rows)
  for (int e = threadIdx.x; e < 2 * np * M; e += blockDim.x) {
    const int q_ = e / (M), i = e - q_ * (M);  // item (half, patch, i)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const T* src = sR + p * MM + i * M;
    T* dst = sF + p * MM + i * M;
    auto put = [&](int c, T v) { dst[c] = v; };
    if (half == 0)
      fdm_fwd_canon<T, K, 0>(fdm_s, src, 1, put);
    else
      fdm_fwd_canon<T, K, 1>(fdm_s, src, 1, put);
  }
  __syncthreads();
  // G = D^-1 S^T F (columns), into sR
  for (int e = threadIdx.x; e < 2 * np * M; e += blockDim.x) {
    const int q_ = e / (M), c0 = e - q_ * (M);  // item (half, patch, c0)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const T* src = sF + p * MM + c0;
    T* dst = sR + p * MM + c0;
    const T* dv = sDinv + c0;  // type combination 0 (interior x interior)
    auto put = [&](int c1, T v) { dst[c1 * M] = v * dv[c1 * M]; };
    if (half == 0)
      fdm_fwd_canon<T, K, 0>(fdm_s, src, M, put);
    else
      fdm_fwd_canon<T, K, 1>(fdm_s, src, M, put);
  }
  __syncthreads();
  // F = S G (columns)
  for (int e = threadIdx.x; e < 2 * np * M; e += blockDim.x) {
    const int q_ = e / (M), c0 = e - q_ * (M);  // item (half, patch, c0)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const T* src = sR + p * MM + c0;
    T* dst = sF + p * MM + c0;
    auto put = [&](int i, T v) { dst[i * M] = v; };
    if (half == 0)
      fdm_bwd_canon<T, K, 0>(fdm_s, src, M, put);
    else
      fdm_bwd_canon<T, K, 1>(fdm_s, src, M, put);
  }
  __syncthreads();
  // x_v += pscale F S^T (rows)
  const T ps = (T)a.pscale;
  for (int e = threadIdx.x; e < 2 * np * M; e += blockDim.x) {
    const int q_ = e / (M), i = e - q_ * (M);  // item (half, patch, i)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const T* src = sF + p * MM + i * M;
    const int gy = K * (sVi[p][1] - 1) + i + 1, gx0 = K * (sVi[p][0] - 1) + 1;
    T* xrow = a.x + (int64_t)(gy - 1) * n + (gx0 - 1);
    const T* xv = win_row(p, K + 1 + i) + K + 1;  // x on the row's patch nodes (PREFETCH)
    auto put = [&](int j, T v) {
      if constexpr (C::PREFETCH)
        xrow[j] = xv[j] + ps * v;
      else
        xrow[j] += ps * v;
    };
    if (half == 0)
      fdm_bwd_canon<T, K, 0>(fdm_s, src, 1, put);
    else
      fdm_bwd_canon<T, K, 1>(fdm_s, src, 1, put);
  }
}

// true on every thread iff all np patches of the tile lie away from the boundary
template <typename T>
__device__ __forceinline__ bool mvs2_tile_is_interior(const MvsArgs<T>& a, int first, int np) {
  int ok = 1;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    const int vid = a.verts[first + p];
    const int v0 = vid % (a.N - 1) + 1, v1 = vid / (a.N - 1) + 1;
    ok &= (v0 >= 2 && v0 <= a.N - 2 && v1 >= 2 && v1 <= a.N - 2) ? 1 : 0;
  }
  return __syncthreads_and(ok) != 0;
}

template <typename T, int K>
__global__ void __launch_bounds__(256) mvs2_color_kernel(const __grid_constant__ MvsTab<T, K> tab,
                                                         const MvsArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int first = blockIdx.x * a.pb;
  const int np = min(a.pb, a.count - first);
  if (np <= 0) return;
  // FP32 interior tiles read the parameter tables as constant operands; the
  // tables staged in shared memory come from the device copy (a parameter
  // read with a different address per thread would be serialized)
  const auto* dt = static_cast<const Tables<T, K>*>(a.dtab);
  if (mvs2_tile_is_interior(a, first, np)) {
    if constexpr (sizeof(T) == 4)
      mvs2_tile_interior<T, K, true>(tab.op, tab.fdm, a, first, np, smem_raw);
    else
      mvs2_tile_interior<T, K>(dt->op, dt->fdm, a, first, np, smem_raw);
  } else {
    mvs2_tile<T, K>(dt->op, dt->fdm, a, first, np, smem_raw);
  }
}

}  // namespace bh
