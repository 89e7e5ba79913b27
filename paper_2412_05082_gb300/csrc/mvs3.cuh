// Fused kernel of one color of the colored multiplicative vertex-patch smoother
// (Sec. 3) in 3D: for every patch v of the color,
//
//   x_v += omega A~_v^-1 R_v (b - A x)
//
// with the residual computed only on the patch's (2k-1)^3 nodes by sum
// factorization of Eq. (c0iptensorvp3D) and the inverse applied by fast
// diagonalization (Sec. 4.1).  As in 2D, same-color patches are A-orthogonal,
// so the patch residual reads x only in the window of nodes k(v_a - 2) ..
// k(v_a + 2) (W = 4k+1 per axis) and never a value another patch of the color
// writes.  The sweeps only touch the window lines the next sweep needs:
//
//   x-split  T_M = M_x x  on window rows (y, z) of the cross C = {z middle}
//            union {y middle} (middle = the 2k+1 rows k..3k),
//            T_L = L_x x, T_B = B_x x on the middle x middle rows;
//   y-mix    U_B = M_y T_M (all window z), U_M = M_y T_B + B_y T_M + 2 L_y T_L,
//            U_L = 2 (L_y T_M + M_y T_L) (middle z), on the patch (y, x);
//   z        r = b - ascale (M_z U_M + B_z U_B + L_z U_L) on the patch nodes;
//   FDM      S^T along x, y, z, scaling by 1 / (l_x + l_y + l_z), S along z, y, x
//            (folded form of fdm_line.cuh along the axes where the patch is interior).
//
// x is read from global memory (L1/L2) by the x-split; two shared-memory
// regions hold the intermediates and ping-pong through the FDM.
#pragma once
#include "mvs.cuh"

namespace bh {

template <typename T, int K>
struct Mvs3Cfg {
  static constexpr int M = 2 * K - 1, W = 4 * K + 1, WM = 2 * K + 1;
  static constexpr int NC = 3 * K + 1, BW = 4 * K + 1, M3 = M * M * M;
  static constexpr int CROSS = WM * W + 2 * K * WM;  // rows (y, z) of T_M
  static constexpr int TM = CROSS * M, TLB = WM * WM * M;
  static constexpr int UB = W * M * M, UML = WM * M * M;
  static constexpr int RA = (TM + 2 * TLB) > M3 ? (TM + 2 * TLB) : M3;  // region A
  static constexpr int RB = (UB + 2 * UML) > M3 ? (UB + 2 * UML) : M3;  // region B
  static constexpr int PER = RA + RB;
  static constexpr int TABLES = 3 * NC * BW + 4 * M * M;
  static constexpr int BUDGET = 220 * 1024;
  static constexpr int FIT = (BUDGET / (int)sizeof(T) - TABLES) / PER;
  static constexpr int PB_MAX = FIT < 1 ? 1 : (FIT > 16 ? 16 : FIT);
  // threads per block: where one or two blocks per SM hold the large
  // intermediates of a few patches, the block brings more threads to each
  // stage.  Measured on the 3D sweep: FP64 MVS steps 4-9 % faster at
  // k = 3..5 (at k = 6 and 7 the 128 registers that 512 threads leave are too
  // few: spills, 2 % slower at k = 6); FP32 V-cycles 6 % and 17 % faster at
  // k = 3 and 4, 10 % slower at k = 5 (spills)
  static constexpr int THREADS =
      ((sizeof(T) == 4 && (K == 3 || K == 4 || K >= 6)) || (sizeof(T) == 8 && K >= 3 && K <= 5))
          ? 512
          : 256;
  static size_t smem_bytes(int pb) { return sizeof(T) * (size_t)(TABLES + pb * PER) + 64; }
};

// row index of (y, z) in the T_M cross storage, -1 if (y, z) is not in C
template <int K>
__device__ __forceinline__ int cross_row(int y, int z) {
  constexpr int W = 4 * K + 1, WM = 2 * K + 1;
  if (z >= K && z <= 3 * K) return (z - K) * W + y;
  if (y < K || y > 3 * K) return -1;
  const int zo = z < K ? z : z - WM;  // 0 .. 2K-1
  return WM * W + zo * WM + (y - K);
}

// a line of the patch through positions 1..m along one axis, split in halves
// (positions 1..k, k+1..2k-1); out[pos] = sum_t C[q][t] in(pos + t) over the
// band of OP; in(i) = src[(i + OFF) * stride] (OFF maps patch position to
// source row), written to dst[(pos - 1) * dstride] (accumulate if ADD, scaled
// by SC)
template <typename T, int K, int HALF, int OP, int OFF, bool ADD>
__device__ __forceinline__ void line_half(const T* tab, bool canon, int g0, int N, const T* src,
                                          int stride, T* dst, int dstride, T sc) {
  constexpr int BW = 4 * K + 1;
#pragma unroll
  for (int j = Half<K, HALF>::J0; j <= Half<K, HALF>::J1; ++j) {
    const int cls = canon ? j % K : row_class<K>(g0 + j, N);
    T s = T(0);
#pragma unroll
    for (int t = band_lo(OP, j % K, K); t <= band_hi(OP, j % K, K); ++t)
      s = fma(tab[cls * BW + t + 2 * K], src[(j + t + OFF) * stride], s);
    T* o = dst + (j - 1) * dstride;
    *o = ADD ? fma(sc, s, *o) : sc * s;
  }
}

// INTERIOR: every patch of the tile lies away from the boundary in all three
// directions, so the row classes and patch types are compile-time constants
// (coefficients at fixed offsets, folded FDM on every axis)
template <typename T, int K, bool INTERIOR = false>
__device__ __forceinline__ void mvs3_tile(const OpTab<T, K>& op, const FdmTab<T, K>& fdm,
                                          const MvsArgs<T>& a, int first, int np,
                                          unsigned char* smem_raw) {
  using C = Mvs3Cfg<T, K>;
  constexpr int M = C::M, W = C::W, WM = C::WM, NC = C::NC, BW = C::BW, MM = M * M;
  constexpr int M3 = C::M3;
  T* sM = reinterpret_cast<T*>(smem_raw);
  T* sL = sM + NC * BW;
  T* sB = sL + NC * BW;
  T* sS = sB + NC * BW;  // [4][M][M]
  const int pb = a.pb;
  T* regA = sS + 4 * MM;        // [pb][RA]
  T* regB = regA + pb * C::RA;  // [pb][RB]
  __shared__ int sV[16][3], sTy[16][3], sCombo[16];

  if (np <= 0) return;
  const int N = a.N, n = a.n;
  const int64_t n2 = (int64_t)n * n;
  constexpr bool DIRECT = INTERIOR && sizeof(T) == 4;
  if constexpr (!DIRECT) {
    for (int e = threadIdx.x; e < NC * BW; e += blockDim.x) {
      sM[e] = (&op.M[0][0])[e];
      sL[e] = (&op.L[0][0])[e];
      sB[e] = (&op.B[0][0])[e];
    }
    for (int e = threadIdx.x; e < 4 * MM; e += blockDim.x) sS[e] = (&fdm.S[0][0][0])[e];
  }
  const T* tM = DIRECT ? &op.M[0][0] : sM;
  const T* tL = DIRECT ? &op.L[0][0] : sL;
  const T* tB = DIRECT ? &op.B[0][0] : sB;
  const T* tS = DIRECT ? &fdm.S[0][0][0] : sS;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    int vid = a.verts[first + p];
    int combo = 0, mul = 1;
    for (int ax = 0; ax < 3; ++ax) {
      const int v = vid % (N - 1) + 1;
      vid /= (N - 1);
      const int t = (N == 2) ? 3 : (v == 1 ? 1 : (v == N - 1 ? 2 : 0));
      sV[p][ax] = v;
      sTy[p][ax] = t;
      combo += t * mul;
      mul *= 4;
    }
    sCombo[p] = combo;
  }
  __syncthreads();
  const T one = T(1);
  // ---- x-split: T_M on the cross rows, T_L and T_B on the middle rows --------
  // items (half, patch, row); x read from global memory, zero outside 1..n
  for (int e = threadIdx.x; e < 2 * np * C::CROSS; e += blockDim.x) {
    const int q_ = e / (C::CROSS), row = e - q_ * (C::CROSS);  // item (half, patch, row)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    int y, z;
    if (row < WM * W) {
      z = K + row / W;
      y = row % W;
    } else {
      const int r2 = row - WM * W, zo = r2 / WM;
      z = zo < K ? zo : zo + WM;
      y = K + r2 % WM;
    }
    const int gx0 = K * (sV[p][0] - 1);  // global x node of patch position j: gx0 + j
    const int gy = K * (sV[p][1] - 2) + y, gz = K * (sV[p][2] - 2) + z;
    T w[2 * K + 1];  // window columns K..3K = patch positions 0..2K
    const bool inside = gy >= 1 && gy <= n && gz >= 1 && gz <= n;
    const T* xrow = a.x + (int64_t)(gz - 1) * n2 + (int64_t)(gy - 1) * n + (gx0 - 1);
#pragma unroll
    for (int i = 0; i <= 2 * K; ++i) {
      const int gx = gx0 + i;
      w[i] = (inside && gx >= 1 && gx <= n) ? xrow[i] : T(0);
    }
    T* tm = regA + p * C::RA + row * M;
    const bool canon = INTERIOR || sTy[p][0] == 0;
    if (half == 0)
      line_half<T, K, 0, 0, 0, false>(tM, canon, gx0, N, w, 1, tm, 1, one);
    else
      line_half<T, K, 1, 0, 0, false>(tM, canon, gx0, N, w, 1, tm, 1, one);
  }
  for (int e = threadIdx.x; e < 2 * np * WM * WM; e += blockDim.x) {
    const int q_ = e / (WM * WM), r = e - q_ * (WM * WM);  // item (half, patch, r)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const int y = K + r % WM, z = K + r / WM;
    const int gx0 = K * (sV[p][0] - 1);
    const int gy = K * (sV[p][1] - 2) + y, gz = K * (sV[p][2] - 2) + z;
    T w[W];  // window columns 0..4K = patch positions -K..3K
    const bool inside = gy >= 1 && gy <= n && gz >= 1 && gz <= n;
    const T* xrow = a.x + (int64_t)(gz - 1) * n2 + (int64_t)(gy - 1) * n + (gx0 - K - 1);
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const int gx = gx0 - K + i;
      w[i] = (inside && gx >= 1 && gx <= n) ? xrow[i] : T(0);
    }
    T* tl = regA + p * C::RA + C::TM + r * M;
    T* tb = tl + C::TLB;
    const bool canon = INTERIOR || sTy[p][0] == 0;
    if (half == 0) {
      line_half<T, K, 0, 1, K, false>(tL, canon, gx0, N, w, 1, tl, 1, one);
      line_half<T, K, 0, 2, K, false>(tB, canon, gx0, N, w, 1, tb, 1, one);
    } else {
      line_half<T, K, 1, 1, K, false>(tL, canon, gx0, N, w, 1, tl, 1, one);
      line_half<T, K, 1, 2, K, false>(tB, canon, gx0, N, w, 1, tb, 1, one);
    }
  }
  __syncthreads();
  // ---- y-mix: lines along y for a fixed (z, x position j) ---------------------
  // U_B[z][i][j] = (M_y T_M)(i) for every window z (T_M rows y = K..3K)
  for (int e = threadIdx.x; e < 2 * np * W * M; e += blockDim.x) {
    const int q_ = e / (W * M), r = e - q_ * (W * M);  // item (half, patch, r)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const int z = r / M, j = r % M;
    const T* A = regA + p * C::RA;
    // T_M column at (y = K + pos, z): rows of the cross are not evenly spaced in
    // y for the outer z, so gather the 2K+1 values first
    T col[2 * K + 1];
#pragma unroll
    for (int i = 0; i <= 2 * K; ++i) col[i] = A[cross_row<K>(K + i, z) * M + j];
    T* ub = regB + p * C::RB + z * MM + j;  // [z][i][j], i stride M
    const bool canon = INTERIOR || sTy[p][1] == 0;
    const int gy0 = K * (sV[p][1] - 1);
    if (half == 0)
      line_half<T, K, 0, 0, 0, false>(tM, canon, gy0, N, col, 1, ub, M, one);
    else
      line_half<T, K, 1, 0, 0, false>(tM, canon, gy0, N, col, 1, ub, M, one);
  }
  // U_M and U_L on the middle z
  for (int e = threadIdx.x; e < 2 * np * WM * M; e += blockDim.x) {
    const int q_ = e / (WM * M), r = e - q_ * (WM * M);  // item (half, patch, r)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
    const int zr = r / M, j = r % M, z = K + zr;
    const T* A = regA + p * C::RA;
    T cm[W], cl[WM], cb[WM];
#pragma unroll
    for (int y = 0; y < W; ++y) cm[y] = A[((z - K) * W + y) * M + j];  // middle z: full y
#pragma unroll
    for (int y = 0; y < WM; ++y) {
      cl[y] = A[C::TM + (zr * WM + y) * M + j];
      cb[y] = A[C::TM + C::TLB + (zr * WM + y) * M + j];
    }
    T* um = regB + p * C::RB + C::UB + zr * MM + j;
    T* ul = um + C::UML;
    const bool canon = INTERIOR || sTy[p][1] == 0;
    const int gy0 = K * (sV[p][1] - 1);
    const T two = T(2);
    if (half == 0) {
      line_half<T, K, 0, 0, 0, false>(tM, canon, gy0, N, cb, 1, um, M, one);
      line_half<T, K, 0, 2, K, true>(tB, canon, gy0, N, cm, 1, um, M, one);
      line_half<T, K, 0, 1, 0, true>(tL, canon, gy0, N, cl, 1, um, M, two);
      line_half<T, K, 0, 1, K, false>(tL, canon, gy0, N, cm, 1, ul, M, two);
      line_half<T, K, 0, 0, 0, true>(tM, canon, gy0, N, cl, 1, ul, M, two);
    } else {
      line_half<T, K, 1, 0, 0, false>(tM, canon, gy0, N, cb, 1, um, M, one);
      line_half<T, K, 1, 2, K, true>(tB, canon, gy0, N, cm, 1, um, M, one);
      line_half<T, K, 1, 1, 0, true>(tL, canon, gy0, N, cl, 1, um, M, two);
      line_half<T, K, 1, 1, K, false>(tL, canon, gy0, N, cm, 1, ul, M, two);
      line_half<T, K, 1, 0, 0, true>(tM, canon, gy0, N, cl, 1, ul, M, two);
    }
  }
  __syncthreads();
  // ---- z-combination and residual on the patch nodes (region A) ---------------
  const T asc = (T)a.ascale;
  for (int e = threadIdx.x; e < 2 * np * MM; e += blockDim.x) {
    const int q_ = e / (MM), r = e - q_ * (MM);  // item (half, patch, r)
    const int half = q_ >= np ? 1 : 0, p = q_ - half * np;  // r = i (y) * M + j (x)
    const T* Bp = regB + p * C::RB;
    T cub[W], cum[WM], cul[WM];
#pragma unroll
    for (int z = 0; z < W; ++z) cub[z] = Bp[z * MM + r];
#pragma unroll
    for (int z = 0; z < WM; ++z) {
      cum[z] = Bp[C::UB + z * MM + r];
      cul[z] = Bp[C::UB + C::UML + z * MM + r];
    }
    T* R = regA + p * C::RA + r;  // R[kz][i][j], kz stride MM
    const bool canon = INTERIOR || sTy[p][2] == 0;
    const int gz0 = K * (sV[p][2] - 1);
    if (half == 0) {
      line_half<T, K, 0, 0, 0, false>(tM, canon, gz0, N, cum, 1, R, MM, one);
      line_half<T, K, 0, 2, K, true>(tB, canon, gz0, N, cub, 1, R, MM, one);
      line_half<T, K, 0, 1, 0, true>(tL, canon, gz0, N, cul, 1, R, MM, one);
    } else {
      line_half<T, K, 1, 0, 0, false>(tM, canon, gz0, N, cum, 1, R, MM, one);
      line_half<T, K, 1, 2, K, true>(tB, canon, gz0, N, cub, 1, R, MM, one);
      line_half<T, K, 1, 1, 0, true>(tL, canon, gz0, N, cul, 1, R, MM, one);
    }
    // r = b - ascale * (A x) on this column's patch nodes of the half
    const int i = r / M, j = r % M;
    const int gx = K * (sV[p][0] - 1) + j + 1, gy = K * (sV[p][1] - 1) + i + 1;
    const int z0 = half == 0 ? 1 : K + 1, z1 = half == 0 ? K : M;
    for (int kz = z0; kz <= z1; ++kz) {
      const int gz = gz0 + kz;
      T* rp = R + (kz - 1) * MM;
      *rp = a.b[(int64_t)(gz - 1) * n2 + (int64_t)(gy - 1) * n + (gx - 1)] - asc * *rp;
    }
  }
  __syncthreads();
  // ---- fast diagonalization (region A <-> region B, M^3 values each) ---------
  // stage s along axis x, y, z (S^T; the third scaled by 1 / (l_x + l_y + l_z)),
  // then z, y, x (S; the last adds pscale * result to x); k >= 3: one half-line
  // per item, folded along the axes where the patch is interior
  if constexpr (K == 2) {
    // m = 3: folding saves little, one output per item keeps more threads busy
    for (int stage = 0; stage < 6; ++stage) {
      const int ax = stage < 3 ? stage : 5 - stage;  // x, y, z, then z, y, x
      const bool trans = stage < 3;
      const int st = ax == 0 ? 1 : (ax == 1 ? M : MM);
      const T* in = (stage % 2 == 0) ? regA : regB;
      T* outp = (stage % 2 == 0) ? regB : regA;
      const int istride = (stage % 2 == 0) ? C::RA : C::RB;
      const int ostride = (stage % 2 == 0) ? C::RB : C::RA;
      for (int e = threadIdx.x; e < np * M3; e += blockDim.x) {
        const int p = e / M3, l = e % M3;
        const int c_ax = (l / st) % M, l0 = l - c_ax * st;
        const T* S = tS + sTy[p][ax] * MM;
        const T* src = in + p * istride + l0;
        T s = T(0);
#pragma unroll
        for (int c = 0; c < M; ++c)
          s = fma(trans ? S[c * M + c_ax] : S[c_ax * M + c], src[c * st], s);
        if (stage == 2) s *= a.dinv[(int64_t)sCombo[p] * M3 + l];
        if (stage < 5) {
          outp[p * ostride + l] = s;
        } else {
          const int j = l % M, i = (l / M) % M, kz = l / MM;
          const int gx = K * (sV[p][0] - 1) + j + 1, gy = K * (sV[p][1] - 1) + i + 1,
                    gz = K * (sV[p][2] - 1) + kz + 1;
          a.x[(int64_t)(gz - 1) * n2 + (int64_t)(gy - 1) * n + (gx - 1)] += (T)a.pscale * s;
        }
      }
      __syncthreads();
    }
  } else {
    const T ps = (T)a.pscale;
    for (int stage = 0; stage < 6; ++stage) {
      const int ax = stage < 3 ? stage : 5 - stage;  // x, y, z, then z, y, x
      const int st = ax == 0 ? 1 : (ax == 1 ? M : MM);
      const T* in = (stage % 2 == 0) ? regA : regB;
      T* outp = (stage % 2 == 0) ? regB : regA;
      const int istride = (stage % 2 == 0) ? C::RA : C::RB;
      const int ostride = (stage % 2 == 0) ? C::RB : C::RA;
      for (int e = threadIdx.x; e < 2 * np * MM; e += blockDim.x) {
        const int q_ = e / (MM), q = e - q_ * (MM);  // item (half, patch, q)
        const int half = q_ >= np ? 1 : 0, p = q_ - half * np;
        // first element of line q (the two other coordinates) in [z][y][x] order
        const int l0 = ax == 0 ? q * M : (ax == 1 ? (q / M) * MM + q % M : q);
        const int t = INTERIOR ? 0 : sTy[p][ax];
        const T* S = tS + t * MM;
        const T* src = in + p * istride + l0;
        T* dst = outp + p * ostride + l0;
        if (stage == 2) {
          fdm_line<T, K, true, kFdmScaled>(half, S, t == 0, src, st, dst, st,
                                           a.dinv + (int64_t)sCombo[p] * M3 + l0, st, T(0));
        } else if (stage < 3) {
          fdm_line<T, K, true, kFdmStore>(half, S, t == 0, src, st, dst, st, nullptr, 0, T(0));
        } else if (stage < 5) {
          fdm_line<T, K, false, kFdmStore>(half, S, t == 0, src, st, dst, st, nullptr, 0, T(0));
        } else {  // x lines: q = kz M + i
          const int i = q % M, kz = q / M;
          const int gy = K * (sV[p][1] - 1) + i + 1, gz = K * (sV[p][2] - 1) + kz + 1;
          T* xrow = a.x + (int64_t)(gz - 1) * n2 + (int64_t)(gy - 1) * n + K * (sV[p][0] - 1);
          fdm_line<T, K, false, kFdmAdd>(half, S, t == 0, src, 1, xrow, 1, nullptr, 0, ps);
        }
      }
      __syncthreads();
    }
  }
}

// true on every thread iff all np patches of the tile lie away from the boundary
template <typename T>
__device__ __forceinline__ bool mvs3_tile_is_interior(const MvsArgs<T>& a, int first, int np) {
  int ok = 1;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    int vid = a.verts[first + p];
    for (int ax = 0; ax < 3; ++ax) {
      const int v = vid % (a.N - 1) + 1;
      vid /= (a.N - 1);
      ok &= (v >= 2 && v <= a.N - 2) ? 1 : 0;
    }
  }
  return __syncthreads_and(ok) != 0;
}

template <typename T, int K>
__global__ void __launch_bounds__(Mvs3Cfg<T, K>::THREADS)
    mvs3_color_kernel(const __grid_constant__ MvsTab<T, K> tab, const MvsArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int first = blockIdx.x * a.pb;
  const int np = min(a.pb, a.count - first);
  if (np <= 0) return;
  // FP32 interior tiles read the parameter tables as constant operands; the
  // tables staged in shared memory come from the device copy
  const auto* dt = static_cast<const Tables<T, K>*>(a.dtab);
  if (mvs3_tile_is_interior(a, first, np)) {
    if constexpr (sizeof(T) == 4)
      mvs3_tile<T, K, true>(tab.op, tab.fdm, a, first, np, smem_raw);
    else
      mvs3_tile<T, K, true>(dt->op, dt->fdm, a, first, np, smem_raw);
  } else {
    mvs3_tile<T, K, false>(dt->op, dt->fdm, a, first, np, smem_raw);
  }
}

}  // namespace bh
