// One line of the fast-diagonalization transform (Sec. 4.1) along one axis of
// a patch tensor, split in two halves so that two threads share a line.
//
// S is the m x m matrix of generalized eigenvectors of one patch type (S[j][c]:
// component j of eigenvector c, m = 2K-1).  For the interior type the 1D patch
// pencil (B_v, M_v) is centrosymmetric, and the host orders its eigenvectors
// even ones first (columns 0..K-1, s_j = s_{m-1-j}) and odd ones after
// (columns K..m-1, s_j = -s_{m-1-j}, s_{K-1} = 0).  Then only the first K rows
// of S are needed and
//
//   (S^T v)_c = sum_{j<K} S[j][c] a_j,   a_j = v_j + v_{m-1-j}, a_{K-1} = v_{K-1}  (c even)
//   (S^T v)_c = sum_{j<K-1} S[j][c] b_j, b_j = v_j - v_{m-1-j}                     (c odd)
//   (S g)_i = e_i + o_i, (S g)_{m-1-i} = e_i - o_i, (S g)_{K-1} = e_{K-1},
//   e_i = sum_{c<K} S[i][c] g_c, o_i = sum_{c>=K} S[i][c] g_c,
//
// 2K^2 - 1 FP operations per line instead of (2K-1)^2 (the "folded" form).
// Other types take the full product.
#pragma once

namespace bh {

// output modes: store, store scaled by a per-output factor, accumulate scaled
enum { kFdmStore = 0, kFdmScaled = 1, kFdmAdd = 2 };

template <typename T, int MODE>
__device__ __forceinline__ void fdm_put(T* dst, int os, const T* dsc, int ds, T sc, int c, T s) {
  T* o = dst + c * os;
  if (MODE == kFdmStore)
    *o = s;
  else if (MODE == kFdmScaled)
    *o = s * dsc[c * ds];
  else
    *o = fma(sc, s, *o);
}

// FWD: out = S^T in (eigen-coefficients), else out = S in.  in(j) = src[j * is],
// out(c) goes to dst[c * os] per MODE (dsc[c * ds]: per-output factor; sc:
// scale of the accumulation).  HALF 0 / 1 produce complementary outputs.
template <typename T, int K, bool FWD, int HALF, int MODE>
__device__ __forceinline__ void fdm_half(const T* S, bool folded, const T* src, int is, T* dst,
                                         int os, const T* dsc, int ds, T sc) {
  constexpr int M = 2 * K - 1;
  if (FWD) {
    if (folded) {
      if (HALF == 0) {
        T f[K];
#pragma unroll
        for (int j = 0; j < K - 1; ++j) f[j] = src[j * is] + src[(M - 1 - j) * is];
        f[K - 1] = src[(K - 1) * is];
#pragma unroll
        for (int c = 0; c < K; ++c) {
          T s = T(0);
#pragma unroll
          for (int j = 0; j < K; ++j) s = fma(S[j * M + c], f[j], s);
          fdm_put<T, MODE>(dst, os, dsc, ds, sc, c, s);
        }
      } else {
        T f[K - 1];
#pragma unroll
        for (int j = 0; j < K - 1; ++j) f[j] = src[j * is] - src[(M - 1 - j) * is];
#pragma unroll
        for (int c = K; c < M; ++c) {
          T s = T(0);
#pragma unroll
          for (int j = 0; j < K - 1; ++j) s = fma(S[j * M + c], f[j], s);
          fdm_put<T, MODE>(dst, os, dsc, ds, sc, c, s);
        }
      }
    } else {
      T f[M];
#pragma unroll
      for (int j = 0; j < M; ++j) f[j] = src[j * is];
      constexpr int C0 = HALF == 0 ? 0 : K, C1 = HALF == 0 ? K : M;
#pragma unroll
      for (int c = C0; c < C1; ++c) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < M; ++j) s = fma(S[j * M + c], f[j], s);
        fdm_put<T, MODE>(dst, os, dsc, ds, sc, c, s);
      }
    }
  } else {
    T g[M];
#pragma unroll
    for (int c = 0; c < M; ++c) g[c] = src[c * is];
    if (folded) {
      // position pairs (i, m-1-i): half 0 takes i < K/2, half 1 the rest
      constexpr int I0 = HALF == 0 ? 0 : K / 2, I1 = HALF == 0 ? K / 2 : K;
#pragma unroll
      for (int i = I0; i < I1; ++i) {
        T e = T(0);
#pragma unroll
        for (int c = 0; c < K; ++c) e = fma(S[i * M + c], g[c], e);
        if (i < K - 1) {
          T o = T(0);
#pragma unroll
          for (int c = K; c < M; ++c) o = fma(S[i * M + c], g[c], o);
          fdm_put<T, MODE>(dst, os, dsc, ds, sc, i, e + o);
          fdm_put<T, MODE>(dst, os, dsc, ds, sc, M - 1 - i, e - o);
        } else {
          fdm_put<T, MODE>(dst, os, dsc, ds, sc, i, e);
        }
      }
    } else {
      constexpr int I0 = HALF == 0 ? 0 : K, I1 = HALF == 0 ? K : M;
#pragma unroll
      for (int i = I0; i < I1; ++i) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < M; ++c) s = fma(S[i * M + c], g[c], s);
        fdm_put<T, MODE>(dst, os, dsc, ds, sc, i, s);
      }
    }
  }
}

// both halves by one call site: half selected at run time
template <typename T, int K, bool FWD, int MODE>
__device__ __forceinline__ void fdm_line(int half, const T* S, bool folded, const T* src, int is,
                                         T* dst, int os, const T* dsc, int ds, T sc) {
  if (half == 0)
    fdm_half<T, K, FWD, 0, MODE>(S, folded, src, is, dst, os, dsc, ds, sc);
  else
    fdm_half<T, K, FWD, 1, MODE>(S, folded, src, is, dst, os, dsc, ds, sc);
}

}  // namespace bh
