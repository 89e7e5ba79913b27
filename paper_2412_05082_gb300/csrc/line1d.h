// Heap-free core of the host-side 1D setup (Sec. 2 and Sec. 4, Eq. (matrix1d)
// with the face terms of Eq. (ev)/(eh)): the Q_k Lagrange basis on Gauss-
// Lobatto-Legendre points, Gauss quadrature, the reference cell matrices, the
// global 1D matrices M, L, B of a line of unit cells, and their row-class
// tables.  Every routine writes into arrays the caller provides, so both the
// context setup (setup.cpp, std::vector storage) and the allocation-free apply
// (noalloc.cu, static storage) build the 1D data with this one code.
#pragma once
#include <cmath>

namespace bh {
namespace line1d {

constexpr int kMaxDegree = 7;
// nodes of the longest reference line (7 cells of degree 7)
constexpr int kMaxLineNodes = 7 * kMaxDegree + 1;

// Legendre P_n(x) and P_{n-1}(x) by the three-term recurrence.
inline void legendre(int n, double x, double& pn, double& pnm1) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    pn = 1.0;
    pnm1 = 0.0;
    return;
  }
  for (int m = 1; m < n; ++m) {
    const double p2 = ((2.0 * m + 1.0) * x * p1 - m * p0) / (m + 1.0);
    p0 = p1;
    p1 = p2;
  }
  pn = p1;
  pnm1 = p0;
}

// Gauss-Lobatto-Legendre points z[0..k] on [0, 1]: the end points and the
// roots of P_k', found by Newton's method from the Chebyshev-Gauss-Lobatto
// points (P_k' and P_k'' from the Legendre differential equation); ascending.
inline void gll(int k, double* z) {
  z[0] = -1.0;
  z[k] = 1.0;
  for (int j = 1; j < k; ++j) {
    double t = -std::cos(M_PI * j / k);
    for (int it = 0; it < 100; ++it) {
      double pn, pm;
      legendre(k, t, pn, pm);
      const double d1 = k * (t * pn - pm) / (t * t - 1.0);
      const double d2 = (2.0 * t * d1 - k * (k + 1.0) * pn) / (1.0 - t * t);
      const double dt = d1 / d2;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    z[j] = t;
  }
  for (int j = 0; j <= k; ++j) z[j] = 0.5 * (z[j] + 1.0);
  z[0] = 0.0;
  z[k] = 1.0;
}

// Gauss-Legendre rule with q points x[0..q-1], weights w on [0, 1].
inline void gauss(int q, double* x, double* w) {
  for (int j = 0; j < q; ++j) {
    double t = std::cos(M_PI * (j + 0.75) / (q + 0.5)), d1 = 1.0, pn, pm;
    for (int it = 0; it < 100; ++it) {
      legendre(q, t, pn, pm);
      d1 = q * (t * pn - pm) / (t * t - 1.0);
      const double dt = pn / d1;
      t -= dt;
      if (std::fabs(dt) < 1e-17) break;
    }
    legendre(q, t, pn, pm);
    d1 = q * (t * pn - pm) / (t * t - 1.0);
    x[j] = 0.5 * (t + 1.0);
    w[j] = 1.0 / ((1.0 - t * t) * d1 * d1);  // 2/((1-t^2)P'^2), halved for [0,1]
  }
}

// deriv-th derivative (0..2) at x of the Lagrange basis function i on the n
// nodes z: l_i = prod_{j != i} (x - z_j)/(z_i - z_j), derivatives by the
// product rule.
inline double lagrange(const double* z, int n, int i, double x, int deriv) {
  auto fac = [&](int j) { return (x - z[j]) / (z[i] - z[j]); };
  double s = 0.0;
  if (deriv == 0) {
    s = 1.0;
    for (int j = 0; j < n; ++j)
      if (j != i) s *= fac(j);
  } else if (deriv == 1) {
    for (int m = 0; m < n; ++m) {
      if (m == i) continue;
      double p = 1.0 / (z[i] - z[m]);
      for (int j = 0; j < n; ++j)
        if (j != i && j != m) p *= fac(j);
      s += p;
    }
  } else {
    for (int m = 0; m < n; ++m) {
      if (m == i) continue;
      for (int l = 0; l < n; ++l) {
        if (l == i || l == m) continue;
        double p = 1.0 / ((z[i] - z[m]) * (z[i] - z[l]));
        for (int j = 0; j < n; ++j)
          if (j != i && j != m && j != l) p *= fac(j);
        s += p;
      }
    }
  }
  return s;
}

// Reference cell (size 1) mass, stiffness and second-derivative matrices,
// (k+1)^2 row-major: int phi_i phi_j, int phi_i' phi_j', int phi_i'' phi_j''
// by the (k+2)-point Gauss rule (exact for these polynomial integrands).
inline void cell_matrices(int k, const double* z, double* cM, double* cL, double* cB) {
  double x[kMaxDegree + 2], w[kMaxDegree + 2];
  gauss(k + 2, x, w);
  const int n = k + 1;
  for (int e = 0; e < n * n; ++e) cM[e] = cL[e] = cB[e] = 0.0;
  for (int q = 0; q < k + 2; ++q) {
    double v0[kMaxDegree + 1], v1[kMaxDegree + 1], v2[kMaxDegree + 1];
    for (int i = 0; i < n; ++i) {
      v0[i] = lagrange(z, n, i, x[q], 0);
      v1[i] = lagrange(z, n, i, x[q], 1);
      v2[i] = lagrange(z, n, i, x[q], 2);
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        cM[i * n + j] += w[q] * v0[i] * v0[j];
        cL[i * n + j] += w[q] * v1[i] * v1[j];
        cB[i * n + j] += w[q] * v2[i] * v2[j];
      }
  }
}

// Global 1D matrices on a line of `cells` unit cells, nodes 0..k*cells,
// row-major with leading dimension ld (>= k*cells + 1): the assembled cell
// matrices, plus on B the face-point terms of the interior penalty form: at
// every face point, gamma [[u']][[v']] - {u''}[[v']] - [[u']]{v''} with the
// jump [[.]] = sum of the outward derivatives and the mean {.} = half their sum
// (one-sided at the two boundary points).
inline void line_matrices(int k, double gamma, int cells, double* M, double* L, double* B,
                          int ld) {
  double z[kMaxDegree + 1];
  gll(k, z);
  const int c1 = k + 1, n = k * cells + 1;
  double cM[(kMaxDegree + 1) * (kMaxDegree + 1)], cL[(kMaxDegree + 1) * (kMaxDegree + 1)],
      cB[(kMaxDegree + 1) * (kMaxDegree + 1)];
  cell_matrices(k, z, cM, cL, cB);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) M[i * ld + j] = L[i * ld + j] = B[i * ld + j] = 0.0;
  for (int c = 0; c < cells; ++c)
    for (int i = 0; i < c1; ++i)
      for (int j = 0; j < c1; ++j) {
        const int o = (k * c + i) * ld + (k * c + j);
        M[o] += cM[i * c1 + j];
        L[o] += cL[i * c1 + j];
        B[o] += cB[i * c1 + j];
      }
  // derivative traces at the cell end points
  double d1l[kMaxDegree + 1], d1r[kMaxDegree + 1], d2l[kMaxDegree + 1], d2r[kMaxDegree + 1];
  for (int i = 0; i < c1; ++i) {
    d1l[i] = lagrange(z, c1, i, 0.0, 1);
    d1r[i] = lagrange(z, c1, i, 1.0, 1);
    d2l[i] = lagrange(z, c1, i, 0.0, 2);
    d2r[i] = lagrange(z, c1, i, 1.0, 2);
  }
  for (int f = 0; f <= cells; ++f) {
    int ids[2 * kMaxDegree + 2], cnt = 0;
    double J[2 * kMaxDegree + 2], Mu[2 * kMaxDegree + 2];
    const bool interior = f > 0 && f < cells;
    if (f > 0)  // cell f-1 on the left, outward normal +x
      for (int i = 0; i < c1; ++i, ++cnt) {
        ids[cnt] = k * (f - 1) + i;
        J[cnt] = d1r[i];
        Mu[cnt] = d2r[i] * (interior ? 0.5 : 1.0);
      }
    if (f < cells)  // cell f on the right, outward normal -x
      for (int i = 0; i < c1; ++i, ++cnt) {
        ids[cnt] = k * f + i;
        J[cnt] = -d1l[i];
        Mu[cnt] = d2l[i] * (interior ? 0.5 : 1.0);
      }
    for (int a = 0; a < cnt; ++a)
      for (int b = 0; b < cnt; ++b)
        B[ids[a] * ld + ids[b]] += gamma * J[a] * J[b] - J[a] * Mu[b] - Mu[a] * J[b];
  }
}

// Band row t = -2k..2k (row[t + 2k]) of interior row g of a line of `cells`
// cells; columns outside the interior nodes 1..k*cells-1 are zero.
inline void class_row(const double* P, int ld, int k, int cells, int g, double* row) {
  const int last = k * cells - 1;
  for (int t = -2 * k; t <= 2 * k; ++t) {
    const int col = g + t;
    row[t + 2 * k] = (col >= 1 && col <= last) ? P[g * ld + col] : 0.0;
  }
}

// Row-class tables [3k+1][4k+1] of M, L, B (classes: canonical q = g mod k,
// left k + g - 1, right 2k + g - (kN - k), both 3k; see setup.h) from the
// matrices of a 7-cell line (every canonical row's band lies inside; ld7) and
// a 2-cell line (the single vertex touching both faces; ld2).
inline void class_tables(int k, const double* M7, const double* L7, const double* B7, int ld7,
                         const double* M2, const double* L2, const double* B2, int ld2,
                         double* tabM, double* tabL, double* tabB) {
  const int bw = 4 * k + 1;
  auto put = [&](int cls, const double* M, const double* L, const double* B, int ld, int cells,
                 int g) {
    class_row(M, ld, k, cells, g, tabM + cls * bw);
    class_row(L, ld, k, cells, g, tabL + cls * bw);
    class_row(B, ld, k, cells, g, tabB + cls * bw);
  };
  for (int q = 0; q < k; ++q) put(q, M7, L7, B7, ld7, 7, 3 * k + q);          // canonical
  for (int g = 1; g <= k; ++g) put(k + g - 1, M7, L7, B7, ld7, 7, g);          // touch x = 0
  for (int g = 6 * k; g <= 7 * k - 1; ++g) put(2 * k + g - 6 * k, M7, L7, B7, ld7, 7, g);  // x = 1
  put(3 * k, M2, L2, B2, ld2, 2, k);                                           // N = 2
}

}  // namespace line1d
}  // namespace bh
