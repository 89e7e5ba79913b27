// Host-side FP64 setup: Q_k basis on Gauss-Lobatto-Legendre points, the 1D
// matrices of Eq. (matrix1d) with the face terms of Eq. (ev)/(eh), their row
// classes, the vertex-patch submatrices, the generalized eigenpairs of the
// fast diagonalization method (Sec. 4.1) and dense SPD inverses for the exact
// local and coarse solvers.
#include "setup.h"

#include "line1d.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <stdexcept>

namespace bh {

std::vector<double> gll_points(int k) {
  std::vector<double> z(k + 1);
  line1d::gll(k, z.data());
  return z;
}

void gauss_rule(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  line1d::gauss(q, x.data(), w.data());
}

double lagrange(const std::vector<double>& z, int i, double x, int deriv) {
  return line1d::lagrange(z.data(), (int)z.size(), i, x, deriv);
}

static void cell_matrices(int k, const std::vector<double>& z, std::vector<double>& M,
                          std::vector<double>& L, std::vector<double>& B) {
  const int n = k + 1;
  M.assign(n * n, 0.0);
  L.assign(n * n, 0.0);
  B.assign(n * n, 0.0);
  line1d::cell_matrices(k, z.data(), M.data(), L.data(), B.data());
}

void global_1d(int k, double gamma, int cells, std::vector<double>& M, std::vector<double>& L,
               std::vector<double>& B) {
  const int n = k * cells + 1;
  M.assign((size_t)n * n, 0.0);
  L.assign((size_t)n * n, 0.0);
  B.assign((size_t)n * n, 0.0);
  line1d::line_matrices(k, gamma, cells, M.data(), L.data(), B.data(), n);
}

static void cholesky_lower(int n, double* A) {
  // A = L L^T, L overwrites the lower triangle (row-major); upper part zeroed.
  for (int j = 0; j < n; ++j) {
    double* rj = A + (size_t)j * n;
    double s = rj[j];
    for (int p = 0; p < j; ++p) s -= rj[p] * rj[p];
    if (!(s > 0.0)) throw std::runtime_error("matrix not positive definite");
    const double ljj = std::sqrt(s);
    rj[j] = ljj;
#pragma omp parallel for schedule(static) if (n > 256)
    for (int i = j + 1; i < n; ++i) {
      double* ri = A + (size_t)i * n;
      double t = ri[j];
      for (int p = 0; p < j; ++p) t -= ri[p] * rj[p];
      ri[j] = t / ljj;
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) A[(size_t)i * n + j] = 0.0;
}

bool spd_inverse(int n, double* A) {
  try {
    cholesky_lower(n, A);
  } catch (...) {
    return false;
  }
  // U = (L^-1)^T, row-major upper triangular: U[i][p] = Linv[p][i]
  std::vector<double> U((size_t)n * n, 0.0);
#pragma omp parallel for schedule(dynamic, 8) if (n > 256)
  for (int j = 0; j < n; ++j) {  // column j of L^-1: forward substitution
    std::vector<double> x(n, 0.0);
    for (int i = j; i < n; ++i) {
      const double* ri = A + (size_t)i * n;
      double t = (i == j) ? 1.0 : 0.0;
      for (int p = j; p < i; ++p) t -= ri[p] * x[p];
      x[i] = t / ri[i];
    }
    for (int i = j; i < n; ++i) U[(size_t)j * n + i] = x[i];
  }
  // A^-1 = L^-T L^-1: (A^-1)_ij = sum_{p >= max(i,j)} U[i][p] U[j][p]
#pragma omp parallel for schedule(dynamic, 8) if (n > 256)
  for (int i = 0; i < n; ++i) {
    const double* ui = U.data() + (size_t)i * n;
    for (int j = i; j < n; ++j) {
      const double* uj = U.data() + (size_t)j * n;
      double s = 0.0;
      for (int p = j; p < n; ++p) s += ui[p] * uj[p];
      A[(size_t)i * n + j] = s;
      A[(size_t)j * n + i] = s;
    }
  }
  return true;
}

bool gen_eig(int n, const double* B, const double* M, double* S, double* lambda) {
  // M = L L^T; C = L^-1 B L^-T; C = Q diag(lambda) Q^T by cyclic Jacobi
  // rotations; S = L^-T Q.
  std::vector<double> Lm(M, M + (size_t)n * n);
  try {
    cholesky_lower(n, Lm.data());
  } catch (...) {
    return false;
  }
  auto Lat = [&](int i, int j) { return Lm[(size_t)i * n + j]; };
  std::vector<double> Y((size_t)n * n), C((size_t)n * n);
  for (int c = 0; c < n; ++c)  // Y = L^-1 B, column by column
    for (int i = 0; i < n; ++i) {
      double t = B[(size_t)i * n + c];
      for (int p = 0; p < i; ++p) t -= Lat(i, p) * Y[(size_t)p * n + c];
      Y[(size_t)i * n + c] = t / Lat(i, i);
    }
  for (int c = 0; c < n; ++c)  // C = L^-1 Y^T
    for (int i = 0; i < n; ++i) {
      double t = Y[(size_t)c * n + i];
      for (int p = 0; p < i; ++p) t -= Lat(i, p) * C[(size_t)p * n + c];
      C[(size_t)i * n + c] = t / Lat(i, i);
    }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double s = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
      C[(size_t)i * n + j] = C[(size_t)j * n + i] = s;
    }
  std::vector<double> Q((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double v = C[(size_t)i * n + j] * C[(size_t)i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = C[(size_t)p * n + q];
        if (apq == 0.0) continue;
        double app = C[(size_t)p * n + p], aqq = C[(size_t)q * n + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < n; ++r) {  // columns p, q
          double crp = C[(size_t)r * n + p], crq = C[(size_t)r * n + q];
          C[(size_t)r * n + p] = c * crp - s * crq;
          C[(size_t)r * n + q] = s * crp + c * crq;
        }
        for (int r = 0; r < n; ++r) {  // rows p, q
          double cpr = C[(size_t)p * n + r], cqr = C[(size_t)q * n + r];
          C[(size_t)p * n + r] = c * cpr - s * cqr;
          C[(size_t)q * n + r] = s * cpr + c * cqr;
        }
        for (int r = 0; r < n; ++r) {
          double qrp = Q[(size_t)r * n + p], qrq = Q[(size_t)r * n + q];
          Q[(size_t)r * n + p] = c * qrp - s * qrq;
          Q[(size_t)r * n + q] = s * qrp + c * qrq;
        }
      }
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return C[(size_t)a * n + a] < C[(size_t)b * n + b]; });
  // S = L^-T Q (back substitution with L^T), columns reordered by eigenvalue
  for (int jj = 0; jj < n; ++jj) {
    const int j = order[jj];
    lambda[jj] = C[(size_t)j * n + j];
    std::vector<double> x(n);
    for (int i = n - 1; i >= 0; --i) {
      double t = Q[(size_t)i * n + j];
      for (int p = i + 1; p < n; ++p) t -= Lat(p, i) * x[p];
      x[i] = t / Lat(i, i);
    }
    for (int i = 0; i < n; ++i) S[(size_t)i * n + jj] = x[i];
  }
  return true;
}

// Generalized eigenpairs of a centrosymmetric pencil (J B J = B, J M J = M with
// J the exchange matrix, m = 2k - 1): the even and odd subspaces decouple, so
// the problem is solved in each (orthonormal bases (e_i +- e_{m-1-i}) / sqrt 2
// and e_{k-1}).  Columns 0..k-1 of S are the even eigenvectors (s_j =
// s_{m-1-j}), columns k..m-1 the odd ones (s_j = -s_{m-1-j}, s_{k-1} = 0),
// both exactly, as the folded FDM transform requires.
bool gen_eig_centro(int m, const double* B, const double* M, double* S, double* lambda) {
  const int k = (m + 1) / 2, ko = k - 1;
  const double r = std::sqrt(0.5);
  // folded basis vectors: even column a (a < k), odd column a (a < k - 1)
  auto qe = [&](int i, int a) -> double {
    if (a == k - 1) return i == k - 1 ? 1.0 : 0.0;
    return (i == a || i == m - 1 - a) ? r : 0.0;
  };
  auto qo = [&](int i, int a) -> double { return i == a ? r : (i == m - 1 - a ? -r : 0.0); };
  auto project = [&](const double* A, int c, bool even, std::vector<double>& out) {
    out.assign((size_t)c * c, 0.0);
    for (int a = 0; a < c; ++a)
      for (int b = 0; b < c; ++b) {
        double t = 0.0;
        for (int i = 0; i < m; ++i)
          for (int j = 0; j < m; ++j)
            t += (even ? qe(i, a) : qo(i, a)) * A[(size_t)i * m + j] * (even ? qe(j, b) : qo(j, b));
        out[(size_t)a * c + b] = t;
      }
  };
  std::vector<double> Me, Be, Mo, Bo, Se((size_t)k * k), So((size_t)ko * ko), le(k), lo(ko);
  project(M, k, true, Me);
  project(B, k, true, Be);
  if (!gen_eig(k, Be.data(), Me.data(), Se.data(), le.data())) return false;
  if (ko > 0) {
    project(M, ko, false, Mo);
    project(B, ko, false, Bo);
    if (!gen_eig(ko, Bo.data(), Mo.data(), So.data(), lo.data())) return false;
  }
  for (int i = 0; i < m; ++i) {
    for (int c = 0; c < k; ++c) {
      double t = 0.0;
      for (int a = 0; a < k; ++a) t += qe(i, a) * Se[(size_t)a * k + c];
      S[(size_t)i * m + c] = t;
    }
    for (int c = 0; c < ko; ++c) {
      double t = 0.0;
      for (int a = 0; a < ko; ++a) t += qo(i, a) * So[(size_t)a * ko + c];
      S[(size_t)i * m + k + c] = t;
    }
  }
  for (int c = 0; c < k; ++c) lambda[c] = le[c];
  for (int c = 0; c < ko; ++c) lambda[k + c] = lo[c];
  return true;
}

void build_setup(int k, double gamma, Setup1D& s) {
  if (k < 2 || k > kMaxK) throw std::runtime_error("degree out of range");
  s.k = k;
  s.gamma = gamma;
  s.z = gll_points(k);
  cell_matrices(k, s.z, s.cellM, s.cellL, s.cellB);
  const int nc = n_classes(k), bw = band(k), m = 2 * k - 1;
  s.tabM.assign(nc * bw, 0.0);
  s.tabL.assign(nc * bw, 0.0);
  s.tabB.assign(nc * bw, 0.0);
  // Reference lines of 7 cells (every canonical row's full band lies inside)
  // and of 2 cells (the single patch touching both faces).
  std::vector<double> M7, L7, B7, M2, L2, B2;
  global_1d(k, gamma, 7, M7, L7, B7);
  global_1d(k, gamma, 2, M2, L2, B2);
  const int n7 = 7 * k + 1, n2 = 2 * k + 1;
  line1d::class_tables(k, M7.data(), L7.data(), B7.data(), n7, M2.data(), L2.data(), B2.data(),
                       n2, s.tabM.data(), s.tabL.data(), s.tabB.data());
  // patch submatrices: nodes (first .. first + m - 1) of the reference line;
  // patch vertices v = 3 (interior), 1 (left), 6 (right) of 7 cells, 1 of 2 cells
  struct Src { const std::vector<double>* M; const std::vector<double>* L; const std::vector<double>* B; int n; int first; };
  const Src src[4] = {{&M7, &L7, &B7, n7, 2 * k + 1}, {&M7, &L7, &B7, n7, 1},
                      {&M7, &L7, &B7, n7, 5 * k + 1}, {&M2, &L2, &B2, n2, 1}};
  for (int t = 0; t < 4; ++t) {
    s.patchM[t].assign(m * m, 0.0);
    s.patchL[t].assign(m * m, 0.0);
    s.patchB[t].assign(m * m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        size_t o = (size_t)(src[t].first + i) * src[t].n + (src[t].first + j);
        s.patchM[t][i * m + j] = (*src[t].M)[o];
        s.patchL[t][i * m + j] = (*src[t].L)[o];
        s.patchB[t][i * m + j] = (*src[t].B)[o];
      }
    s.fdmS[t].assign(m * m, 0.0);
    s.fdmLam[t].assign(m, 0.0);
    // the interior patch pencil is centrosymmetric: even / odd eigenvectors
    const bool ok = t == 0 ? gen_eig_centro(m, s.patchB[t].data(), s.patchM[t].data(),
                                            s.fdmS[t].data(), s.fdmLam[t].data())
                           : gen_eig(m, s.patchB[t].data(), s.patchM[t].data(), s.fdmS[t].data(),
                                     s.fdmLam[t].data());
    if (!ok)
      throw std::runtime_error("generalized eigenproblem failed (B_v not definite: gamma too small?)");
  }
  // prolongation: fine nodes of the two fine cells inside a coarse cell
  s.prolong.assign(2 * k * (k + 1), 0.0);
  for (int r = 0; r < 2 * k; ++r) {
    const double xi = (r < k) ? 0.5 * s.z[r] : 0.5 * (1.0 + s.z[r - k]);
    for (int q = 0; q <= k; ++q) s.prolong[r * (k + 1) + q] = lagrange(s.z, q, xi, 0);
  }
}

void patch_matrix(const Setup1D& s, int d, const int* types, bool mixed, std::vector<double>& A) {
  const int m = 2 * s.k - 1;
  int sz = 1;
  for (int a = 0; a < d; ++a) sz *= m;
  A.assign((size_t)sz * sz, 0.0);
  // terms: (coefficient, operator per axis: 0 = M, 1 = L, 2 = B)
  std::vector<std::pair<double, std::vector<int>>> terms;
  if (d == 2) {
    terms = {{1.0, {2, 0}}, {1.0, {0, 2}}};
    if (mixed) terms.push_back({2.0, {1, 1}});
  } else {
    terms = {{1.0, {2, 0, 0}}, {1.0, {0, 2, 0}}, {1.0, {0, 0, 2}}};
    if (mixed) {
      terms.push_back({2.0, {1, 1, 0}});
      terms.push_back({2.0, {0, 1, 1}});
      terms.push_back({2.0, {1, 0, 1}});
    }
  }
  for (int I = 0; I < sz; ++I) {
    int ii[3] = {I % m, (I / m) % m, I / (m * m)};
    for (int J = 0; J < sz; ++J) {
      int jj[3] = {J % m, (J / m) % m, J / (m * m)};
      double v = 0.0;
      for (auto& t : terms) {
        double p = t.first;
        for (int a = 0; a < d; ++a) {
          const std::vector<double>* P = t.second[a] == 0 ? &s.patchM[types[a]]
                                        : t.second[a] == 1 ? &s.patchL[types[a]]
                                                           : &s.patchB[types[a]];
          p *= (*P)[ii[a] * m + jj[a]];
        }
        v += p;
      }
      A[(size_t)I * sz + J] = v;
    }
  }
}

}  // namespace bh
