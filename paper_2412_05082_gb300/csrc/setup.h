// Host-side FP64 setup of the 1D data the kernels use (Sec. 4, Eq. (matrix1d),
// Sec. 4.1).  Everything is computed on cells of size 1 ("reference scale");
// the level scaling is exact and applied by the caller:
//   M ~ h, L ~ 1/h, B ~ 1/h^3  =>  A_l = h^(d-4) A_ref,  A_v^-1 = h^(4-d) A_ref,v^-1.
#pragma once
#include <vector>

namespace bh {

constexpr int kMaxK = 7;

// Row classes of the global 1D matrices on the interior nodes g = 1..kN-1:
//   canonical q = g mod k (rows whose cells do not touch the boundary),
//   left  k + g - 1        for g = 1..k        (touch the face x = 0),
//   right 2k + g - (kN-k)  for g = kN-k..kN-1  (touch the face x = 1),
//   both  3k               for N = 2, g = k    (touch both faces).
// A class row holds the band entries t = -2k..2k of the row (column g + t).
inline int n_classes(int k) { return 3 * k + 1; }
inline int band(int k) { return 4 * k + 1; }

// Patch types per direction of a vertex patch (Sec. 3): 0 interior, 1 touches
// x = 0, 2 touches x = 1, 3 both (the single patch of N = 2).
enum PatchType { kInterior = 0, kLeft = 1, kRight = 2, kBoth = 3 };

struct Setup1D {
  int k = 0;
  double gamma = 0;
  std::vector<double> z;                  // GLL points on [0,1], k+1
  std::vector<double> cellM, cellL, cellB;  // (k+1)^2 reference cell matrices
  // class tables, [n_classes][band], for M, L, B
  std::vector<double> tabM, tabL, tabB;
  // patch submatrices on the m = 2k-1 patch-interior nodes, per type, m*m
  std::vector<double> patchM[4], patchL[4], patchB[4];
  // fast diagonalization per type: S (m*m row-major, column j = eigvec j), lambda (m)
  std::vector<double> fdmS[4], fdmLam[4];
  // prolongation: fine offset r in [0, 2k) inside a coarse cell -> coarse local q in [0, k]
  std::vector<double> prolong;            // [2k][k+1]
};

// Full-node 1D matrices on `cells` cells of size 1 (nodes 0..k*cells), row-major.
void global_1d(int k, double gamma, int cells, std::vector<double>& M, std::vector<double>& L,
               std::vector<double>& B);

void build_setup(int k, double gamma, Setup1D& s);

// GLL points (k+1) on [0,1].
std::vector<double> gll_points(int k);
// Gauss-Legendre rule with q points on [0,1].
void gauss_rule(int q, std::vector<double>& x, std::vector<double>& w);
// deriv-th derivative (0..2) of the Lagrange basis function i on nodes z at x.
double lagrange(const std::vector<double>& z, int i, double x, int deriv);

// Generalized symmetric-definite eigenproblem B s = lambda M s (n x n,
// row-major): S with S^T M S = I, S^T B S = diag(lambda), lambda ascending.
bool gen_eig(int n, const double* B, const double* M, double* S, double* lambda);
// the same for a centrosymmetric pencil, eigenvectors ordered even (columns
// 0..k-1) then odd (k..m-1), m = 2k - 1
bool gen_eig_centro(int m, const double* B, const double* M, double* S, double* lambda);

// In-place inverse of a symmetric positive definite n x n matrix (row-major).
bool spd_inverse(int n, double* A);

// Dense local matrix A_v (exact local solver, Sec. 3) at reference scale for
// the per-direction patch types t[0..d-1]: the Kronecker form restricted to the
// patch, local order x fastest.  mixed=false drops the 2 L(x)L terms.
void patch_matrix(const Setup1D& s, int d, const int* types, bool mixed, std::vector<double>& A);

}  // namespace bh
