"""Global 1D matrices and the Kronecker forms of the C0IP matrix (Sec. 4).

On a Cartesian mesh the C0IP matrix is a sum of Kronecker products of 1D
matrices over the interior nodes of one coordinate line:

    2D  A = B (x) M + 2 L (x) L + M (x) B                  Eq. (c0iptensorvp)
    3D  A = B M M + M B M + M M B + 2 (L L M + M L L + L M L)
                                                           Eq. (c0iptensorvp3D)

with M_ij = int phi_j phi_i, L_ij = int phi_j' phi_i' (Eq. (matrix1d)) and B
the 1D bulk integral of phi_j'' phi_i'' plus the 1D point terms of the face
integrals Eq. (ev) / Eq. (eh).  This module builds the 1D matrices by plain 1D
assembly (cells and face points), independently of ``assemble``; the tests
check that the Kronecker sum equals the directly assembled matrix.

Index convention: arrays hold the unknowns with x fastest, so an operator
acting along x is the LAST factor of scipy's ``kron``.

TEST INFRASTRUCTURE ONLY -- see the package docstring.
"""

import numpy as np
import scipy.sparse as sp

from .assemble import default_gamma
from .basis import basis_table, gauss


def reference_cell_matrices(k):
    """1D cell matrices on [0, 1]: mass, phi'phi' and phi''phi'' integrals."""
    t, w = gauss(k + 2)
    V0, V1, V2 = (basis_table(k, t, n) for n in range(3))
    return (V0 * w) @ V0.T, (V1 * w) @ V1.T, (V2 * w) @ V2.T


def global_1d(k, N, gamma=None, full=False):
    """Global 1D matrices (M, L, B) on a line of N cells of size h = 1/N.

    Returned on the interior nodes 1..kN-1 (dense), or on all nodes 0..kN
    when full=True.  B = sum over cells of the phi'' phi'' integral plus, for
    each face point, gamma/h [[phi']][[phi']] - {phi''}[[phi']] - [[phi']]{phi''}
    with [[.]] the sum of outward derivatives and {.} the mean (one-sided at
    the two boundary points)."""
    if gamma is None:
        gamma = default_gamma(k)
    h = 1.0 / N
    n = k * N + 1
    Mr, Lr, Br = reference_cell_matrices(k)
    M = np.zeros((n, n))
    L = np.zeros((n, n))
    B = np.zeros((n, n))
    for c in range(N):
        sl = slice(k * c, k * c + k + 1)
        M[sl, sl] += h * Mr
        L[sl, sl] += Lr / h
        B[sl, sl] += Br / h ** 3
    d1 = {t: basis_table(k, [t], 1)[:, 0] / h for t in (0.0, 1.0)}
    d2 = {t: basis_table(k, [t], 2)[:, 0] / h ** 2 for t in (0.0, 1.0)}
    for f in range(N + 1):
        ids, jump, mean = [], [], []
        if f > 0:                       # cell f-1 lies on the left: normal +x
            ids.append(np.arange(k * (f - 1), k * f + 1))
            jump.append(d1[1.0])
            mean.append(d2[1.0] * (0.5 if f < N else 1.0))
        if f < N:                       # cell f lies on the right: normal -x
            ids.append(np.arange(k * f, k * f + k + 1))
            jump.append(-d1[0.0])
            mean.append(d2[0.0] * (0.5 if f > 0 else 1.0))
        ids = np.concatenate(ids)
        jump = np.concatenate(jump)
        mean = np.concatenate(mean)
        F = (gamma / h) * np.outer(jump, jump) - np.outer(jump, mean) - np.outer(mean, jump)
        np.add.at(B, (ids[:, None], ids[None, :]), F)
    if full:
        return M, L, B
    s = slice(1, n - 1)
    return M[s, s], L[s, s], B[s, s]


def kron_matrix(d, k, N, gamma=None, mixed=True):
    """Eq. (c0iptensorvp) / Eq. (c0iptensorvp3D) as a sparse matrix.

    mixed=False drops the 2 L (x) L terms: Eq. (localsolverbila)."""
    M, L, B = (sp.csr_matrix(x) for x in global_1d(k, N, gamma))
    K = lambda *f: f[0] if len(f) == 1 else sp.kron(K(*f[:-1]), f[-1], format="csr")
    if d == 2:
        A = K(M, B) + K(B, M)
        if mixed:
            A = A + 2.0 * K(L, L)
    elif d == 3:
        A = K(M, M, B) + K(M, B, M) + K(B, M, M)
        if mixed:
            A = A + 2.0 * (K(M, L, L) + K(L, L, M) + K(L, M, L))
    else:
        raise ValueError(d)
    return A.tocsr()


def apply_along(P, X, axis):
    """Apply the 1D matrix P along one axis of the d-dimensional array X
    (axis 0 = x, the fastest index, which is the LAST numpy axis)."""
    ax = X.ndim - 1 - axis
    Xm = np.moveaxis(X, ax, -1)
    Y = (P @ Xm.reshape(-1, Xm.shape[-1]).T).T.reshape(Xm.shape)
    return np.moveaxis(Y, -1, ax)


class KronOperator:
    """y = A x by the Kronecker form, for sizes where the assembled CSR matrix
    does not fit in host memory.  Each term is a product of 1D sparse
    matrix applications; nothing is fused or reordered beyond that."""

    def __init__(self, d, k, N, gamma=None, mixed=True):
        self.d, self.n = d, k * N - 1
        self.M, self.L, self.B = (sp.csr_matrix(x) for x in global_1d(k, N, gamma))
        if d == 2:
            self.terms = [(1.0, (self.B, self.M)), (1.0, (self.M, self.B))]
            if mixed:
                self.terms.append((2.0, (self.L, self.L)))
        else:
            M, L, B = self.M, self.L, self.B
            self.terms = [(1.0, (B, M, M)), (1.0, (M, B, M)), (1.0, (M, M, B))]
            if mixed:
                self.terms += [(2.0, (L, L, M)), (2.0, (M, L, L)), (2.0, (L, M, L))]
        self.shape = (self.n ** d, self.n ** d)

    def __matmul__(self, x):
        X = np.asarray(x).reshape((self.n,) * self.d)
        Y = np.zeros_like(X)
        for c, ops in self.terms:
            T = X
            for axis, P in enumerate(ops):      # ops[axis] acts along that axis
                T = apply_along(P, T, axis)
            Y += c * T
        return Y.ravel()

    dot = __matmul__
