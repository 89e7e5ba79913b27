"""Transfers and the multigrid V-cycle (Algorithm 1, Sec. 3).

Levels: level l has N = 2^l cells per direction.  Reading: the coarse mesh
of Sec. 5.1 is the 2^d-cell decomposition of the unit square/cube, so the
coarsest level is l = 1 (N = 2), which holds exactly one vertex patch.

Prolongation (Sec. 3): the matrix of the canonical embedding V_{l-1} -> V_l.
A fine coefficient is the value of the coarse function at the fine support
point; for tensor-product basis functions this is the Kronecker product of
the 1D embedding matrices.  Restriction is its transpose.

Coarse solver (Sec. 5.1 smooths the coarse grid once): reading -- the default
solves the coarse system exactly (dense LU), which equals one exact-local-
solver step with omega = 1 from a zero start because the coarse level is a
single patch; coarse="smooth" applies one step of the level's smoother
instead.

Algorithm 1 with its missing "else": at the coarse level return the coarse
solve; otherwise pre-smooth, restrict b - A x, recurse from zero,
prolongate-add, post-smooth.

TEST INFRASTRUCTURE ONLY -- see the package docstring.
"""

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .assemble import c0ip_matrix, default_gamma
from .basis import basis_table, gll_points
from .patches import LocalSolvers
from .smoothers import default_omega, smooth


def prolongation_1d(k, Nc, full=False):
    """Coarse basis functions (N = Nc) evaluated at the fine support points
    (N = 2 Nc); rows fine nodes, columns coarse nodes."""
    Nf = 2 * Nc
    z = gll_points(k)
    P = np.zeros((k * Nf + 1, k * Nc + 1))
    for cf in range(Nf):
        C = cf // 2
        xi = ((cf - 2 * C) + z) / 2.0           # reference coordinate in C
        vals = basis_table(k, xi, 0)             # [q, i]
        for i in range(k + 1):
            P[k * cf + i, k * C:k * C + k + 1] = vals[:, i]
    if full:
        return P
    return P[1:-1, 1:-1]


def prolongation(d, k, Nc):
    """The embedding V_(l-1) -> V_l on interior unknowns (Sec. 3): the
    Kronecker product of the 1D embedding over the d axes."""
    P1 = sp.csr_matrix(prolongation_1d(k, Nc))
    P = P1
    for _ in range(d - 1):
        P = sp.kron(P1, P, format="csr")
    return P


class Hierarchy:
    """Levels 1..L of one problem: the rediscretized matrices A_l of Eq.
    (bfc0ip), the local solvers of each level, the embeddings, and the
    coarse factorization; vcycle is Algorithm 1."""

    def __init__(self, d, k, L, gamma=None, smoother="mvs", local_solver="inexact",
                 omega=None, pre=1, post=1, coarse="exact", operators=None):
        if gamma is None:
            gamma = default_gamma(k)
        self.d, self.k, self.L = d, k, L
        self.smoother, self.local_solver = smoother, local_solver
        self.omega = default_omega(smoother, d, local_solver) if omega is None else omega
        self.pre, self.post, self.coarse = pre, post, coarse
        self.A, self.local, self.P = {}, {}, {}
        for l in range(1, L + 1):
            N = 2 ** l
            A = c0ip_matrix(d, k, N, gamma) if operators is None else operators[l]
            self.A[l] = A
            src = A if local_solver == "exact" else c0ip_matrix(d, k, N, gamma, mixed=False)
            self.local[l] = LocalSolvers(src, d, k, N)
            if l > 1:
                self.P[l] = prolongation(d, k, 2 ** (l - 1))
        self.coarse_lu = sla.lu_factor(self.A[1].toarray())

    def coarse_solve(self, b):
        """Level 1: the exact solve, or one smoothing step (Sec. 5.1)."""
        if self.coarse == "exact":
            return sla.lu_solve(self.coarse_lu, b)
        return smooth(self.smoother, self.A[1], self.local[1], b, np.zeros_like(b),
                      self.omega, 1)

    def vcycle(self, l, x, b):
        """MG_l(x, b) of Algorithm 1."""
        if l == 1:
            return self.coarse_solve(b)
        A, loc = self.A[l], self.local[l]
        x = smooth(self.smoother, A, loc, b, x, self.omega, self.pre)
        bc = self.P[l].T @ (b - A @ x)
        e = self.vcycle(l - 1, np.zeros_like(bc), bc)
        x = x + self.P[l] @ e
        x = smooth(self.smoother, A, loc, b, x, self.omega, self.post)
        return x

    def preconditioner(self, v):
        """One V-cycle from a zero start on the finest level: z = MG_L(0, v)."""
        return self.vcycle(self.L, np.zeros_like(v), v)
