"""Vertex patches, localization R_v, colors and local solvers (Sec. 3).

A vertex patch Omega_v is the union of the 2^d cells at an interior vertex
v = (v_0, .., v_{d-1}), 1 <= v_a <= N-1.  V_v holds the finite element
functions supported in Omega_v: the (2k-1)^d support points strictly inside
the patch, global nodes k(v_a - 1) + 1 .. k(v_a + 1) - 1 in every direction.
R_v selects these unknowns (local order: x fastest).

Colors (Sec. 3 and Fig. 1): patches are split into 2^d non-overlapping groups
by the parity of v, and each group is split again red-black, giving 8 colors
in 2D and 16 in 3D.  Reading (the paper fixes the construction and the
count, not the numbering or the order):

    color(v) = 2 * sum_a (v_a mod 2) 2^a + ((sum_a floor(v_a / 2)) mod 2)

processed in increasing color.

Local solvers: ``exact`` inverts A_v = R_v A R_v^T; ``inexact`` inverts the
restriction of the form without the mixed second derivatives, which is the
separable A~_v of Eq. (localsolverbila).  Both by dense LU.

TEST INFRASTRUCTURE ONLY -- see the package docstring.
"""

import itertools

import numpy as np
import scipy.linalg as sla


def vertices(d, N):
    """Interior vertices, lexicographic with v_0 fastest."""
    return [tuple(v[::-1]) for v in itertools.product(range(1, N), repeat=d)]


def color(v):
    """MVS color of vertex v (Sec. 3, Fig. 1): the parity class of v, split
    red-black by the parity of sum_a floor(v_a / 2) (the numbering is the
    reading in the module docstring)."""
    par = sum((va % 2) << a for a, va in enumerate(v))
    rb = sum(va // 2 for va in v) % 2
    return 2 * par + rb


def n_colors(d):
    """8 colors in 2D, 16 in 3D (Sec. 3)."""
    return 2 ** (d + 1)


def patch_dofs(d, k, N, v):
    """Unknown indices of V_v, local order x fastest."""
    n = k * N - 1
    ranges = [np.arange(k * (va - 1) + 1, k * (va + 1)) - 1 for va in v]
    return _lex(ranges, n)


def _lex(ranges, n):
    """Flat indices of the box ranges[0] x .. x ranges[d-1] (x fastest)."""
    d = len(ranges)
    grids = np.meshgrid(*ranges[::-1], indexing="ij")      # slowest axis first
    idx = np.zeros(grids[0].shape, dtype=np.int64)
    for a in range(d):
        idx += grids[d - 1 - a] * n ** a
    return idx.ravel()


class LocalSolvers:
    """Dense LU factors of the local matrices, one per patch."""

    def __init__(self, A_local_source, d, k, N):
        self.d, self.k, self.N = d, k, N
        self.src = A_local_source.tocsr()
        self._lu = {}

    def dofs(self, v):
        """R_v as an index list (Sec. 3)."""
        return patch_dofs(self.d, self.k, self.N, v)

    def matrix(self, v):
        """The local matrix R_v A R_v^T of the source matrix: A_v (exact) or
        the separable A~_v (Eq. (localsolverbila))."""
        I = self.dofs(v)
        return self.src[I][:, I].toarray()

    def solve(self, v, r):
        """The local solve (local matrix)^-1 r by dense LU, factored once."""
        if v not in self._lu:
            self._lu[v] = sla.lu_factor(self.matrix(v))
        return sla.lu_solve(self._lu[v], r)
