"""Mesh-dependent energy norm of Eq. (hnorm) for the discretization error.

|v|_l^2 = sum_K |v|_{H^2(K)}^2 + sum_e gamma/h_e || [[d_n v]] ||_e^2

evaluated for v = u - u_l with the manufactured u = prod_a sin^2(pi x_a).
u is smooth and clamped, so [[d_n u]] = 0 on every face and the face part
is that of u_l alone.  The Proposition of Sec. 2 gives |u - u_l|_l = O(h^{k-1}).

TEST INFRASTRUCTURE ONLY -- see the package docstring.
"""

import itertools

import numpy as np

from .assemble import _face_traces, _node_ids, _tensor, default_gamma, interior_node_ids
from .basis import basis_table, gauss


def _u_hessian(x, a, b):
    """d^2 u / dx_a dx_b for u = prod sin^2(pi x_c); x has shape (..., d)."""
    d = x.shape[-1]
    s0 = np.sin(np.pi * x) ** 2
    s1 = np.pi * np.sin(2.0 * np.pi * x)
    s2 = 2.0 * np.pi ** 2 * np.cos(2.0 * np.pi * x)
    out = np.ones(x.shape[:-1])
    for c in range(d):
        n = int(a == c) + int(b == c)
        out = out * (s0, s1, s2)[n][..., c]
    return out


def energy_error(d, k, N, u_interior, gamma=None):
    """|u - u_l|_l of Eq. (hnorm) for the manufactured u and the discrete
    solution u_l given by its interior coefficients: the broken H^2
    seminorm by Gauss quadrature cell by cell, plus the penalty-weighted
    jumps of the normal derivative of u_l on every face."""
    if gamma is None:
        gamma = default_gamma(k)
    h = 1.0 / N
    ng = k * N + 1
    full = np.zeros(ng ** d)
    full[interior_node_ids(d, k, N)] = u_interior
    cells = np.array(list(itertools.product(range(N), repeat=d)))[:, ::-1]
    coef = full[_node_ids(d, k, N, cells)]               # [cells, (k+1)^d]

    t, w = gauss(k + 3)
    V = [basis_table(k, t, n) / h ** n for n in range(3)]
    W = _tensor([w[None, :] * h] * d).ravel()
    qpts = np.array(list(itertools.product(range(len(t)), repeat=d)))[:, ::-1]
    X = (cells[:, None, :] + t[qpts][None, :, :]) * h
    bulk = 0.0
    for a in range(d):
        for b in range(d):
            orders = [int(a == c) + int(b == c) for c in range(d)]
            D = _tensor([V[orders[c]] for c in range(d)])
            diff = _u_hessian(X, a, b) - coef @ D
            bulk += np.sum(diff ** 2 * W[None, :])

    faces = 0.0
    for a in range(d):
        Jm, _, Wf = _face_traces(d, k, h, a, 1.0)
        Jp, _, _ = _face_traces(d, k, h, a, 0.0)
        lo = cells[cells[:, a] < N - 1]
        hi = lo.copy()
        hi[:, a] += 1
        jm = full[_node_ids(d, k, N, lo)] @ Jm
        jp = full[_node_ids(d, k, N, hi)] @ Jp
        faces += gamma / h * np.sum((jm - jp) ** 2 * Wf[None, :])
        for t_axis, layer in ((0.0, 0), (1.0, N - 1)):
            Jb, _, Wb = _face_traces(d, k, h, a, t_axis)
            bc = cells[cells[:, a] == layer]
            jb = full[_node_ids(d, k, N, bc)] @ Jb
            faces += gamma / h * np.sum(jb ** 2 * Wb[None, :])
    return np.sqrt(bulk + faces)
