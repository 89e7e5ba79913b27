"""Direct assembly of the C0IP matrix and right-hand side (Sec. 2).

The mesh is the uniform Cartesian mesh of (0, 1)^d with N cells per
direction, h = 1/N.  Global support points are numbered lexicographically
with x fastest: node (g_0, .., g_{d-1}), 0 <= g_a <= kN.  The unknowns are
the interior nodes 1 <= g_a <= kN-1 (V_l is a subspace of H^1_0, Eq.
(fespace); the clamped condition u = 0 is imposed strongly), numbered the
same way with index sum_a (g_a - 1) (kN-1)^a.

``c0ip_matrix`` is Eq. (bfc0ip) written out: a bulk integral of the Hessian
contraction over every cell plus, over every face, the penalty, consistency
and adjoint-consistency integrals with the jump of the normal derivative
(sum of outward normal derivatives of the two sides) and the mean of the
second normal derivative (half the sum of the two sides; one-sided on a
boundary face).  h_e = h (the harmonic mean of the two normal cell extents on
a uniform mesh, Sec. 2).  Integrals use Gauss rules exact for the
polynomial integrands.

Reading: the paper leaves the penalty constant open ("gamma only depends on
k", Sec. 2); the default here is gamma = k(k+1).

TEST INFRASTRUCTURE ONLY -- see the package docstring.
"""

import itertools

import numpy as np
import scipy.sparse as sp

from .basis import basis_table, gauss


def default_gamma(k):
    """Penalty constant gamma(k) = k(k+1) (reading; the paper gives none)."""
    return float(k * (k + 1))


def n_unknowns(d, k, N):
    """Number of unknowns of V_l (Eq. (fespace)): the interior support points,
    k N - 1 per direction, the boundary values being fixed to zero."""
    return (k * N - 1) ** d


def _tensor(tables, axes_first=True):
    """Outer product of per-axis tables T_a[i_a, q_a] -> [(i), (q)] with the
    axis-0 index fastest in both the function and the point index."""
    d = len(tables)
    # einsum over reversed axes so that axis 0 ends up fastest.
    letters_i = "abcd"[:d]
    letters_q = "pqrs"[:d]
    subs = ",".join(letters_i[a] + letters_q[a] for a in range(d))
    out = letters_i[::-1] + letters_q[::-1]
    arr = np.einsum(subs + "->" + out, *tables)
    ni = int(np.prod([t.shape[0] for t in tables]))
    nq = int(np.prod([t.shape[1] for t in tables]))
    return arr.reshape(ni, nq)


def _node_ids(d, k, N, cells):
    """Global node ids (full node grid) of the (k+1)^d local nodes of cells."""
    ng = k * N + 1
    local = np.array(list(itertools.product(range(k + 1), repeat=d)))[:, ::-1]
    # local[:, a] is i_a with i_0 fastest in the local lexicographic order
    g = cells[:, None, :] * k + local[None, :, :]
    strides = ng ** np.arange(d)
    return (g * strides).sum(axis=2)


def cell_matrix(d, k, h, mixed=True):
    """Bulk term int_K Hess(phi_J) : Hess(phi_I) dx on one cell of size h.

    mixed=False keeps only the pure second derivatives d^2/dx_a^2, which is
    the bulk part of the separable local solver of Eq. (localsolverbila)."""
    t, w = gauss(k + 2)
    V = [basis_table(k, t, n) / h ** n for n in range(3)]
    W = _tensor([w[None, :] * h] * d).ravel()
    K = np.zeros(((k + 1) ** d,) * 2)
    for a in range(d):
        for b in range(d):
            if a != b and not mixed:
                continue
            orders = [int(a == c) + int(b == c) for c in range(d)]
            D = _tensor([V[orders[c]] for c in range(d)])
            K += (D * W) @ D.T
    return K


def _face_traces(d, k, h, axis, t_axis):
    """Normal first and second derivative traces of the (k+1)^d cell basis
    functions on the cell face {reference x_axis = t_axis}, at the tensor
    Gauss points of the face, together with the face quadrature weights."""
    t, w = gauss(k + 2)
    V0 = basis_table(k, t, 0)
    d1 = basis_table(k, [t_axis], 1) / h
    d2 = basis_table(k, [t_axis], 2) / h ** 2
    one = np.ones((1, 1))
    J_tabs, M_tabs, W_tabs = [], [], []
    for c in range(d):
        if c == axis:
            J_tabs.append(d1)
            M_tabs.append(d2)
            W_tabs.append(one)
        else:
            J_tabs.append(V0)
            M_tabs.append(V0)
            W_tabs.append(w[None, :] * h)
    return _tensor(J_tabs), _tensor(M_tabs), _tensor(W_tabs).ravel()


def face_matrix(jump, mean, W, gamma, h):
    """int_e gamma/h [[d_n u]][[d_n v]] - {d_nn u}[[d_n v]] - [[d_n u]]{d_nn v}
    for local functions with jump / mean coefficient rows (entry [test, trial])."""
    JW = jump * W
    return (gamma / h) * JW @ jump.T - JW @ mean.T - (mean * W) @ jump.T


def c0ip_matrix(d, k, N, gamma=None, mixed=True):
    """The C0IP matrix A_l of Eq. (bfc0ip) on the interior unknowns (CSR).

    mixed=False assembles the same form without the mixed second-derivative
    bulk terms; its patch restrictions are the inexact local matrices
    A~_v of Eq. (localsolverbila)."""
    if gamma is None:
        gamma = default_gamma(k)
    h = 1.0 / N
    ng = k * N + 1
    rows, cols, vals = [], [], []

    def add(ids_test, ids_trial, mat):
        nc = ids_test.shape[0]
        rows.append(np.repeat(ids_test, ids_trial.shape[1], axis=1).ravel())
        cols.append(np.tile(ids_trial, (1, ids_test.shape[1])).ravel())
        vals.append(np.broadcast_to(mat.ravel(), (nc, mat.size)).ravel())

    all_cells = np.array(list(itertools.product(range(N), repeat=d)))[:, ::-1]
    ids = _node_ids(d, k, N, all_cells)
    add(ids, ids, cell_matrix(d, k, h, mixed))

    for a in range(d):
        # interior faces between cell c (x_a below the face) and c + e_a
        Jm, Mm, W = _face_traces(d, k, h, a, 1.0)
        Jp, Mp, _ = _face_traces(d, k, h, a, 0.0)
        jump = np.vstack([Jm, -Jp])      # outward normals +e_a and -e_a
        mean = np.vstack([0.5 * Mm, 0.5 * Mp])
        F = face_matrix(jump, mean, W, gamma, h)
        lo = all_cells[all_cells[:, a] < N - 1]
        hi = lo.copy()
        hi[:, a] += 1
        fid = np.hstack([_node_ids(d, k, N, lo), _node_ids(d, k, N, hi)])
        add(fid, fid, F)
        # boundary faces: one-sided jump (outward derivative) and mean
        for t_axis, sign, layer in ((0.0, -1.0, 0), (1.0, 1.0, N - 1)):
            Jb, Mb, Wb = _face_traces(d, k, h, a, t_axis)
            Fb = face_matrix(sign * Jb, Mb, Wb, gamma, h)
            bc = all_cells[all_cells[:, a] == layer]
            bid = _node_ids(d, k, N, bc)
            add(bid, bid, Fb)

    n_full = ng ** d
    A = sp.coo_matrix(
        (np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
        shape=(n_full, n_full)).tocsr()
    interior = interior_node_ids(d, k, N)
    return A[interior][:, interior].tocsr()


def interior_node_ids(d, k, N):
    """Full-grid node ids of the unknowns, in unknown order."""
    ng = k * N + 1
    g = np.array(list(itertools.product(range(1, k * N), repeat=d)))[:, ::-1]
    return (g * (ng ** np.arange(d))).sum(axis=1)


# ----------------------------------------------------------------------------
# right-hand side F(v) = int f v (Eq. (bfandrhs))
# ----------------------------------------------------------------------------

def _s(x, n):
    """n-th derivative of s(x) = sin^2(pi x) for n in {0, 2, 4}."""
    if n == 0:
        return np.sin(np.pi * x) ** 2
    if n == 2:
        return 2.0 * np.pi ** 2 * np.cos(2.0 * np.pi * x)
    if n == 4:
        return -8.0 * np.pi ** 4 * np.cos(2.0 * np.pi * x)
    raise ValueError(n)


def manufactured_u(x):
    """u = prod_a sin^2(pi x_a): satisfies u = du/dn = 0 on the boundary.

    x has shape (..., d)."""
    return np.prod(_s(x, 0), axis=-1)


def manufactured_f(x):
    """f = Delta^2 u for u = prod_a sin^2(pi x_a).

    Reading: the model problem is printed as -Delta^2 u = f, but the weak
    form a(u, v) = (f, v) with a(u, v) = int Hess u : Hess v requires
    f = +Delta^2 u; this oracle uses the weak form's sign."""
    d = x.shape[-1]
    s0 = [_s(x[..., a], 0) for a in range(d)]
    s2 = [_s(x[..., a], 2) for a in range(d)]
    s4 = [_s(x[..., a], 4) for a in range(d)]
    f = np.zeros(x.shape[:-1])
    for a in range(d):
        term = s4[a]
        for b in range(d):
            if b != a:
                term = term * s0[b]
        f += term
    for a in range(d):
        for b in range(a + 1, d):
            term = 2.0 * s2[a] * s2[b]
            for c in range(d):
                if c not in (a, b):
                    term = term * s0[c]
            f += term
    return f


def paper_sine_f(x):
    """f = Delta^2 u for u = prod_a sin(pi x_a), the right-hand side of the
    paper's iteration-count experiments (Sec. 5.1): Delta^2 u = d^2 pi^4 u."""
    d = x.shape[-1]
    return (d * np.pi ** 2) ** 2 * np.prod(np.sin(np.pi * x), axis=-1)


def load_vector(d, k, N, f):
    """b_i = int_Omega f phi_i dx for the interior unknowns (Gauss, k+3 points
    per direction on every cell)."""
    h = 1.0 / N
    t, w = gauss(k + 3)
    V0 = basis_table(k, t, 0)
    Phi = _tensor([V0] * d)                       # [(k+1)^d, Q^d]
    W = _tensor([w[None, :] * h] * d).ravel()
    cells = np.array(list(itertools.product(range(N), repeat=d)))[:, ::-1]
    qpts = np.array(list(itertools.product(range(len(t)), repeat=d)))[:, ::-1]
    ref = t[qpts]                                  # [Q^d, d], axis 0 fastest
    X = (cells[:, None, :] + ref[None, :, :]) * h  # [cells, Q^d, d]
    F = f(X)                                       # [cells, Q^d]
    loc = (F * W[None, :]) @ Phi.T                 # [cells, (k+1)^d]
    ids = _node_ids(d, k, N, cells)
    ng = k * N + 1
    full = np.bincount(ids.ravel(), weights=loc.ravel(), minlength=ng ** d)
    return full[interior_node_ids(d, k, N)]
