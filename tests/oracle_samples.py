"""Oracle values of single patches and rows at full size, for parity tests of
the CUDA path at sizes where the oracle cannot run a whole smoothing step:
each value is evaluated from the oracle's global 1D factors (Eq. (c0iptensorvp)
/ Eq. (c0iptensorvp3D)) on the neighbourhood of one patch or row, patch by
patch, with the local solve of Eq. (localsolverbila) by dense LU.  Test
infrastructure (imports the oracle)."""
import itertools

import numpy as np

from oracle import kron
from oracle.patches import color as color_of


def along(P, X, a):
    """Rectangular 1D matrix P applied along method axis a of X (axis 0 = x,
    numpy's last axis)."""
    ax = X.ndim - 1 - a
    return np.moveaxis(np.moveaxis(X, ax, -1) @ P.T, -1, ax)


def factors(d, k, N):
    """The global 1D M, L, B (dense) and the Kronecker terms of A."""
    M1, L1, B1 = (np.asarray(m.todense()) if hasattr(m, "todense") else np.asarray(m)
                  for m in kron.global_1d(k, N))
    terms = ([(1.0, (B1, M1)), (1.0, (M1, B1)), (2.0, (L1, L1))] if d == 2 else
             [(1.0, (B1, M1, M1)), (1.0, (M1, B1, M1)), (1.0, (M1, M1, B1)),
              (2.0, (L1, L1, M1)), (2.0, (M1, L1, L1)), (2.0, (L1, M1, L1))])
    return terms


def color_vertices(d, N, color):
    return [v for v in itertools.product(range(1, N), repeat=d) if color_of(v) == color]


def check_color_on_sampled_patches(d, k, N, color, x, b, got, omega, samples=24, seed=11,
                                   tol=1e-10, exact=False):
    """One color of the colored MVS (Sec. 3) applied to x gave `got`: every node
    outside the color's patches is unchanged bit for bit, and on `samples`
    sampled patches x_v + omega A~_v^-1 R_v (b - A x) matches to `tol`, with
    the separable local matrix A~_v of Eq. (localsolverbila), or with the exact
    A_v = R_v A R_v^T (all terms) when exact is set."""
    n1 = k * N - 1
    terms = factors(d, k, N)
    X0 = x.reshape((n1,) * d)          # numpy axes: slowest first, axis 0 = x is last
    G = got.reshape((n1,) * d)
    covered = np.zeros((n1,) * d, dtype=bool)
    verts = color_vertices(d, N, color)
    for v in verts:
        covered[tuple(slice(k * (v[a] - 1), k * (v[a] + 1) - 1) for a in reversed(range(d)))] = True
    assert np.array_equal(G[~covered], X0[~covered])
    rng = np.random.default_rng(seed)
    for vi in rng.choice(len(verts), min(samples, len(verts)), replace=False):
        v = verts[vi]
        rows = [np.arange(k * (v[a] - 1), k * (v[a] + 1) - 1) for a in range(d)]
        # the band of every patch row stays inside k(v-3) .. k(v+3) (zeros beyond its reach)
        win = [np.arange(max(0, k * (v[a] - 3)), min(n1, k * (v[a] + 3))) for a in range(d)]
        xw = X0[np.ix_(*[win[a] for a in reversed(range(d))])]
        Ax = np.zeros([len(rows[a]) for a in reversed(range(d))])
        At = 0.0
        for c, ops in terms:
            T = xw
            for a, P in enumerate(ops):
                T = along(P[np.ix_(rows[a], win[a])], T, a)
            Ax = Ax + c * T
            if c == 1.0 or exact:   # the separable local matrix drops the mixed terms
                blk = np.ones((1, 1))
                for a in reversed(range(d)):
                    blk = np.kron(blk, ops[a][np.ix_(rows[a], rows[a])])
                At = At + c * blk
        sel = np.ix_(*[rows[a] for a in reversed(range(d))])
        r = (b.reshape((n1,) * d)[sel] - Ax).ravel()
        expect = X0[sel].ravel() + omega * np.linalg.solve(At, r)
        dg, de = G[sel].ravel() - X0[sel].ravel(), expect - X0[sel].ravel()
        assert np.abs(dg - de).max() <= tol * max(np.abs(de).max(), 1e-300), v
