"""Additive and multiplicative vertex-patch smoothers (Sec. 3).

AVS:  x <- x + omega sum_v R_v^T A_v^{-1} R_v (b - A x)
MVS:  for v in a fixed order:  x <- x + omega R_v^T A_v^{-1} R_v (b - A x)

Reading: the paper prints "x - [...] (b - A x)"; with the residual b - A x
the correction has to be added for the smoother to reduce the error (the
correction solves A e = r), so these functions add it.

The colored MVS of Sec. 3 updates all patches of one color at once.  Patches
of one color are A-orthogonal (R_v A R_w^T = 0), so the colored sweep equals
this sequential sweep over the vertices sorted by color; ``mvs_order``
gives that order (within one color, lexicographic).  The colored and the
atomic AVS of Sec. 5 are two race-free implementations of the same AVS
update, so the oracle has one AVS.

TEST INFRASTRUCTURE ONLY -- see the package docstring.
"""

import numpy as np

from .patches import color, vertices


def avs_step(A, local, b, x, omega, verts=None):
    """One additive vertex-patch step (Sec. 3): one residual, every patch's
    local correction damped by omega and added."""
    if verts is None:
        verts = vertices(local.d, local.N)
    r = b - A @ x
    y = x.copy()
    for v in verts:
        I = local.dofs(v)
        y[I] += omega * local.solve(v, r[I])
    return y


def mvs_order(d, N):
    """The vertex order of the colored MVS: by color, lexicographic inside."""
    vs = vertices(d, N)
    return sorted(vs, key=lambda v: (color(v), v[::-1]))


def mvs_step(A, local, b, x, omega, order=None):
    """Sequential multiplicative sweep with a fresh residual for every patch."""
    if order is None:
        order = mvs_order(local.d, local.N)
    x = x.copy()
    for v in order:
        I = local.dofs(v)
        r_v = b[I] - A[I] @ x
        x[I] += omega * local.solve(v, r_v)
    return x


def mvs_colored_step(A, local, b, x, omega):
    """Colored form: one residual per color, all its patches updated at once.
    Equal to ``mvs_step`` because same-color patches are A-orthogonal."""
    d, N = local.d, local.N
    x = x.copy()
    vs = vertices(d, N)
    for c in range(2 ** (d + 1)):
        r = b - A @ x
        upd = np.zeros_like(x)
        for v in vs:
            if color(v) == c:
                I = local.dofs(v)
                upd[I] += omega * local.solve(v, r[I])
        x += upd
    return x


def smooth(kind, A, local, b, x, omega, steps):
    """`steps` applications of S_l (x, b) with the AVS or MVS of Sec. 3."""
    for _ in range(steps):
        if kind == "avs":
            x = avs_step(A, local, b, x, omega)
        elif kind == "mvs":
            x = mvs_step(A, local, b, x, omega)
        else:
            raise ValueError(kind)
    return x


def default_omega(kind, d, local_solver):
    """Damping from Sec. 5.1: AVS 1/4 in 2D (1/2^d natural, 1/8 exact in 3D)
    and 0.1 in 3D with the inexact solver; MVS 1 in 2D and 0.7 in 3D.

    Reading: the paper does not state omega for the 2D MVS with the inexact
    solver; 1 is used, as for the exact one."""
    if kind == "avs":
        if d == 2:
            return 0.25
        return 0.125 if local_solver == "exact" else 0.1
    return 1.0 if d == 2 else 0.7
