"""Q_k Lagrange basis on the reference interval [0, 1] (Sec. 2, "standard
Lagrange finite elements ... Q_k").

Reading (the paper does not say where the support points lie): the k+1
support points are the Gauss-Lobatto-Legendre points, the default of the
deal.II FE_Q element the paper's experiments use (Sec. 5).

TEST INFRASTRUCTURE ONLY -- see the package docstring.
"""

import numpy as np
from numpy.polynomial import legendre as _leg


def gll_points(k):
    """The k+1 Gauss-Lobatto-Legendre points mapped to [0, 1], ascending.

    They are the end points plus the roots of P_k', the derivative of the
    Legendre polynomial of degree k."""
    if k < 1:
        raise ValueError("degree must be >= 1")
    dP = _leg.Legendre.basis(k).deriv()
    inner = np.sort(np.real(dP.roots()))
    d2P = dP.deriv()
    for _ in range(3):                       # Newton polish of the roots
        inner = inner - dP(inner) / d2P(inner)
    pts = np.concatenate([[-1.0], inner, [1.0]])
    return (pts + 1.0) / 2.0


def lagrange_derivative(nodes, i, x, deriv):
    """deriv-th derivative (0, 1 or 2) of the Lagrange polynomial
    l_i(x) = prod_{j != i} (x - z_j) / (z_i - z_j), by the product rule
    applied to the product form (no power-basis cancellation)."""
    z = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    others = [j for j in range(len(z)) if j != i]
    fac = {j: (x - z[j]) / (z[i] - z[j]) for j in others}

    def prod_except(skip):
        out = np.ones_like(x)
        for j in others:
            if j not in skip:
                out = out * fac[j]
        return out

    if deriv == 0:
        return prod_except(())
    if deriv == 1:
        return sum(prod_except((m,)) / (z[i] - z[m]) for m in others)
    if deriv == 2:
        total = np.zeros_like(x)
        for m in others:
            for l in others:
                if l != m:
                    total = total + prod_except((m, l)) / ((z[i] - z[m]) * (z[i] - z[l]))
        return total
    raise ValueError("deriv must be 0, 1 or 2")


def basis_table(k, x, deriv=0):
    """Values of the deriv-th derivative of the k+1 Q_k basis functions.

    Returns an array of shape (k+1, len(x)) on the reference interval."""
    z = gll_points(k)
    return np.array([lagrange_derivative(z, i, x, deriv) for i in range(k + 1)])


def gauss(q, a=0.0, b=1.0):
    """q-point Gauss-Legendre rule on [a, b] (exact for degree 2q-1)."""
    t, w = _leg.leggauss(q)
    return a + (b - a) * (t + 1.0) / 2.0, w * (b - a) / 2.0
