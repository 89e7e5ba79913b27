"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module holds no arithmetic of the method: it only fixes problem sizes
and draws random numbers.  Both the CPU oracle and the GPU library take the
vectors it produces as inputs, so a parity test compares the two on the same
bits.

Workloads (the paper uses no dataset; these follow the sizes of its
experiments, Sec. 5):

* ``SMALL_2D``  2D Q2 on 8 x 8 cells, manufactured right-hand side.
* ``SWEEP_2D``  2D Q2-Q4 on 512^2 cells and Q5-Q7 on 256^2 cells.
* ``SWEEP_3D``  3D Q2, Q3 on 128^3 cells and Q4-Q7 on 64^3 cells.
* ``batch_problems``   64 independent 2D problems, k ~ U{2..7}, levels with
  1e4 <= (k 2^L + 1)^2 <= 1e6.
* ``serving_requests`` a Poisson-arrival stream of 2D/3D solves.
"""

import numpy as np

# (dim, degree, cells per direction)
SMALL_2D = [(2, 2, 8)]
SWEEP_2D = [(2, 2, 512), (2, 3, 512), (2, 4, 512), (2, 5, 256), (2, 6, 256), (2, 7, 256)]
SWEEP_3D = [(3, 2, 128), (3, 3, 128), (3, 4, 64), (3, 5, 64), (3, 6, 64), (3, 7, 64)]


def level_of(N):
    """Level l of a mesh with N = 2^l cells per direction."""
    L = int(N).bit_length() - 1
    if 2 ** L != N or L < 1:
        raise ValueError("N must be a power of two >= 2")
    return L


def n_unknowns(d, k, N):
    """Interior support points (kN - 1)^d."""
    return (k * N - 1) ** d


def paper_dofs(d, k, N):
    """Support points including the boundary, (kN + 1)^d: the DoF count the
    paper's throughput tables use."""
    return (k * N + 1) ** d


def rhs_uniform(n, seed):
    """i.i.d. uniform[-1, 1] coefficient vector (numpy PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=n)


def vector_uniform(n, seed):
    """A second seeded vector (initial guesses, apply inputs)."""
    return rhs_uniform(n, seed + 7919)


def batch_problems(count=64, seed=1234):
    """(k, L) for the batched form: k ~ U{2..7}, L ~ U over the levels with
    1e4 <= (k 2^L + 1)^2 <= 1e6."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        k = int(rng.integers(2, 8))
        levels = [L for L in range(1, 12) if 1e4 <= (k * 2 ** L + 1) ** 2 <= 1e6]
        L = int(levels[rng.integers(0, len(levels))])
        out.append((2, k, L))
    return out


def serving_requests(count=1000, rate=200.0, seed=2024, max_dofs=2e7):
    """Poisson arrivals (rate per second) of (arrival_s, d, k, L, rhs_seed)
    with d ~ U{2,3}, k ~ U{2..7} and L ~ U over 1e4 <= (k 2^L + 1)^d <= max_dofs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        d = int(rng.integers(2, 4))
        k = int(rng.integers(2, 8))
        levels = [L for L in range(1, 12) if 1e4 <= (k * 2 ** L + 1) ** d <= max_dofs]
        L = int(levels[rng.integers(0, len(levels))])
        out.append((t, d, k, L, seed * 100003 + i))
    return out
