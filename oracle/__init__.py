"""CPU FP64 oracle for the C0 interior-penalty biharmonic multigrid.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA library (``paper_2412_05082_gb300``); the two
meet only through the seeded input generators in ``workload``.

Every function here is the plain definition of what the paper's method
computes, written for a reader who checks it against the paper by eye:

* ``basis``     -- Q_k Lagrange basis on Gauss-Lobatto-Legendre points (Sec. 2).
* ``assemble``  -- the C0IP matrix A_l assembled cell by cell and face by face
                   from the bilinear form Eq. (bfc0ip), the separable variant
                   without mixed second derivatives (Eq. localsolverbila), and
                   the right-hand side F(v) of Eq. (bfandrhs).
* ``kron``      -- global 1D matrices M, L, B and the Kronecker forms
                   Eq. (c0iptensorvp) / Eq. (c0iptensorvp3D) (used as a
                   cross-check of ``assemble`` and as the apply at sizes where
                   the assembled matrix does not fit).
* ``patches``   -- vertex patches, R_v, colors, local matrices (Sec. 3).
* ``smoothers`` -- additive and multiplicative vertex-patch smoothers (Sec. 3).
* ``mg``        -- embedding prolongation, restriction, V-cycle (Algorithm 1).
* ``krylov``    -- right-preconditioned restarted GMRES and nu_frac (Sec. 5.1).
* ``errors``    -- the mesh-dependent energy norm of Eq. (hnorm).

All arithmetic is float64.  Every function is pinned by ``tests/test_oracle_*``
against closed forms, invariants, brute force or the paper's printed values;
the only exception is documented in ``krylov`` (absolute iteration counts
against the paper's tables are a soft comparison, because the paper leaves
the penalty constant, node placement and GMRES restart unstated).
"""

from . import basis, assemble, kron, patches, smoothers, mg, krylov, errors  # noqa: F401
