"""Pins for the oracle's C0IP matrix (Eq. (bfc0ip)), its Kronecker form
(Eq. (c0iptensorvp), Eq. (c0iptensorvp3D)), the right-hand side and the
energy-error estimate of the Proposition in Sec. 2."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

from oracle import assemble, errors, kron

CASES = [(2, 2, 4), (2, 3, 4), (2, 5, 3), (2, 7, 2), (3, 2, 3), (3, 3, 2), (3, 4, 2)]


@pytest.mark.parametrize("d,k,N", CASES)
def test_direct_assembly_equals_kronecker_form(d, k, N):
    for mixed in (True, False):
        A = assemble.c0ip_matrix(d, k, N, mixed=mixed)
        K = kron.kron_matrix(d, k, N, mixed=mixed)
        assert abs(A - K).max() <= 1e-13 * abs(A).max()


@pytest.mark.parametrize("d,k,N", CASES[:5])
def test_symmetric_positive_definite(d, k, N):
    A = assemble.c0ip_matrix(d, k, N).toarray()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def test_kron_apply_equals_matrix():
    for d, k, N in [(2, 3, 4), (3, 2, 4)]:
        A = assemble.c0ip_matrix(d, k, N)
        x = np.random.default_rng(0).standard_normal(A.shape[0])
        y = kron.KronOperator(d, k, N) @ x
        assert np.linalg.norm(y - A @ x) <= 1e-13 * np.linalg.norm(A @ x)


@pytest.mark.parametrize("d", [2, 3])
def test_h_scaling_of_interior_block(d):
    # A_l scales like h^{d-4}: a patch block away from the boundary matches
    # between N and 2N after scaling (B ~ h^-3, M ~ h, L ~ 1/h per direction).
    from oracle.patches import patch_dofs
    k = 2
    A4 = assemble.c0ip_matrix(d, k, 4)
    A8 = assemble.c0ip_matrix(d, k, 8)
    I4 = patch_dofs(d, k, 4, (2,) * d)
    I8 = patch_dofs(d, k, 8, (4,) * d)
    blk4 = A4[I4][:, I4].toarray()
    blk8 = A8[I8][:, I8].toarray()
    assert np.allclose(blk8, blk4 * 2.0 ** (4 - d), rtol=1e-12, atol=1e-10 * abs(blk8).max())


def test_gamma_enters_only_the_penalty():
    # A(gamma) is affine in gamma: A(3g) - A(2g) = A(2g) - A(g)
    d, k, N = 2, 3, 3
    g = 5.0
    A1, A2, A3 = (assemble.c0ip_matrix(d, k, N, gamma=s * g) for s in (1, 2, 3))
    assert abs((A3 - A2) - (A2 - A1)).max() < 1e-9 * abs(A1).max()


def test_manufactured_f_is_bilaplacian_of_u():
    sympy = pytest.importorskip("sympy")
    for d in (2, 3):
        xs = sympy.symbols("x0:%d" % d)
        u = sympy.Mul(*[sympy.sin(sympy.pi * x) ** 2 for x in xs])
        lap = lambda e: sum(sympy.diff(e, x, 2) for x in xs)
        f = sympy.lambdify(xs, lap(lap(u)), "numpy")
        pts = np.random.default_rng(1).uniform(0, 1, (20, d))
        ref = np.array([f(*p) for p in pts], dtype=float)
        assert np.allclose(assemble.manufactured_f(pts), ref, rtol=1e-12, atol=1e-9)
        us = sympy.lambdify(xs, u, "numpy")
        assert np.allclose(assemble.manufactured_u(pts), [us(*p) for p in pts], atol=1e-14)
    # the paper's sine solution: Delta^2 u = d^2 pi^4 u
    pts = np.random.default_rng(2).uniform(0, 1, (5, 2))
    assert np.allclose(assemble.paper_sine_f(pts),
                       4 * np.pi ** 4 * np.sin(np.pi * pts[:, 0]) * np.sin(np.pi * pts[:, 1]))


def test_load_vector_reproduces_mass_times_interpolant():
    # for f in Q_k, int f phi_i = (M (x) M) f_nodes over all nodes
    d, k, N = 2, 3, 3
    Mf, _, _ = kron.global_1d(k, N, full=True)
    import scipy.sparse as sp
    from oracle.basis import gll_points
    z = gll_points(k)
    x1 = np.concatenate([(c + z[:-1]) / N for c in range(N)] + [[1.0]])
    f = lambda X: (X[..., 0] ** 3 - X[..., 0]) * (2 * X[..., 1] ** 2 + 1)
    X = np.stack(np.meshgrid(x1, x1, indexing="xy"), axis=-1)   # [y, x, 2]
    fn = f(X).ravel()
    full = sp.kron(Mf, Mf) @ fn
    ng = k * N + 1
    inner = assemble.interior_node_ids(d, k, N)
    assert np.allclose(assemble.load_vector(d, k, N, f), full[inner], atol=1e-13)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_energy_error_converges_at_rate_k_minus_1(k):
    errs = []
    for N in (4, 8, 16):
        A = assemble.c0ip_matrix(2, k, N)
        b = assemble.load_vector(2, k, N, assemble.manufactured_f)
        u = spl.spsolve(A.tocsc(), b)
        errs.append(errors.energy_error(2, k, N, u))
    rate = np.log2(errs[1] / errs[2])
    assert k - 1 - 0.15 < rate < k - 1 + 0.4, (errs, rate)


def test_energy_error_converges_3d():
    errs = []
    for N in (2, 4):
        A = assemble.c0ip_matrix(3, 2, N)
        b = assemble.load_vector(3, 2, N, assemble.manufactured_f)
        errs.append(errors.energy_error(3, 2, N, spl.spsolve(A.tocsc(), b)))
    assert errs[1] < errs[0] / 1.6


def test_energy_error_of_exact_interpolant_is_small_and_nonzero():
    # the error functional sees a wrong sign in the jump: perturbing u_h raises it
    d, k, N = 2, 3, 8
    A = assemble.c0ip_matrix(d, k, N)
    b = assemble.load_vector(d, k, N, assemble.manufactured_f)
    u = spl.spsolve(A.tocsc(), b)
    e0 = errors.energy_error(d, k, N, u)
    e1 = errors.energy_error(d, k, N, u * 1.01)
    assert e1 > e0
