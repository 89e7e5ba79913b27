"""Pins for vertex patches, colors, local solvers and smoothers (Sec. 3,
Sec. 4.1)."""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assemble, kron, smoothers
from oracle.patches import LocalSolvers, color, patch_dofs, vertices


def test_patch_count_and_size():
    for d, k, N in [(2, 2, 4), (2, 5, 3), (3, 3, 3)]:
        vs = vertices(d, N)
        assert len(vs) == (N - 1) ** d
        for v in vs:
            I = patch_dofs(d, k, N, v)
            assert len(I) == (2 * k - 1) ** d
            assert len(set(I.tolist())) == len(I)


def test_patches_cover_all_unknowns():
    d, k, N = 2, 3, 4
    cover = np.zeros((k * N - 1) ** d, dtype=int)
    for v in vertices(d, N):
        cover[patch_dofs(d, k, N, v)] += 1
    assert cover.min() >= 1 and cover.max() <= 2 ** d


def test_patch_support_is_inside_patch():
    # R_v^T e_i has support in the 2^d cells at v: the rows of A coupling a
    # patch dof reach at most one cell beyond the patch
    d, k, N = 2, 2, 6
    v = (3, 2)
    I = patch_dofs(d, k, N, v)
    n = k * N - 1
    gx, gy = I % n + 1, I // n + 1
    assert gx.min() == k * (v[0] - 1) + 1 and gx.max() == k * (v[0] + 1) - 1
    assert gy.min() == k * (v[1] - 1) + 1 and gy.max() == k * (v[1] + 1) - 1


@pytest.mark.parametrize("d,N,nc", [(2, 9, 8), (3, 6, 16)])
def test_color_count_and_a_orthogonality(d, N, nc):
    k = 2
    A = assemble.c0ip_matrix(d, k, N).tocsr()
    vs = vertices(d, N)
    assert len({color(v) for v in vs}) == nc
    worst = 0.0
    for v, w in itertools.combinations(vs, 2):
        if color(v) == color(w):
            blk = A[patch_dofs(d, k, N, v)][:, patch_dofs(d, k, N, w)]
            if blk.nnz:
                worst = max(worst, abs(blk).max())
    assert worst == 0.0
    # and the coloring is tight: patches sharing a face-neighbor cell differ
    v, w = (2,) * d, (3,) + (2,) * (d - 1)
    assert color(v) != color(w)
    assert abs(A[patch_dofs(d, k, N, v)][:, patch_dofs(d, k, N, w)]).max() > 0


@pytest.mark.parametrize("d,k,N", [(2, 2, 4), (2, 4, 3), (3, 2, 3), (3, 3, 3)])
def test_inexact_local_matrix_is_separable_fdm(d, k, N):
    """Eq. (localsolverbila) + Eq. (inverse): the patch restriction of the
    form without mixed derivatives is B_v (x) M_v + M_v (x) B_v (3D: three
    terms) with the 1D patch submatrices, and fast diagonalization with the
    generalized eigenpairs B s = lambda M s inverts it exactly."""
    At = assemble.c0ip_matrix(d, k, N, mixed=False)
    M, _, B = kron.global_1d(k, N)
    for v in [(1,) * d, (N - 1,) * d, tuple(range(1, d + 1))]:
        v = tuple(min(max(va, 1), N - 1) for va in v)
        I = patch_dofs(d, k, N, v)
        loc = At[I][:, I].toarray()
        sub = [np.arange(k * (va - 1), k * (va + 1) - 1) for va in v]
        Ms = [M[np.ix_(s, s)] for s in sub]
        Bs = [B[np.ix_(s, s)] for s in sub]
        K = lambda mats: mats[0] if len(mats) == 1 else np.kron(K(mats[:-1]), mats[-1])
        sep = sum(K([Bs[a] if a == c else Ms[a] for a in range(d)][::-1]) for c in range(d))
        assert np.abs(loc - sep).max() <= 1e-12 * np.abs(loc).max()
        # FDM
        Ss, Ls = [], []
        for a in range(d):
            lam, S = sla.eigh(Bs[a], Ms[a])
            assert np.allclose(S.T @ Ms[a] @ S, np.eye(len(lam)), atol=1e-12)
            assert np.all(lam > 0)
            Ss.append(S)
            Ls.append(lam)
        Sk = K(Ss[::-1])
        lam = sum(np.meshgrid(*Ls[::-1], indexing="ij")[d - 1 - a] for a in range(d)).ravel()
        inv = Sk @ np.diag(1.0 / lam) @ Sk.T
        assert np.abs(inv @ loc - np.eye(len(I))).max() < 1e-9


def _dense_operator(fun, n):
    return np.column_stack([fun(e) for e in np.eye(n)])


@pytest.mark.parametrize("d,k,N", [(2, 2, 4), (2, 3, 3), (3, 2, 3)])
def test_avs_exact_error_propagation_spectrum(d, k, N):
    """With exact local solvers sum_v R_v^T A_v^-1 R_v A is a sum of
    A-orthogonal projections P_v; same-color projections are mutually
    orthogonal, so its spectrum lies in (0, n_colors].  With the paper's
    omega = 1/2^d the error propagation I - omega sum P_v is a contraction
    on these meshes (spectrum inside (-1, 1))."""
    A = assemble.c0ip_matrix(d, k, N)
    loc = LocalSolvers(A, d, k, N)
    n = A.shape[0]
    # E e = e - omega sum R^T A_v^-1 R A e  (the smoother applied to b = 0)
    BA = np.eye(n) - _dense_operator(lambda e: smoothers.avs_step(A, loc, np.zeros(n), e, 1.0), n)
    ev = np.linalg.eigvals(BA)
    assert np.abs(ev.imag).max() < 1e-8
    assert ev.real.min() > 1e-6 and ev.real.max() <= 2 ** (d + 1) + 1e-9
    om = 1.0 / 2 ** d
    evE = 1.0 - om * ev.real
    assert evE.min() > -1.0 and evE.max() < 1.0


@pytest.mark.parametrize("d,k,N,ls", [(2, 2, 4, "exact"), (2, 3, 3, "exact"), (2, 2, 4, "inexact"),
                                    (3, 2, 3, "exact")])
def test_mvs_error_propagation_is_a_contraction(d, k, N, ls):
    A = assemble.c0ip_matrix(d, k, N)
    src = A if ls == "exact" else assemble.c0ip_matrix(d, k, N, mixed=False)
    loc = LocalSolvers(src, d, k, N)
    n = A.shape[0]
    E = _dense_operator(lambda e: smoothers.mvs_step(A, loc, np.zeros(n), e, 1.0), n)
    Ah = sla.sqrtm(A.toarray()).real
    normA = np.linalg.norm(Ah @ E @ np.linalg.inv(Ah), 2)
    assert normA < 1.0
    if ls == "exact":
        # an exact multiplicative Schwarz sweep is an A-orthogonal projection product
        assert np.abs(np.linalg.eigvals(E)).max() < 1.0


@pytest.mark.parametrize("d,k,N", [(2, 2, 6), (2, 3, 5), (3, 2, 4)])
def test_colored_mvs_equals_sequential_mvs(d, k, N):
    A = assemble.c0ip_matrix(d, k, N)
    loc = LocalSolvers(assemble.c0ip_matrix(d, k, N, mixed=False), d, k, N)
    rng = np.random.default_rng(3)
    b, x = rng.standard_normal((2, A.shape[0]))
    y1 = smoothers.mvs_step(A, loc, b, x, 0.7)
    y2 = smoothers.mvs_colored_step(A, loc, b, x, 0.7)
    # a different order inside each color gives the same result too
    order = smoothers.mvs_order(d, N)
    shuffled = sorted(order, key=lambda v: (color(v), -hash(v) % 97))
    y3 = smoothers.mvs_step(A, loc, b, x, 0.7, order=shuffled)
    assert np.abs(y1 - y2).max() <= 1e-12 * np.abs(y1).max()
    assert np.abs(y1 - y3).max() <= 1e-12 * np.abs(y1).max()


def test_avs_fixed_point_is_the_solution():
    d, k, N = 2, 3, 4
    A = assemble.c0ip_matrix(d, k, N)
    loc = LocalSolvers(assemble.c0ip_matrix(d, k, N, mixed=False), d, k, N)
    b = np.random.default_rng(4).standard_normal(A.shape[0])
    u = np.linalg.solve(A.toarray(), b)
    assert np.allclose(smoothers.avs_step(A, loc, b, u, 0.25), u, atol=1e-12 * np.abs(u).max())
    assert np.allclose(smoothers.mvs_step(A, loc, b, u, 1.0), u, atol=1e-12 * np.abs(u).max())


def test_single_patch_exact_step_solves():
    # N = 2: one patch; an exact step with omega = 1 is the coarse solve
    for d, k in [(2, 3), (3, 2)]:
        A = assemble.c0ip_matrix(d, k, 2)
        loc = LocalSolvers(A, d, k, 2)
        b = np.random.default_rng(5).standard_normal(A.shape[0])
        x = smoothers.avs_step(A, loc, b, np.zeros_like(b), 1.0)
        assert np.allclose(A @ x, b, atol=1e-10 * np.abs(b).max())


@pytest.mark.parametrize("d,k", [(2, 4), (3, 3)])
def test_patch_matrices_related_by_reflection_and_axis_permutation(d, k):
    """Every exact patch matrix A_v (N = 4: left-boundary, interior and right-
    boundary vertices in each direction) equals a canonical one (no right-
    boundary direction, boundary directions first) with the right-boundary
    axes reversed and the axes permuted: the reflection and permutation
    symmetry of the tensor form, which lets the library invert 4 (3D) instead
    of 27 patch matrices."""
    N, m = 4, 2 * k - 1
    loc = LocalSolvers(assemble.c0ip_matrix(d, k, N), d, k, N)
    mats = {v: loc.matrix(v) for v in itertools.product(range(1, N), repeat=d)}
    kind = {1: "left", 2: "interior", 3: "right"}
    for v, Av in mats.items():
        t = [kind[x] for x in v]
        refl = [ti == "right" for ti in t]
        bnd = [ti != "interior" for ti in t]
        order = sorted(range(d), key=lambda a: not bnd[a])      # boundary axes first
        vc = tuple(1 if bnd[a] else 2 for a in order)           # canonical vertex
        idx = []
        for I in range(m ** d):
            ii = [(I // m ** a) % m for a in range(d)]
            idx.append(sum((m - 1 - ii[order[b]] if refl[order[b]] else ii[order[b]]) * m ** b
                           for b in range(d)))
        idx = np.array(idx)
        G = mats[vc][np.ix_(idx, idx)]
        assert np.abs(G - Av).max() <= 1e-13 * np.abs(Av).max(), v
