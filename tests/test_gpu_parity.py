"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on
the same seeded inputs.  Tolerances (relative, infinity norm, from the
arithmetic: FP64 sums of O(100) terms each carry ~1e-15 relative rounding):
apply_A and transfers 1e-12, one smoothing step and one V-cycle 1e-10, solves
reach the same 1e-8 relative residual with iteration counts within +-1."""
import functools

import numpy as np
import scipy.sparse as sp
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle_samples  # noqa: E402
import workload  # noqa: E402
from oracle import assemble, kron, krylov, mg, smoothers  # noqa: E402
from oracle.patches import LocalSolvers  # noqa: E402


@pytest.fixture(scope="module")
def bh():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: the -m gpu tests need a GB300")
    import paper_2412_05082_gb300 as m
    m.load()
    return m


def cuda(v):
    return torch.tensor(np.asarray(v), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@functools.lru_cache(maxsize=None)
def oracle_A(d, k, N, mixed=True):
    return assemble.c0ip_matrix(d, k, N, mixed=mixed)


@functools.lru_cache(maxsize=None)
def oracle_local(d, k, N, ls):
    src = oracle_A(d, k, N) if ls == "exact" else oracle_A(d, k, N, False)
    return LocalSolvers(src, d, k, N)


def make_ctx(bh, d, k, L, **kw):
    return bh.Context(bh.default_params(d, k, L, **kw))


APPLY_CASES = [(2, k, N) for k in range(2, 8) for N in (2, 4, 8)] + \
    [(2, 3, 32), (2, 2, 64), (3, 2, 2), (3, 2, 4), (3, 2, 8), (3, 3, 4), (3, 4, 4), (3, 5, 2),
     (3, 7, 2)]


@pytest.mark.parametrize("d,k,N", APPLY_CASES)
def test_apply_A(bh, d, k, N):
    L = workload.level_of(N)
    with make_ctx(bh, d, k, L) as ctx:
        n = ctx.num_unknowns(L)
        x = workload.vector_uniform(n, seed=10 + k)
        X, Y = cuda(x), torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.apply_A(L, X, Y)
        ref = oracle_A(d, k, N) @ x
        assert relerr(host(Y), ref) <= 1e-12
        # residual mode
        b = workload.rhs_uniform(n, seed=3)
        R = torch.empty_like(X)
        ctx.residual(L, X, cuda(b), R)
        assert relerr(host(R), b - ref) <= 1e-12


def test_apply_A_every_level_of_a_hierarchy(bh):
    d, k, L = 2, 3, 5
    with make_ctx(bh, d, k, L) as ctx:
        for l in range(1, L + 1):
            n = ctx.num_unknowns(l)
            x = workload.vector_uniform(n, seed=l)
            Y = torch.empty(n, dtype=torch.float64, device="cuda")
            ctx.apply_A(l, cuda(x), Y)
            assert relerr(host(Y), oracle_A(d, k, 2 ** l) @ x) <= 1e-12


@pytest.mark.parametrize("d,k,N", [(2, 2, 8), (2, 3, 4), (2, 7, 4), (3, 2, 4), (3, 3, 4)])
def test_transfers(bh, d, k, N):
    L = workload.level_of(N)
    P = mg.prolongation(d, k, N // 2)
    with make_ctx(bh, d, k, L) as ctx:
        nf, nc = ctx.num_unknowns(L), ctx.num_unknowns(L - 1)
        xc = workload.vector_uniform(nc, 1)
        xf = workload.vector_uniform(nf, 2)
        XF = cuda(xf)
        ctx.prolongate_add(L, cuda(xc), XF)
        assert relerr(host(XF), xf + P @ xc) <= 1e-12
        BC = torch.empty(nc, dtype=torch.float64, device="cuda")
        ctx.restrict(L, cuda(xf), BC)
        assert relerr(host(BC), P.T @ xf) <= 1e-12


SMOOTH_CASES = [
    (2, 2, 8, "avs", "inexact"), (2, 3, 8, "avs", "inexact"), (2, 5, 4, "avs", "inexact"),
    (2, 7, 4, "avs", "inexact"), (2, 2, 16, "mvs", "inexact"), (2, 4, 8, "mvs", "inexact"),
    (2, 6, 4, "mvs", "inexact"), (2, 3, 8, "mvs", "exact"), (2, 4, 4, "avs", "exact"),
    (3, 2, 4, "avs", "inexact"), (3, 2, 8, "mvs", "inexact"), (3, 3, 4, "mvs", "inexact"),
    (3, 2, 4, "mvs", "exact"), (2, 3, 2, "mvs", "inexact"), (3, 4, 2, "avs", "inexact"),
    (3, 4, 4, "mvs", "inexact"), (3, 5, 4, "mvs", "inexact"), (3, 7, 2, "mvs", "inexact"),
    (3, 6, 2, "mvs", "inexact"), (3, 3, 8, "mvs", "inexact"),
    (2, 3, 16, "mvs", "inexact"), (2, 5, 8, "mvs", "inexact"), (2, 7, 8, "mvs", "inexact"),
    # exact local solvers: per-patch products (3D k = 4) and, for patches of
    # m^3 >= 512 unknowns, one dense product per run of a type combination
    # (the library's own FP64 tensor-core GEMM, gemm.cu)
    (3, 4, 4, "mvs", "exact"), (3, 5, 4, "avs", "exact"), (3, 5, 2, "mvs", "exact"),
    (3, 5, 4, "mvs", "exact"), (3, 6, 2, "mvs", "exact"), (3, 6, 4, "mvs", "exact"),
    (3, 7, 2, "mvs", "exact"),
]


@pytest.mark.parametrize("d,k,N,kind,ls", SMOOTH_CASES)
def test_one_smoothing_step(bh, d, k, N, kind, ls):
    L = workload.level_of(N)
    A = oracle_A(d, k, N)
    loc = oracle_local(d, k, N, ls)
    omega = smoothers.default_omega(kind, d, ls)
    n = A.shape[0]
    b = workload.rhs_uniform(n, seed=5)
    x = workload.vector_uniform(n, seed=6)
    ref = smoothers.smooth(kind, A, loc, b, x, omega, 1)
    variants = [bh.MVS_COLORED] if kind == "mvs" else [bh.AVS_ATOMIC, bh.AVS_COLORED]
    for sm in variants:
        with make_ctx(bh, d, k, L, smoother=sm, local_solver=bh.EXACT if ls == "exact" else bh.FDM) as ctx:
            X = cuda(x)
            ctx.smooth(L, X, cuda(b), 1)
            assert relerr(host(X) - x, ref - x) <= 1e-10, sm


@pytest.mark.parametrize("k,tile", [(2, 5), (4, 1), (4, 7), (4, 12), (6, 3)])
def test_mvs_step_for_every_tile_shape(bh, k, tile):
    """One colored MVS step with a given number of patches per thread block:
    tiles of interior patches take the folded, compile-time-coefficient path,
    tiles touching the boundary the general one, and a ragged last tile mixes
    both kinds of patch."""
    d, N = 2, 16
    L = workload.level_of(N)
    A = oracle_A(d, k, N)
    loc = oracle_local(d, k, N, "inexact")
    n = A.shape[0]
    b = workload.rhs_uniform(n, seed=8)
    x = workload.vector_uniform(n, seed=9)
    ref = smoothers.smooth("mvs", A, loc, b, x, 1.0, 1)
    with make_ctx(bh, d, k, L) as ctx:
        ctx.set_tile(tile)
        X = cuda(x)
        ctx.smooth(L, X, cuda(b), 1)
        assert relerr(host(X) - x, ref - x) <= 1e-10


def test_colored_avs_is_deterministic_and_equals_atomic(bh):
    d, k, L = 2, 3, 4
    n = (k * 2 ** L - 1) ** d
    b, x = workload.rhs_uniform(n, 1), workload.vector_uniform(n, 2)
    outs = []
    for sm in (bh.AVS_COLORED, bh.AVS_COLORED, bh.AVS_ATOMIC):
        with make_ctx(bh, d, k, L, smoother=sm) as ctx:
            X = cuda(x)
            ctx.smooth(L, X, cuda(b), 2)
            outs.append(host(X))
    assert np.array_equal(outs[0], outs[1])
    assert relerr(outs[2], outs[0]) <= 1e-13


@pytest.mark.parametrize("d,k,L,kind,ls", [(2, 2, 3, "mvs", "inexact"), (2, 3, 3, "avs", "inexact"),
                                          (2, 4, 2, "mvs", "exact"), (3, 2, 3, "mvs", "inexact")])
def test_one_vcycle(bh, d, k, L, kind, ls):
    steps = 2 if kind == "avs" else 1
    H = mg.Hierarchy(d, k, L, smoother=kind, local_solver=ls, pre=steps, post=steps)
    n = H.A[L].shape[0]
    b = workload.rhs_uniform(n, 11)
    x = workload.vector_uniform(n, 12)
    ref = H.vcycle(L, x.copy(), b)
    sm = bh.MVS_COLORED if kind == "mvs" else bh.AVS_ATOMIC
    with make_ctx(bh, d, k, L, smoother=sm, pre_steps=steps, post_steps=steps,
                  local_solver=bh.EXACT if ls == "exact" else bh.FDM) as ctx:
        X = cuda(x)
        ctx.vcycle(L, X, cuda(b))
        assert relerr(host(X), ref) <= 1e-10


@pytest.mark.parametrize("d,k,L,side", [(2, 2, 4, "right"), (2, 3, 4, "right"), (2, 5, 3, "right"),
                                        (2, 3, 4, "left"), (3, 2, 3, "right"), (3, 3, 2, "left")])
def test_solve_matches_oracle(bh, d, k, L, side):
    H = mg.Hierarchy(d, k, L)
    b = assemble.load_vector(d, k, 2 ** L, assemble.manufactured_f)
    xr, it_ref, hist, rr_ref = krylov.gmres(H.A[L], b, H.preconditioner, 1e-8, side=side)
    with make_ctx(bh, d, k, L, gmres_side=bh.LEFT if side == "left" else bh.RIGHT) as ctx:
        X = torch.empty(len(b), dtype=torch.float64, device="cuda")
        it, rr = ctx.solve(cuda(b), X, 1e-8, 100)
        est = ctx.stats()["last_estimate"]
    assert abs(it - it_ref) <= 1
    if side == "right":
        assert rr <= 1.0001e-8
    assert relerr(host(X), xr) <= 1e-6
    # the stopping test's ratio (preconditioned for left GMRES), which the
    # fractional iteration counts of Sec. 5.1 are computed from
    assert est <= 1e-8
    if it == it_ref:
        assert abs(est / (hist[-1] / hist[0]) - 1.0) <= 1e-3, (est, hist[-1] / hist[0])


def mixed_mode(bh, mode):
    return {"fp32": bh.MIXED_FP32, "r64": bh.MIXED_FP32_R64, "rc": bh.MIXED_FP32_RC}[mode]


@pytest.mark.parametrize("d,k,L", [(2, 2, 4), (2, 4, 4), (2, 5, 3), (2, 7, 3), (3, 2, 3),
                                   (3, 4, 2), (3, 7, 2)])
def test_compensated_defect_matches_fp64_defect(bh, d, k, L):
    """bh_defect_compensated, the defect of BH_MIXED_FP32_RC, for an FP32
    iterate: at every node within 2^-36 of S = (|B| (x) |M| + 2 |L| (x) |L| +
    |M| (x) |B|) |x| + |b| (3D: the six terms) of the exact defect b - A x,
    evaluated by the oracle's Kronecker form in FP64.  The bound is the
    worst case of the double-float sums (n^2 2^-48 of the largest partial
    sum for n <= 4k+1 band terms, three sweeps); FP32 arithmetic would leave
    errors of about 2^-24 S.  Checked on a random b and on b = A x, where the
    defect cancels to rounding."""
    N = 2 ** L
    A = kron.kron_matrix(d, k, N).tocsr()
    M, Lm, B = (abs(np.asarray(m)) for m in kron.global_1d(k, N))
    if d == 2:
        S = sp.kron(M, B) + 2 * sp.kron(Lm, Lm) + sp.kron(B, M)
    else:
        def k3(a, b2, c):
            return sp.kron(sp.kron(a, b2), c)
        S = (k3(M, M, B) + k3(M, B, M) + k3(B, M, M)
             + 2 * (k3(M, Lm, Lm) + k3(Lm, M, Lm) + k3(Lm, Lm, M)))
    n = A.shape[0]
    rng = np.random.default_rng(1000 + 10 * d + k)
    x32 = rng.uniform(-1.0, 1.0, n).astype(np.float32)
    xd = x32.astype(np.float64)
    with make_ctx(bh, d, k, L, precision=bh.MIXED_FP32_RC, gmres_side=bh.RIGHT) as ctx:
        X = torch.tensor(x32, device="cuda")
        for case, b in (("random", rng.uniform(-1.0, 1.0, n)), ("cancel", A @ xd)):
            ref = b - A @ xd
            bound = 2.0 ** -36 * (S @ np.abs(xd) + np.abs(b))
            R = torch.empty(n, dtype=torch.float64, device="cuda")
            ctx.defect_compensated(L, X, cuda(b), R)
            err = np.abs(host(R) - ref)
            assert np.all(err <= bound), (case, float((err / bound).max()))
    with make_ctx(bh, d, k, L) as ctx64:          # an FP64 context has no FP32 tables
        with pytest.raises(bh.BiharmError):
            ctx64.defect_compensated(L, X, cuda(xd), torch.empty(n, dtype=torch.float64,
                                                                 device="cuda"))


@pytest.mark.parametrize("d,k,L,mode", [(2, 2, 5, "fp32"), (2, 3, 5, "fp32"), (2, 4, 4, "fp32"),
                                         (3, 2, 3, "fp32"), (3, 3, 3, "fp32"),
                                         (2, 2, 5, "r64"), (2, 4, 4, "r64"), (2, 6, 3, "r64"),
                                         (2, 7, 3, "r64"), (3, 3, 3, "r64"), (3, 5, 2, "r64"),
                                         (2, 2, 5, "rc"), (2, 4, 4, "rc"), (2, 6, 3, "rc"),
                                         (2, 7, 3, "rc"), (3, 3, 3, "rc"), (3, 5, 2, "rc")])
def test_mixed_precision_solve(bh, d, k, L, mode):
    """FP32 V-cycle inside flexible FP64 GMRES (Sec. 5.2, shown there for
    Q2-Q4), and the variants with FP64 or compensated FP32 defects before each
    restriction: the same 1e-8 true residual, at most one more iteration than
    FP64, and the same solution (both within 1e-6 of the dense solve)."""
    n = (k * 2 ** L - 1) ** d
    b = workload.rhs_uniform(n, 21)
    exact = np.linalg.solve(oracle_A(d, k, 2 ** L).toarray(), b)
    prec = mixed_mode(bh, mode)
    res = {}
    for pr in (bh.FP64, prec):
        with make_ctx(bh, d, k, L, precision=pr, gmres_side=bh.RIGHT) as ctx:
            X = torch.empty(n, dtype=torch.float64, device="cuda")
            res[pr] = ctx.solve(cuda(b), X, 1e-8, 100) + (host(X),)
    it64, rr64, x64 = res[bh.FP64]
    it32, rr32, x32 = res[prec]
    assert rr32 <= 1.0001e-8 and rr64 <= 1.0001e-8
    assert it32 <= it64 + 1, (it32, it64)
    assert relerr(x64, exact) <= 1e-6 and relerr(x32, exact) <= 1e-6


@pytest.mark.parametrize("kw", [{"gmres_side": "right"}, {"gmres_side": "left"},
                                {"krylov": "cg"}], ids=["right", "left", "cg"])
def test_solve_resumes_from_a_guess(bh, kw):
    """An interrupted solve (maxit = 2) resumed with bh_solve_guess reaches the
    solve-from-zero tolerance and the dense solution; a converged guess
    returns at once."""
    d, k, L = 2, 3, 5
    n = (k * 2 ** L - 1) ** d
    b = workload.rhs_uniform(n, 17)
    exact = np.linalg.solve(oracle_A(d, k, 2 ** L).toarray(), b)
    opts = {}
    if kw.get("krylov") == "cg":
        opts = dict(krylov=bh.CG, smoother=bh.AVS_ATOMIC, pre_steps=2, post_steps=2)
    else:
        opts = dict(gmres_side=bh.RIGHT if kw["gmres_side"] == "right" else bh.LEFT)
    with make_ctx(bh, d, k, L, **opts) as ctx:
        B = cuda(b)
        X0 = torch.empty(n, dtype=torch.float64, device="cuda")
        it_cold, _ = ctx.solve(B, X0, 1e-8, 200)
        X = torch.empty(n, dtype=torch.float64, device="cuda")
        it1, rr1 = ctx.solve(B, X, 1e-8, 2, raise_on_noconv=False)
        assert it1 == 2 and rr1 > 1e-8
        it2, rr2 = ctx.solve_guess(B, X, 1e-8, 200)
        assert it1 + it2 <= it_cold + 3, (it1, it2, it_cold)
        if opts.get("gmres_side") != bh.LEFT:
            assert rr2 <= 1.0001e-8
        assert relerr(host(X), exact) <= 1e-6
        it3, rr3 = ctx.solve_guess(B, X0, 1e-8, 200)   # already converged
        assert it3 == 0


def test_mixed_precision_exact_local_solver_3d(bh):
    """3D k = 5 with exact local solvers (one dense product per run of a type
    combination, the library's FP64 and FP32 GEMM): FP64 and the FP32 V-cycle with FP64
    defects reach the 1e-8 true residual, at most one iteration apart, both
    within 1e-6 of the dense solve."""
    d, k, L = 3, 5, 2
    n = (k * 2 ** L - 1) ** d
    b = workload.rhs_uniform(n, 23)
    exact = np.linalg.solve(oracle_A(d, k, 2 ** L).toarray(), b)
    res = {}
    for pr in (bh.FP64, bh.MIXED_FP32_R64):
        with make_ctx(bh, d, k, L, precision=pr, local_solver=bh.EXACT,
                      gmres_side=bh.RIGHT) as ctx:
            X = torch.empty(n, dtype=torch.float64, device="cuda")
            res[pr] = ctx.solve(cuda(b), X, 1e-8, 100) + (host(X),)
    (it64, rr64, x64), (it32, rr32, x32) = res[bh.FP64], res[bh.MIXED_FP32_R64]
    assert rr64 <= 1.0001e-8 and rr32 <= 1.0001e-8
    assert abs(it32 - it64) <= 1, (it32, it64)
    assert relerr(x64, exact) <= 1e-6 and relerr(x32, exact) <= 1e-6


@pytest.mark.parametrize("k", [6, 7])
def test_mixed_precision_3d_high_degree(bh, k):
    """3D, k = 6 and 7 on 4^3 cells (the FP32 3D smoothing kernel at its largest
    patch tensors, 512 threads per block): both FP32 V-cycles reach a 1e-8
    true residual with at most one iteration more than FP64, the residual
    evaluated by the oracle's Kronecker form."""
    d, L = 3, 2
    n = (k * 2 ** L - 1) ** d
    b = workload.rhs_uniform(n, 41)
    Aop = kron.KronOperator(d, k, 2 ** L)
    res = {}
    for pr in (bh.FP64, bh.MIXED_FP32, bh.MIXED_FP32_R64, bh.MIXED_FP32_RC):
        with make_ctx(bh, d, k, L, precision=pr, gmres_side=bh.RIGHT) as ctx:
            X = torch.empty(n, dtype=torch.float64, device="cuda")
            res[pr] = ctx.solve(cuda(b), X, 1e-8, 100) + (host(X),)
    it64 = res[bh.FP64][0]
    for pr, (it, rr, x) in res.items():
        true = np.linalg.norm(b - Aop @ x) / np.linalg.norm(b)
        assert rr <= 1.0001e-8 and true <= 1.01e-8, (pr, rr, true)
        assert it <= it64 + 1, (pr, it, it64)


@pytest.mark.parametrize("k,L", [(6, 8), (7, 7)])
def test_fp64_defects_keep_the_fp32_vcycle_converging_on_fine_meshes(bh, k, L):
    """2D, high degree, fine mesh (2.4 M and 0.8 M unknowns): with FP64 or
    compensated FP32 defects before each restriction the FP32 V-cycle needs at
    most two more GMRES iterations than the FP64 one and reaches the same true
    residual floor (the plain FP32 V-cycle needs 150 and 33 iterations here)."""
    d = 2
    n = (k * 2 ** L - 1) ** d
    b = cuda(workload.rhs_uniform(n, k))
    res = {}
    for pr in (bh.FP64, bh.MIXED_FP32_R64, bh.MIXED_FP32_RC):
        with make_ctx(bh, d, k, L, precision=pr, gmres_side=bh.RIGHT) as ctx:
            X = torch.empty(n, dtype=torch.float64, device="cuda")
            res[pr] = ctx.solve(b, X, 1e-8, 100)
    it64, rr64 = res[bh.FP64]
    for pr in (bh.MIXED_FP32_R64, bh.MIXED_FP32_RC):
        itr, rrr = res[pr]
        assert itr <= it64 + 2, (pr, itr, it64)
        assert rrr <= 2.0 * max(rr64, 1e-8), (pr, rrr, rr64)


@pytest.mark.parametrize("d,k,L,sm,ls", [(2, 2, 4, "atomic", "inexact"), (2, 3, 4, "colored", "exact"),
                                         (2, 5, 3, "atomic", "inexact"), (2, 7, 3, "colored", "inexact"),
                                         (3, 2, 3, "atomic", "inexact"), (3, 3, 2, "colored", "inexact")])
def test_cg_solve_matches_oracle(bh, d, k, L, sm, ls):
    """CG preconditioned by the V-cycle with two additive smoothing steps
    (Sec. 5.1): same iterations (+-1), same stopping residual, same solution."""
    H = mg.Hierarchy(d, k, L, smoother="avs", local_solver=ls, pre=2, post=2)
    b = assemble.load_vector(d, k, 2 ** L, assemble.manufactured_f)
    xr, it_ref, hist, rr_ref = krylov.cg(H.A[L], b, H.preconditioner, 1e-8)
    with make_ctx(bh, d, k, L, smoother=bh.AVS_ATOMIC if sm == "atomic" else bh.AVS_COLORED,
                  local_solver=bh.EXACT if ls == "exact" else bh.FDM, pre_steps=2, post_steps=2,
                  krylov=bh.CG) as ctx:
        X = torch.empty(len(b), dtype=torch.float64, device="cuda")
        it, rr = ctx.solve(cuda(b), X, 1e-8, 300)
        est = ctx.stats()["last_estimate"]
    assert abs(it - it_ref) <= 1, (it, it_ref)
    assert rr <= 1.5e-8 and rr_ref <= 1.5e-8
    # CG stops on its recursively updated residual, which stays within
    # rounding of the true one on these small problems.  Its last value is
    # not compared with the oracle's: the residual norm of CG is not monotone,
    # and perturbing the oracle's preconditioner by 1e-13 relative already
    # moves it by a few per cent and can add an iteration.
    assert est <= 1e-8 and abs(est - rr) <= 1e-10, (est, rr)
    assert relerr(host(X), xr) <= 1e-6


@pytest.mark.parametrize("d,k,L,mode", [(2, 3, 4, "fp32"), (3, 2, 3, "fp32"), (2, 5, 3, "r64"),
                                         (2, 5, 3, "rc")])
def test_mixed_precision_cg(bh, d, k, L, mode):
    """FP32 V-cycle inside flexible (Polak-Ribiere) FP64 CG: the same 1e-8
    reduction, at most one more iteration than FP64 CG, both within 1e-6 of
    the dense solve."""
    n = (k * 2 ** L - 1) ** d
    b = workload.rhs_uniform(n, 31)
    exact = np.linalg.solve(oracle_A(d, k, 2 ** L).toarray(), b)
    prec = mixed_mode(bh, mode)
    res = {}
    for pr in (bh.FP64, prec):
        with make_ctx(bh, d, k, L, smoother=bh.AVS_ATOMIC, pre_steps=2, post_steps=2,
                      krylov=bh.CG, precision=pr) as ctx:
            X = torch.empty(n, dtype=torch.float64, device="cuda")
            res[pr] = ctx.solve(cuda(b), X, 1e-8, 300) + (host(X),)
    it64, rr64, x64 = res[bh.FP64]
    it32, rr32, x32 = res[prec]
    assert rr32 <= 1.5e-8 and rr64 <= 1.5e-8
    assert it32 <= it64 + 1, (it32, it64)
    assert relerr(x64, exact) <= 1e-6 and relerr(x32, exact) <= 1e-6


@pytest.mark.parametrize("mode", ["fp32", "r64", "rc"])
def test_mixed_precision_requires_flexible_gmres(bh, mode):
    prec = mixed_mode(bh, mode)
    with pytest.raises(bh.BiharmError) as e:
        make_ctx(bh, 2, 2, 3, precision=prec, gmres_side=bh.LEFT)
    assert "flexible" in str(e.value)


@pytest.mark.parametrize("mode", ["fp32", "r64", "rc"])
def test_mixed_vcycle_error_against_fp64_oracle(bh, mode):
    d, k, L = 2, 4, 4
    H = mg.Hierarchy(d, k, L)
    n = H.A[L].shape[0]
    b = workload.rhs_uniform(n, 31)
    ref = H.vcycle(L, np.zeros(n), b)
    prec = mixed_mode(bh, mode)
    with make_ctx(bh, d, k, L, precision=prec, gmres_side=bh.RIGHT) as ctx:
        X = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.vcycle(L, X, cuda(b))
        err = relerr(host(X), ref)
    assert err <= 1e-4, err


@pytest.mark.parametrize("d,k,N", [(2, 2, 8), (2, 5, 4), (3, 3, 4)])
def test_rhs(bh, d, k, N):
    L = workload.level_of(N)
    with make_ctx(bh, d, k, L) as ctx:
        n = ctx.num_unknowns(L)
        for kind, f in ((bh.RHS_MANUFACTURED, assemble.manufactured_f),
                        (bh.RHS_PAPER_SINE, assemble.paper_sine_f)):
            B = torch.empty(n, dtype=torch.float64, device="cuda")
            ctx.rhs(L, kind, B)
            assert relerr(host(B), assemble.load_vector(d, k, N, f)) <= 1e-12


def test_small_config_end_to_end(bh):
    """The 8 x 8 Q2 problem: apply, one AVS step and the full solve."""
    d, k, N = workload.SMALL_2D[0]
    L = workload.level_of(N)
    b = assemble.load_vector(d, k, N, assemble.manufactured_f)
    A = oracle_A(d, k, N)
    with make_ctx(bh, d, k, L, smoother=bh.AVS_ATOMIC, pre_steps=2, post_steps=2,
                  gmres_side=bh.RIGHT) as ctx:
        B = torch.empty(len(b), dtype=torch.float64, device="cuda")
        ctx.rhs(L, bh.RHS_MANUFACTURED, B)
        assert relerr(host(B), b) <= 1e-12
        X = torch.empty_like(B)
        it, rr = ctx.solve(B, X, 1e-8, 100)
        assert rr <= 1.0001e-8
        u = np.linalg.solve(A.toarray(), b)
        assert relerr(host(X), u) <= 1e-7
        st = ctx.stats()
        assert st["solves"] == 1 and st["last_iters"] == it and st["last_relres"] == rr
        assert st["last_solve_ms"] > 0.0


def test_full_size_apply_and_sampled_avs(bh):
    """2D Q4 on 512 x 512 cells (the sweep workload): the whole apply against
    the oracle's Kronecker form, and one AVS step on 64 sampled nodes whose
    patch solves the oracle computes one by one."""
    d, k, N = 2, 4, 512
    L = workload.level_of(N)
    n1 = k * N - 1
    with make_ctx(bh, d, k, L, smoother=bh.AVS_ATOMIC) as ctx:
        n = ctx.num_unknowns(L)
        x = workload.vector_uniform(n, 1)
        b = workload.rhs_uniform(n, 2)
        X, B = cuda(x), cuda(b)
        Y = torch.empty_like(X)
        ctx.apply_A(L, X, Y)
        Aop = kron.KronOperator(d, k, N)
        Ax = Aop @ x
        assert relerr(host(Y), Ax) <= 1e-12
        ctx.smooth(L, X, B, 1)
        got = host(X)
    r = b - Ax
    M1, _, B1 = kron.global_1d(k, N)
    rng = np.random.default_rng(7)
    omega = 0.25
    for idx in rng.integers(0, n, 64):
        iy, ix = divmod(int(idx), n1)
        gx, gy = ix + 1, iy + 1
        expect = x[idx]
        # patches containing node (gx, gy): vertices v with k(v-1) < g < k(v+1)
        vxs = [v for v in range(1, N) if k * (v - 1) < gx < k * (v + 1)]
        vys = [v for v in range(1, N) if k * (v - 1) < gy < k * (v + 1)]
        for vy in vys:
            for vx in vxs:
                sx = np.arange(k * (vx - 1), k * (vx + 1) - 1)
                sy = np.arange(k * (vy - 1), k * (vy + 1) - 1)
                Mx, Bx = M1[np.ix_(sx, sx)], B1[np.ix_(sx, sx)]
                My, By = M1[np.ix_(sy, sy)], B1[np.ix_(sy, sy)]
                At = np.kron(My, Bx) + np.kron(By, Mx)
                rv = r.reshape(n1, n1)[np.ix_(sy, sx)].ravel()
                yv = np.linalg.solve(At, rv).reshape(len(sy), len(sx))
                expect += omega * yv[iy - sy[0], ix - sx[0]]
        assert abs(got[idx] - expect) <= 1e-10 * max(abs(expect), np.abs(r).max() * 1e-3)


@pytest.mark.parametrize("d,k,N", [(3, 7, 64), (3, 3, 128), (2, 7, 256)])
def test_full_size_apply_on_sampled_rows(bh, d, k, N):
    """apply_A at the largest sweep sizes (3D Q7 on 64^3 cells: 89 M unknowns;
    3D Q3 on 128^3; 2D Q7 on 256^2) on 256 sampled rows, each evaluated from
    the oracle's 1D factors on the node's neighbourhood."""
    L = workload.level_of(N)
    n1 = k * N - 1
    with make_ctx(bh, d, k, L) as ctx:
        n = ctx.num_unknowns(L)
        x = workload.vector_uniform(n, 12)
        X = cuda(x)
        Y = torch.empty_like(X)
        ctx.apply_A(L, X, Y)
        got = host(Y)
        del X, Y
    M1, L1, B1 = (np.asarray(m.todense()) if hasattr(m, "todense") else np.asarray(m)
                  for m in kron.global_1d(k, N))
    terms = ([(1.0, (B1, M1)), (1.0, (M1, B1)), (2.0, (L1, L1))] if d == 2 else
             [(1.0, (B1, M1, M1)), (1.0, (M1, B1, M1)), (1.0, (M1, M1, B1)),
              (2.0, (L1, L1, M1)), (2.0, (M1, L1, L1)), (2.0, (L1, M1, L1))])
    X0 = x.reshape((n1,) * d)
    rng = np.random.default_rng(13)
    scale = np.abs(got).max()
    for idx in rng.integers(0, n, 256):
        c = np.unravel_index(int(idx), (n1,) * d)[::-1]    # (i_x, i_y[, i_z])
        win = [np.arange(max(0, c[a] - 2 * k - 1), min(n1, c[a] + 2 * k + 2)) for a in range(d)]
        xw = X0[np.ix_(*[win[a] for a in reversed(range(d))])]
        y = 0.0
        for cf, ops in terms:
            T = xw
            for a, P in enumerate(ops):
                T = oracle_samples.along(P[np.ix_([c[a]], win[a])], T, a)
            y += cf * T.item()
        assert abs(got[idx] - y) <= 1e-12 * scale, (idx, got[idx], y)


@pytest.mark.parametrize("d,k,N,color", [(2, 4, 512, 0), (2, 7, 256, 5), (3, 4, 64, 0),
                                         (3, 2, 128, 9), (3, 7, 64, 15)])
def test_full_size_mvs_color_on_sampled_patches(bh, d, k, N, color):
    """One color of the colored MVS at the sweep sizes (2D Q4 on 512^2 and Q7
    on 256^2, 3D Q4 on 64^3 and Q2 on 128^3 cells), in the launch
    configuration of the solver (automatic tile): on 24 sampled patches of the
    color, x_v + omega A~_v^-1 R_v (b - A x) from the oracle's Kronecker
    factors, patch by patch; every node outside the color's patches
    unchanged, bit for bit."""
    L = workload.level_of(N)
    omega = smoothers.default_omega("mvs", d, "inexact")
    with make_ctx(bh, d, k, L) as ctx:
        n = ctx.num_unknowns(L)
        x = workload.vector_uniform(n, 3)
        b = workload.rhs_uniform(n, 4)
        X = cuda(x)
        ctx.smooth_colors(L, X, cuda(b), color, color + 1)
        got = host(X)
    oracle_samples.check_color_on_sampled_patches(d, k, N, color, x, b, got, omega)


@pytest.mark.parametrize("k,color,samples", [(5, 0, 24), (6, 9, 12), (7, 3, 8)])
def test_full_size_exact_mvs_color_on_sampled_patches(bh, k, color, samples):
    """One color of the colored MVS with exact local solvers at the 3D sweep
    size (64^3 cells, m^3 = 729 .. 2197 unknowns per patch: one dense product
    per run of patches of a type combination, by the library's FP64 GEMM):
    on sampled patches x_v + omega A_v^-1 R_v (b - A x) with the exact local
    matrix from the oracle's Kronecker factors; every other node unchanged."""
    d, N = 3, 64
    L = workload.level_of(N)
    omega = smoothers.default_omega("mvs", d, "exact")
    with make_ctx(bh, d, k, L, local_solver=bh.EXACT) as ctx:
        n = ctx.num_unknowns(L)
        x = workload.vector_uniform(n, 5)
        b = workload.rhs_uniform(n, 6)
        X = cuda(x)
        ctx.smooth_colors(L, X, cuda(b), color, color + 1)
        got = host(X)
        del X
    oracle_samples.check_color_on_sampled_patches(d, k, N, color, x, b, got, omega,
                                                  samples=samples, exact=True)


def test_edge_cases(bh):
    d, k, L = 2, 2, 3
    with make_ctx(bh, d, k, L) as ctx:
        n = ctx.num_unknowns(L)
        X = torch.ones(n, dtype=torch.float64, device="cuda")
        it, rr = ctx.solve(torch.zeros(n, dtype=torch.float64, device="cuda"), X)
        assert it == 0 and rr == 0.0 and float(X.abs().max()) == 0.0
        with pytest.raises(bh.BiharmError):
            ctx.apply_A(L + 1, X, X.clone())
        with pytest.raises(bh.BiharmError):
            ctx.apply_A(L, X, X)          # aliasing is rejected
        with pytest.raises(ValueError):
            ctx.apply_A(L, X[:-1], X[:-1].clone())
        with pytest.raises(bh.BiharmError):
            ctx.prolongate_add(1, X, X)   # no level below the coarse one
        bad = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        with pytest.raises(bh.BiharmError):
            ctx.solve(bad, X)
        # level 1 (N = 2): one patch; the V-cycle is the exact coarse solve
        n1 = ctx.num_unknowns(1)
        b1 = workload.rhs_uniform(n1, 3)
        X1 = torch.zeros(n1, dtype=torch.float64, device="cuda")
        ctx.vcycle(1, X1, cuda(b1))
        assert relerr(host(X1), np.linalg.solve(oracle_A(d, k, 2).toarray(), b1)) <= 1e-12
