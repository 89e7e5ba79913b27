"""Batched form, through the C ABI.

Oracle parity of the kernels the batch runs (the batched sweeps, transfers,
patch kernels, coarse solve and vector kernels): one batched V-cycle of a
mixed-degree batch against the oracle's Algorithm 1 per problem (1e-10),
batched GMRES (right and left) against the oracle's GMRES (iterations +-1,
1e-8 true residual, solution to 1e-6), the FP32 V-cycle with FP64 defects
against the FP64 oracle, and one color of the batched MVS kernel inside a
batch that holds the 2D Q4 problem on 512^2 cells on sampled patches.  At
the benchmark's sizes the batched solves are checked by a property that holds
at any size: the true residual evaluated by the oracle's Kronecker operator.
Further: a problem's result does not depend on the mix, and equals its own
single-context solve."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle_samples  # noqa: E402
import workload  # noqa: E402
from oracle import assemble, kron, krylov, mg, smoothers  # noqa: E402
from oracle.patches import color as color_of  # noqa: E402


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


# a mixed-degree batch small enough for the oracle: every degree, levels 1..4
MIX = [(2, 2, 4), (2, 3, 3), (2, 4, 3), (2, 5, 2), (2, 6, 2), (2, 7, 2), (2, 3, 1), (2, 2, 2)]


def hierarchies():
    return [mg.Hierarchy(d, k, L) for d, k, L in MIX]


def rhs_rough_solution(A, seed):
    """b = A x* for a seeded x* ~ U[-1, 1]: the right-hand side of the
    benchmark's solves (the FP64 rounding floor of the true residual is O(eps))."""
    xs = workload.vector_uniform(A.shape[0], seed)
    return A @ xs, xs


def test_batched_vcycle_matches_oracle_per_problem(bh):
    Hs = hierarchies()
    bs = [workload.rhs_uniform(H.A[H.L].shape[0], 200 + i) for i, H in enumerate(Hs)]
    refs = [H.vcycle(H.L, np.zeros_like(b), b) for H, b in zip(Hs, bs)]
    with bh.Batch([bh.default_params(d, k, L) for d, k, L in MIX]) as batch:
        B = [cuda(b) for b in bs]
        X = [torch.full_like(v, float("nan")) for v in B]
        batch.vcycle(B, X)
        for (d, k, L), x, ref in zip(MIX, X, refs):
            assert relerr(host(x), ref) <= 1e-10, (k, L, relerr(host(x), ref))


@pytest.mark.parametrize("precision", ["fp64", "rc"])
def test_batched_vcycle_with_two_penalties_of_one_degree(bh, precision):
    """Problems of one degree with different penalties gamma have different
    tables, which the per-degree patch launches take as a kernel parameter:
    the batch splits them into one launch per table class, and each problem's
    V-cycle equals the oracle's Algorithm 1 with its own gamma (1e-10 in FP64;
    the FP32 V-cycle's 1e-3 bound otherwise)."""
    probs = [(2, 3, 3, None), (2, 3, 3, 20.0), (2, 3, 4, 6.0), (2, 5, 2, None)]
    Hs = [mg.Hierarchy(d, k, L, gamma=g) for d, k, L, g in probs]
    bs = [workload.rhs_uniform(H.A[H.L].shape[0], 800 + i) for i, H in enumerate(Hs)]
    prec = bh.FP64 if precision == "fp64" else bh.MIXED_FP32_RC
    params = []
    for d, k, L, g in probs:
        kw = {"precision": prec}
        if g is not None:
            kw["gamma"] = g
        params.append(bh.default_params(d, k, L, **kw))
    with bh.Batch(params) as batch:
        B = [cuda(b) for b in bs]
        X = [torch.empty_like(v) for v in B]
        batch.vcycle(B, X)
        for (d, k, L, g), H, b, x in zip(probs, Hs, bs, X):
            ref = H.vcycle(H.L, np.zeros_like(b), b)
            tol = 1e-10 if precision == "fp64" else 1e-3
            assert relerr(host(x), ref) <= tol, (k, L, g, relerr(host(x), ref))


@pytest.mark.parametrize("side", ["right", "left"])
def test_batched_solve_matches_oracle_gmres(bh, side):
    Hs = hierarchies()
    bs = [rhs_rough_solution(H.A[H.L], 300 + i)[0] if i % 2 == 0 else
          workload.rhs_uniform(H.A[H.L].shape[0], 300 + i) for i, H in enumerate(Hs)]
    refs = [krylov.gmres(H.A[H.L], b, H.preconditioner, 1e-8, side=side) for H, b in zip(Hs, bs)]
    params = [bh.default_params(d, k, L, gmres_side=bh.RIGHT if side == "right" else bh.LEFT)
              for d, k, L in MIX]
    with bh.Batch(params) as batch:
        B = [cuda(b) for b in bs]
        X = [torch.empty_like(v) for v in B]
        its, rrs = batch.solve(B, X, 1e-8, 100)
        for (d, k, L), x, it, rr, (xr, it_ref, hist, rr_ref), H, b in zip(MIX, X, its, rrs, refs,
                                                                          Hs, bs):
            assert abs(it - it_ref) <= 1, (k, L, it, it_ref)
            xg = host(x)
            assert relerr(xg, xr) <= 1e-6, (k, L)
            true = np.linalg.norm(b - H.A[H.L] @ xg) / np.linalg.norm(b)
            assert abs(true - rr) <= 1e-3 * rr + 1e-15, (k, L, true, rr)
            if side == "right":
                assert rr <= 1.0001e-8, (k, L, rr)


def test_batched_solve_restarts(bh):
    """GMRES(4) on problems that need more than four iterations: the restarted
    batch reaches the tolerance like the oracle's restarted GMRES (iterations
    +-1), and a problem that would need more than maxit iterations reports
    non-convergence without stopping the others."""
    probs = [(2, 2, 4), (2, 4, 3), (2, 6, 2)]
    Hs = [mg.Hierarchy(d, k, L) for d, k, L in probs]
    bs = [rhs_rough_solution(H.A[H.L], 400 + i)[0] for i, H in enumerate(Hs)]
    refs = [krylov.gmres(H.A[H.L], b, H.preconditioner, 1e-8, restart=4) for H, b in zip(Hs, bs)]
    params = [bh.default_params(d, k, L, gmres_restart=4) for d, k, L in probs]
    with bh.Batch(params) as batch:
        B = [cuda(b) for b in bs]
        X = [torch.empty_like(v) for v in B]
        its, rrs = batch.solve(B, X, 1e-8, 100)
        for (d, k, L), it, rr, x, (xr, it_ref, _, _) in zip(probs, its, rrs, X, refs):
            assert it_ref > 4 and abs(it - it_ref) <= 1, (k, L, it, it_ref)
            assert rr <= 1.0001e-8
            assert relerr(host(x), xr) <= 1e-6
        its2, rrs2 = batch.solve(B, X, 1e-8, 3, raise_on_noconv=False)
        assert its2 == [3, 3, 3] and min(rrs2) > 1e-8
        with pytest.raises(bh.BiharmError):
            batch.solve(B, X, 1e-8, 3)


@pytest.mark.parametrize("precision", ["r64", "rc"])
def test_batched_mixed_precision_vcycle_and_solve(bh, precision):
    """The FP32 V-cycle with FP64 defects (BH_MIXED_FP32_R64) or compensated
    FP32 defects (BH_MIXED_FP32_RC) in the batch.
    One V-cycle: within 1e-3 of the FP64 oracle's -- FP32 rounding (eps 6e-8)
    amplified by the condition numbers of the patch problems, which grow with
    the degree (1.5e-4 measured at k = 6) -- and no farther from the same
    V-cycle of a single FP32 context than twice that context's own FP32
    rounding error (the same arithmetic per patch, in another rounding order:
    2.7e-5 measured at k = 4 against an FP32 error of 2e-5).  Then flexible
    GMRES to the 1e-8 true residual with at most one iteration more than the
    oracle's FP64 GMRES, the solution within 1e-6 of it."""
    Hs = hierarchies()
    bs = [rhs_rough_solution(H.A[H.L], 500 + i)[0] for i, H in enumerate(Hs)]
    prec = bh.MIXED_FP32_R64 if precision == "r64" else bh.MIXED_FP32_RC
    params = [bh.default_params(d, k, L, precision=prec) for d, k, L in MIX]
    with bh.Batch(params) as batch:
        B = [cuda(b) for b in bs]
        X = [torch.empty_like(v) for v in B]
        batch.vcycle(B, X)
        for (d, k, L), H, b, x, p in zip(MIX, Hs, bs, X, params):
            ref = H.vcycle(H.L, np.zeros_like(b), b)
            assert relerr(host(x), ref) <= 1e-3, (k, L, relerr(host(x), ref))
            with bh.Context(p) as c:
                xc = torch.zeros_like(x)
                c.vcycle(L, xc, cuda(b))
                own = relerr(host(xc), ref)          # the single context's FP32 error
                assert relerr(host(x), host(xc)) <= 2.0 * own + 1e-7, (k, L, own)
        its, rrs = batch.solve(B, X, 1e-8, 100)
        for (d, k, L), H, b, x, it, rr in zip(MIX, Hs, bs, X, its, rrs):
            xr, it_ref, _, _ = krylov.gmres(H.A[H.L], b, H.preconditioner, 1e-8)
            assert rr <= 1.0001e-8 and it <= it_ref + 1, (k, L, it, it_ref, rr)
            assert relerr(host(x), xr) <= 1e-6


@pytest.mark.parametrize("color", [0, 5])
def test_batched_color_with_the_512_cell_problem(bh, color):
    """One color of the batched MVS kernel in a batch of 2D Q4 on 512^2 cells
    (checked on 24 sampled patches) with two small problems of other degrees
    (checked completely against the oracle's sequential MVS over the color)."""
    probs = [(2, 4, 9), (2, 7, 3), (2, 2, 4)]
    xs, bs = [], []
    for i, (d, k, L) in enumerate(probs):
        n = (k * 2 ** L - 1) ** d
        xs.append(workload.vector_uniform(n, 60 + i))
        bs.append(workload.rhs_uniform(n, 70 + i))
    with bh.Batch([bh.default_params(d, k, L) for d, k, L in probs]) as batch:
        X = [cuda(x) for x in xs]
        batch.smooth_colors(X, [cuda(b) for b in bs], color, color + 1)
        got = [host(x) for x in X]
    d, k, L = probs[0]
    oracle_samples.check_color_on_sampled_patches(d, k, 2 ** L, color, xs[0], bs[0], got[0], 1.0)
    for (d, k, L), x, b, g in zip(probs[1:], xs[1:], bs[1:], got[1:]):
        N = 2 ** L
        A = assemble.c0ip_matrix(d, k, N)
        from oracle.patches import LocalSolvers
        loc = LocalSolvers(assemble.c0ip_matrix(d, k, N, mixed=False), d, k, N)
        order = [v for v in smoothers.mvs_order(d, N) if color_of(v) == color]
        ref = smoothers.mvs_step(A, loc, b, x, 1.0, order=order)
        assert relerr(g - x, ref - x) <= 1e-10, (k, L)


@pytest.mark.parametrize("precision", ["fp64", "r64", "rc"])
def test_batched_sweep_solve_reaches_true_residual(bh, precision):
    """The benchmark's workload (2D Q2-Q4 on 512^2 and Q5-Q7 on 256^2 cells,
    b = A x* with x* ~ U[-1, 1]) solved as one batch by right-preconditioned
    GMRES: the true residual of every returned solution, evaluated by the
    oracle's Kronecker operator, is at most 1e-8 (plus the rounding of its own
    evaluation), and equals the residual the batch reports."""
    probs = workload.SWEEP_2D
    ops = [kron.KronOperator(d, k, N) for d, k, N in probs]
    xstar = [workload.vector_uniform((k * N - 1) ** d, k) for d, k, N in probs]
    bs = [A @ xs for A, xs in zip(ops, xstar)]
    prec = {"fp64": bh.FP64, "r64": bh.MIXED_FP32_R64, "rc": bh.MIXED_FP32_RC}[precision]
    params = [bh.default_params(d, k, workload.level_of(N), precision=prec) for d, k, N in probs]
    with bh.Batch(params) as batch:
        B = [cuda(b) for b in bs]
        X = [torch.empty_like(v) for v in B]
        its, rrs = batch.solve(B, X, 1e-8, 100)
        got = [host(x) for x in X]
    for (d, k, N), A, b, x, it, rr in zip(probs, ops, bs, got, its, rrs):
        true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert rr <= 1.0001e-8 and true <= 1.01e-8, (k, N, rr, true)
        assert abs(true - rr) <= 1e-2 * rr, (k, N, true, rr)
        assert 1 <= it <= 40, (k, N, it)


def single(bh, d, k, L, b):
    with bh.Context(bh.default_params(d, k, L)) as ctx:
        x = torch.empty_like(b)
        it, rr = ctx.solve(b, x, 1e-8, 50)
        torch.cuda.synchronize()
        return it, rr, x.cpu().numpy()


def test_batch_matches_single_solves(bh):
    probs = [(2, 2, 5), (2, 7, 3), (2, 3, 4), (2, 5, 2), (2, 4, 4), (2, 6, 3), (2, 2, 6), (2, 3, 1)]
    params = [bh.default_params(d, k, L) for d, k, L in probs]
    bs = [torch.tensor(workload.rhs_uniform((k * 2 ** L - 1) ** 2, 100 + i), dtype=torch.float64,
                       device="cuda") for i, (d, k, L) in enumerate(probs)]
    xs = [torch.empty_like(b) for b in bs]
    with bh.Batch(params) as batch:
        its, rrs = batch.solve(bs, xs, 1e-8, 50)
        torch.cuda.synchronize()
        got = [x.cpu().numpy() for x in xs]
        # a second call on the same batch gives the same answer
        xs2 = [torch.empty_like(b) for b in bs]
        its2, _ = batch.solve(bs, xs2, 1e-8, 50)
        torch.cuda.synchronize()
        assert its2 == its
        for a, x2 in zip(got, xs2):
            assert np.abs(a - x2.cpu().numpy()).max() <= 1e-12 * np.abs(a).max()
    for (d, k, L), b, it, rr, x in zip(probs, bs, its, rrs, got):
        it1, rr1, x1 = single(bh, d, k, L, b)
        assert abs(it - it1) <= 1, (k, L, it, it1)
        assert np.abs(x - x1).max() <= 1e-9 * np.abs(x1).max(), (k, L)
        # the true residuals of two iterates that agree to 1e-9 relative differ by
        # up to ||A|| 1e-9 ||x|| / ||b||: compare them to 1e-3 relative
        assert abs(rr - rr1) <= 1e-3 * rr1 + 1e-14   # 1e-14: the level-1 exact solve


def test_batch_result_independent_of_the_mix(bh):
    k, L = 4, 4
    n = (k * 2 ** L - 1) ** 2
    b = torch.tensor(workload.rhs_uniform(n, 7), dtype=torch.float64, device="cuda")
    outs = []
    for mix in ([(4, 4)], [(2, 6), (4, 4), (7, 3)], [(4, 4), (3, 5), (5, 3), (6, 2)]):
        params = [bh.default_params(2, kk, LL) for kk, LL in mix]
        bs = [b if (kk, LL) == (k, L) else
              torch.tensor(workload.rhs_uniform((kk * 2 ** LL - 1) ** 2, kk), dtype=torch.float64,
                           device="cuda") for kk, LL in mix]
        xs = [torch.empty_like(v) for v in bs]
        with bh.Batch(params) as batch:
            its, _ = batch.solve(bs, xs, 1e-8, 50)
        i = mix.index((k, L))
        outs.append((its[i], xs[i].cpu().numpy()))
    for it, x in outs[1:]:
        assert it == outs[0][0]
        assert np.abs(x - outs[0][1]).max() <= 1e-12 * np.abs(outs[0][1]).max()


def test_batch_tiles_and_graph(bh):
    params = [bh.default_params(2, k, 4) for k in (2, 3, 4)]
    with bh.Batch(params) as batch:
        t1 = batch.vcycle_time(2)
        batch.set_tile(3, 1)
        t2 = batch.vcycle_time(2)
        assert t1 > 0 and t2 > 0
        with pytest.raises(bh.BiharmError):
            batch.set_tile(7, 33)
    with pytest.raises(bh.BiharmError):
        bh.Batch([bh.default_params(3, 2, 3)])      # batched form is 2D
    with pytest.raises(bh.BiharmError):              # one precision per batch
        bh.Batch([bh.default_params(2, 2, 3),
                  bh.default_params(2, 3, 3, precision=bh.MIXED_FP32_R64)])
    with pytest.raises(bh.BiharmError):              # FP32 V-cycle needs right GMRES
        bh.Batch([bh.default_params(2, 2, 3, precision=bh.MIXED_FP32_R64, gmres_side=bh.LEFT)])
    with bh.Batch([bh.default_params(2, 2, 3, precision=bh.MIXED_FP32_RC)]) as batch:
        with pytest.raises(bh.BiharmError):          # compensated defects: graph form only
            batch.set_persistent(True)


def test_batch_autotuner_keeps_results(bh, tmp_path, monkeypatch):
    """tune_batch times the batch's own V-cycle for candidate tiles, caches the
    choice, and the tuned batch reaches the same solutions as the batch with
    default tiles (a tile shape only decides which patches share a block, and
    whether a patch takes the interior or the general path: rounding-level
    differences)."""
    from paper_2412_05082_gb300 import autotune
    monkeypatch.setenv("BIHARM_TUNE_CACHE", str(tmp_path / "tiles.json"))
    probs = [(2, 2, 5), (2, 5, 3), (2, 7, 3)]
    params = [bh.default_params(d, k, L) for d, k, L in probs]
    bs = [torch.tensor(workload.rhs_uniform((k * 2 ** L - 1) ** 2, 60 + k), dtype=torch.float64,
                       device="cuda") for _, k, L in probs]
    xs0 = [torch.empty_like(b) for b in bs]
    xs1 = [torch.empty_like(b) for b in bs]
    with bh.Batch(params) as batch:
        its0, _ = batch.solve(bs, xs0, 1e-8, 50)
    with bh.Batch(params) as batch:
        tiles = autotune.tune_batch(batch, probs, reps=1)
        assert set(tiles) == {2, 5, 7} and all(pb >= 1 for pb in tiles.values())
        its1, _ = batch.solve(bs, xs1, 1e-8, 50)
    with bh.Batch(params) as batch:        # second call: read from the cache
        assert autotune.tune_batch(batch, probs) == tiles
    assert all(abs(a - b) <= 1 for a, b in zip(its1, its0))
    for a, b in zip(xs0, xs1):
        assert (a - b).abs().max().item() <= 1e-6 * b.abs().max().item()


def test_two_live_batches_with_different_tile_memory(bh):
    """A batch whose tiles need little shared memory, created while another
    batch with large tiles is alive, must not lower the kernel's limit under
    the first batch's captured graph: both keep solving."""
    big = [(2, 7, 4), (2, 6, 4)]
    small = [(2, 2, 5)]
    rhs = {p: torch.tensor(workload.rhs_uniform((p[1] * 2 ** p[2] - 1) ** 2, p[1]),
                           dtype=torch.float64, device="cuda") for p in big + small}
    with bh.Batch([bh.default_params(d, k, L) for d, k, L in big]) as b1:
        b1.set_tile(7, 6)
        xs1 = [torch.empty_like(rhs[p]) for p in big]
        its1, _ = b1.solve([rhs[p] for p in big], xs1, 1e-8, 50)
        with bh.Batch([bh.default_params(d, k, L) for d, k, L in small]) as b2:
            b2.set_tile(2, 1)
            xs2 = [torch.empty_like(rhs[p]) for p in small]
            b2.solve([rhs[p] for p in small], xs2, 1e-8, 50)
            again = [torch.empty_like(rhs[p]) for p in big]
            its2, _ = b1.solve([rhs[p] for p in big], again, 1e-8, 50)
    assert its2 == its1
    for a, b in zip(xs1, again):
        assert torch.equal(a, b)


@pytest.mark.parametrize("precision", ["fp64", "r64"])
def test_persistent_vcycle_equals_the_graph_and_the_oracle(bh, precision):
    """The persistent form (one cooperative launch walking the V-cycle's phases
    with a grid barrier between them) runs the same per-problem arithmetic as
    the captured graph: one V-cycle equals the graph's to rounding and, in
    FP64, the oracle's Algorithm 1 to 1e-10; a right-preconditioned solve takes
    the same iterations and reaches the 1e-8 true residual."""
    Hs = hierarchies()
    bs = [rhs_rough_solution(H.A[H.L], 600 + i)[0] for i, H in enumerate(Hs)]
    prec = bh.FP64 if precision == "fp64" else bh.MIXED_FP32_R64
    with bh.Batch([bh.default_params(d, k, L, precision=prec) for d, k, L in MIX]) as batch:
        B = [cuda(b) for b in bs]
        Xg = [torch.empty_like(v) for v in B]
        Xp = [torch.empty_like(v) for v in B]
        batch.vcycle(B, Xg)
        its_g, rr_g = batch.solve(B, [torch.empty_like(v) for v in B], 1e-8, 100)
        batch.set_persistent(True)
        batch.vcycle(B, Xp)
        its_p, rr_p = batch.solve(B, [torch.empty_like(v) for v in B], 1e-8, 100)
        for (d, k, L), H, b, xg, xp in zip(MIX, Hs, bs, Xg, Xp):
            # up to k = 4 both forms run the same tile code; above it the graph
            # form's interior tiles take the folded fast diagonalization and the
            # persistent kernel the unfolded one, equal up to the rounding of
            # either (FP64), or of the FP32 V-cycle (checked against the oracle)
            ref = H.vcycle(H.L, np.zeros_like(b), b)
            if precision == "fp64":
                assert relerr(host(xp), host(xg)) <= (1e-13 if k <= 4 else 1e-11), (k, L)
                assert relerr(host(xp), ref) <= 1e-10, (k, L)
            else:
                if k <= 4:
                    assert relerr(host(xp), host(xg)) <= 1e-6, (k, L)
                assert relerr(host(xp), ref) <= 1e-3, (k, L)
                assert relerr(host(xg), ref) <= 1e-3, (k, L)
        assert its_p == its_g
        assert all(r <= 1.0001e-8 for r in rr_p)


def test_persistent_barrier_wait_is_bounded(bh):
    """The persistent kernel's grid barrier made to expect one block more than
    the launch has: every block's wait runs out after the given bound, the
    kernel ends with its status word set (BH_ETIMEOUT, no fault, no hang), and
    the batch keeps working afterwards in both forms."""
    import time
    probs = [(2, 2, 4), (2, 5, 3)]
    Hs = [mg.Hierarchy(d, k, L) for d, k, L in probs]
    bs = [workload.rhs_uniform(H.A[H.L].shape[0], 700 + i) for i, H in enumerate(Hs)]
    with bh.Batch([bh.default_params(d, k, L) for d, k, L in probs]) as batch:
        t0 = time.perf_counter()
        st = batch.check_barrier_timeout(50.0)
        dt = time.perf_counter() - t0
        assert st == bh.BH_ETIMEOUT, st
        assert dt < 10.0, dt
        B = [cuda(b) for b in bs]
        for persistent in (False, True):
            batch.set_persistent(persistent)
            X = [torch.empty_like(v) for v in B]
            batch.vcycle(B, X)
            for H, b, x in zip(Hs, bs, X):
                assert relerr(host(x), H.vcycle(H.L, np.zeros_like(b), b)) <= 1e-10
