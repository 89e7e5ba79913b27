"""Serving form: each request's result is the same alone and in a mix of
concurrent requests (within 1e-12 relative: the same kernels in the same
order on another stream), admission by memory footprint evicts idle
hierarchies, and requests larger than the budget are refused."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workload  # noqa: E402


@pytest.fixture(scope="module")
def bh():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: the -m gpu tests need a GB300")
    import paper_2412_05082_gb300 as m
    m.load()
    return m


REQS = [(2, 2, 6), (3, 2, 3), (2, 5, 4), (2, 3, 5), (3, 3, 2), (2, 7, 3), (2, 4, 5), (2, 2, 6),
        (3, 4, 2), (2, 6, 3)]


def alone(bh, d, k, L, b):
    p = bh.default_params(d, k, L, precision=bh.MIXED_FP32_R64, gmres_side=bh.RIGHT,
                          gmres_restart=30)
    with bh.Context(p) as ctx:
        B = torch.tensor(b, dtype=torch.float64, device="cuda")
        X = torch.empty_like(B)
        it, rr = ctx.solve(B, X, 1e-8, 200)
        torch.cuda.synchronize()
        return it, X.cpu().numpy()


def test_results_same_alone_and_in_the_mix(bh):
    rhs = [workload.rhs_uniform((k * 2 ** L - 1) ** d, 500 + i) for i, (d, k, L) in enumerate(REQS)]
    outs = [np.zeros_like(b) for b in rhs]
    with bh.Server(slots=4) as srv:
        tickets = [srv.submit(d, k, L, b, x) for (d, k, L), b, x in zip(REQS, rhs, outs)]
        res = [srv.wait(t, 300.0) for t in tickets]
        st = srv.stats()
        # a shape whose hierarchy is resident and idle reuses it (two requests
        # of one shape that overlap in time need two, so the mix above may
        # have created one per request)
        xr = np.zeros_like(rhs[0])
        again = srv.wait(srv.submit(*REQS[0], rhs[0], xr), 300.0)
        st2 = srv.stats()
    assert st["completed"] == len(REQS)
    assert len(set(REQS)) <= st["created"] <= len(REQS)
    assert again["status"] == bh.BH_OK and st2["created"] == st["created"]
    assert again["iters"] == res[0]["iters"]
    assert np.abs(xr - outs[0]).max() <= 1e-12 * np.abs(outs[0]).max()
    for (d, k, L), b, x, r in zip(REQS, rhs, outs, res):
        assert r["status"] == bh.BH_OK
        assert r["relres"] <= 1.0001e-8
        assert r["latency_s"] >= r["service_s"] > 0
        it, xa = alone(bh, d, k, L, b)
        assert r["iters"] == it
        assert np.abs(x - xa).max() <= 1e-12 * np.abs(xa).max()


def test_admission_by_footprint_evicts_idle_hierarchies(bh):
    # a budget that holds about two of these hierarchies at a time
    shapes = [(2, 4, 6), (2, 5, 5), (2, 6, 5), (2, 3, 6)]
    with bh.Server(slots=2, mem_budget_bytes=260e6) as srv:
        rhs = [workload.rhs_uniform((k * 2 ** L - 1) ** 2, i) for i, (_, k, L) in enumerate(shapes)]
        outs = [np.zeros_like(b) for b in rhs]
        tickets = [srv.submit(d, k, L, b, x) for (d, k, L), b, x in zip(shapes, rhs, outs)]
        res = [srv.wait(t, 300.0) for t in tickets]
        st = srv.stats()
        assert all(r["status"] == bh.BH_OK for r in res)
        assert st["evictions"] >= 1
        assert st["reserved_bytes"] <= 260e6
        big = workload.rhs_uniform((2 * 2 ** 10 - 1) ** 2, 9)
        xb = np.zeros_like(big)
        r = srv.wait(srv.submit(2, 2, 10, big, xb), 300.0)
        assert r["status"] == bh.BH_ENOMEM
