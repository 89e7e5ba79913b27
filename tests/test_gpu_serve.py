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
    p = bh.default_params(d, k, L, precision=bh.MIXED_FP32_RC, gmres_side=bh.RIGHT,
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


def test_forced_allocation_failure_fails_one_request_and_the_server_goes_on(bh):
    """Host-side fault injection: the device allocations of the first request's
    hierarchy fail (BH_ENOMEM, as an out-of-memory cudaMalloc would); that
    request reports the failure, its memory reservation is released, and the
    next request of the same shape is served normally."""
    d, k, L = 2, 3, 4
    b = workload.rhs_uniform((k * 2 ** L - 1) ** d, 11)
    x1, x2 = np.zeros_like(b), np.zeros_like(b)
    with bh.Server(slots=1) as srv:
        bh.fault_inject_alloc(2, 1000)       # the third allocation onwards fails
        try:
            r1 = srv.wait(srv.submit(d, k, L, b, x1), 300.0)
        finally:
            bh.fault_inject_alloc(0, 0)
        st = srv.stats()
        r2 = srv.wait(srv.submit(d, k, L, b, x2), 300.0)
        st2 = srv.stats()
    assert r1["status"] == bh.BH_ENOMEM
    assert st["failed"] == 1 and st["reserved_bytes"] == 0 and st["resident_contexts"] == 0
    assert r2["status"] == bh.BH_OK and r2["relres"] <= 1.0001e-8
    assert st2["created"] == 1 and st2["failed"] == 1
    # a context created under the same injection fails cleanly too
    bh.fault_inject_alloc(0, 1)
    try:
        with pytest.raises(bh.BiharmError) as e:
            bh.Context(bh.default_params(d, k, L))
    finally:
        bh.fault_inject_alloc(0, 0)
    assert e.value.status == bh.BH_ENOMEM
    with bh.Context(bh.default_params(d, k, L)) as ctx:   # and afterwards all is well
        assert ctx.num_unknowns() == (k * 2 ** L - 1) ** d


def test_deadlines_and_cancellation_drop_queued_requests_only(bh):
    """One slot, a long request first: requests queued behind it with a short
    deadline are dropped (BH_ETIMEOUT) when the slot reaches them, a cancelled
    one reports BH_ECANCELED, a running one cannot be cancelled, and the
    requests without a deadline are all served."""
    big = (2, 6, 8)
    small = (2, 2, 4)
    bb = workload.rhs_uniform((big[1] * 2 ** big[2] - 1) ** 2, 1)
    bs = workload.rhs_uniform((small[1] * 2 ** small[2] - 1) ** 2, 2)
    with bh.Server(slots=1) as srv:
        xb = np.zeros_like(bb)
        t_big = srv.submit(*big, bb, xb)
        outs = [np.zeros_like(bs) for _ in range(6)]
        late = [srv.submit(*small, bs, outs[i], deadline=1e-3) for i in range(3)]
        keep = [srv.submit(*small, bs, outs[3 + i]) for i in range(2)]
        cancelled = srv.submit(*small, bs, outs[5])
        srv.cancel(cancelled)
        import time
        while srv.stats()["running"] == 0:
            time.sleep(0.001)
        with pytest.raises(bh.BiharmError) as e:
            srv.cancel(t_big)                   # already running
        assert e.value.status == bh.BH_EBUSY
        r_big = srv.wait(t_big, 300.0)
        r_late = [srv.wait(t, 300.0) for t in late]
        r_keep = [srv.wait(t, 300.0) for t in keep]
        r_can = srv.wait(cancelled, 300.0)
        st = srv.stats()
    assert r_big["status"] == bh.BH_OK
    assert all(r["status"] == bh.BH_ETIMEOUT for r in r_late)
    assert all(r["status"] == bh.BH_OK and r["relres"] <= 1.0001e-8 for r in r_keep)
    assert r_can["status"] == bh.BH_ECANCELED
    assert st["dropped"] == 3 and st["cancelled"] == 1 and st["completed"] == 7


def test_abandoned_tickets_do_not_hold_up_other_clients(bh):
    """A client thread submits requests and goes away without waiting for
    them; the other client's requests are served, the abandoned ones complete
    in the background, and destroying the server releases them."""
    import threading
    d, k, L = 2, 3, 4
    b = workload.rhs_uniform((k * 2 ** L - 1) ** d, 5)
    keep_alive = []
    with bh.Server(slots=2) as srv:
        def client():
            for _ in range(4):
                x = np.zeros_like(b)
                keep_alive.append(x)         # the buffers outlive the thread
                srv.submit(d, k, L, b, x)
        th = threading.Thread(target=client)
        th.start()
        th.join()
        mine = [np.zeros_like(b) for _ in range(3)]
        res = [srv.wait(srv.submit(d, k, L, b, x), 300.0) for x in mine]
        import time
        t0 = time.time()
        while srv.stats()["completed"] < 7 and time.time() - t0 < 60:
            time.sleep(0.01)
        st = srv.stats()
    assert all(r["status"] == bh.BH_OK for r in res)
    assert st["completed"] == 7 and st["failed"] == 0
    for x in keep_alive:                     # the abandoned solves finished too
        assert np.abs(x).max() > 0
