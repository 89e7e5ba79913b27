"""bh_apply_A_noalloc, the allocation-free apply_A, against bh_apply_A.

It is for callers that cannot allocate device memory where they need the
operator (a plugin inside a framework that owns all device allocations, a
latency-critical loop that cannot absorb cudaMalloc's synchronization): its
sweep intermediates live in one static device array shared by all calls.
Two calls in a row must both agree with the context-based entry point to the
apply tolerance of the parity tests (1e-12 relative).  This file is
collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import workload  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module")
def bh():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: the -m gpu tests need a GB300")
    import paper_2412_05082_gb300 as m
    m.load()
    return m


def relerr(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# level 1 (N = 2: the rows touching both faces), small and mid sizes, and the
# largest problems that fit the static array: 2D Q6 on 256^2 cells (2,356,225
# of at most 2,796,202 unknowns) and 3D Q7 on 16^3 cells (1,367,631 of at most
# 1,398,101)
@pytest.mark.parametrize("d,k,L", [(2, 3, 1), (3, 2, 1), (3, 7, 1), (2, 4, 6), (2, 2, 9),
                                   (2, 7, 3), (3, 3, 3), (3, 2, 5), (2, 6, 8), (3, 7, 4)])
def test_noalloc_apply_matches_context_apply_twice(bh, d, k, L):
    with bh.Context(bh.default_params(d, k, L)) as ctx:
        n = ctx.num_unknowns(L)
        for seed in (1, 2):  # two calls in a row on different inputs
            x = torch.tensor(workload.vector_uniform(n, seed), dtype=torch.float64, device="cuda")
            ref = torch.empty_like(x)
            got = torch.full_like(x, float("nan"))
            ctx.apply_A(L, x, ref)
            bh.apply_A_noalloc(d, k, L, 0.0, x, got)
            torch.cuda.synchronize()
            assert relerr(got, ref) <= TOL, (seed, relerr(got, ref))


def test_noalloc_rebuilds_its_cached_table_when_gamma_changes(bh):
    """The operator tables are cached per degree for the last penalty: calls
    that alternate gamma = k(k+1) and 2 k(k+1) each match the context built
    with that gamma."""
    d, k, L = 2, 3, 4
    n = (k * 2 ** L - 1) ** d
    x = torch.tensor(workload.vector_uniform(n, 9), dtype=torch.float64, device="cuda")
    refs = {}
    for g in (12.0, 24.0):
        with bh.Context(bh.default_params(d, k, L, gamma=g)) as ctx:
            refs[g] = torch.empty_like(x)
            ctx.apply_A(L, x, refs[g])
    for g in (12.0, 24.0, 12.0, 0.0):
        got = torch.full_like(x, float("nan"))
        bh.apply_A_noalloc(d, k, L, g, x, got)
        torch.cuda.synchronize()
        assert relerr(got, refs[g if g > 0 else 12.0]) <= TOL, g


def test_noalloc_rejects_sizes_beyond_the_static_maximum(bh):
    d, k, L = 2, 4, 9            # 2047^2 = 4.19 M unknowns > 2.80 M
    n = (k * 2 ** L - 1) ** d
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(bh.BiharmError) as e:
        bh.apply_A_noalloc(d, k, L, 0.0, x, y)
    assert "maximum" in str(e.value)
    # the array is still usable after the rejected call
    xs = torch.tensor(workload.vector_uniform((2 * 8 - 1) ** 2, 3), dtype=torch.float64, device="cuda")
    ys, ref = torch.empty_like(xs), torch.empty_like(xs)
    bh.apply_A_noalloc(2, 2, 3, 0.0, xs, ys)
    with bh.Context(bh.default_params(2, 2, 3)) as ctx:
        ctx.apply_A(3, xs, ref)
    torch.cuda.synchronize()
    assert relerr(ys, ref) <= TOL
