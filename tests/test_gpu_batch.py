"""Batched form: every problem's result equals its own single-context solve
(same iterations, same solution to 1e-9 relative), in any mix."""
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
        assert abs(rr - rr1) <= 1e-6 * max(rr1, 1e-300) + 1e-14


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
