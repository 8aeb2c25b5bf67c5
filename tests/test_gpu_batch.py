"""GPU parity of the batched dense path (many graphs per launch)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402
from paper_1508_06329_gb300 import binding as B  # noqa: E402

from gpu_util import DEV, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = B.Context(0)
    yield c
    c.close()


def run_batch(ctx, graphs, offsets=None):
    tens = [to_dev(g) for g in graphs]
    res = torch.full((len(graphs), 4), -7, dtype=torch.int32, device=DEV)
    total = sum(g.n for g in graphs) if offsets is None else int(max(o + g.n for o, g in zip(offsets, graphs)))
    orders = torch.full((max(total, 1),), -7, dtype=torch.int32, device=DEV)
    B.chordal_test_batch(ctx, [(t, g.n) for t, g in zip(tens, graphs)], res, orders, offsets)
    torch.cuda.synchronize()
    return res.cpu().numpy(), orders.cpu().numpy()


def check(graphs, res, orders, offsets=None):
    off = 0
    for k, g in enumerate(graphs):
        want = oracle.chordal_test(g)
        o = off if offsets is None else offsets[k]
        assert tuple(res[k].tolist()) == want.witness, k
        assert np.array_equal(orders[o:o + g.n], want.order), k
        off += g.n


def test_batch_mixed_sizes(ctx):
    graphs = gg.batch_dense(96, seed=5)
    res, orders = run_batch(ctx, graphs)
    check(graphs, res, orders)


def test_batch_with_empty_and_tiny(ctx):
    graphs = [gg.empty_dense(0), gg.empty_dense(1), gg.cycle(4), gg.clique(3), gg.empty_dense(0),
              gg.subtree_dense(50, 10, 1)]
    res, orders = run_batch(ctx, graphs)
    check(graphs, res, orders)


def test_batch_order_offsets(ctx):
    graphs = [gg.subtree_dense(40, 8, 2), gg.cycle(6), gg.subtree_dense(33, 5, 3)]
    offsets = [100, 3, 50]
    res, orders = run_batch(ctx, graphs, offsets)
    check(graphs, res, orders, offsets)


def test_batch_large_pair(ctx):
    g, h, _ = gg.large_dense_pair()
    res, orders = run_batch(ctx, [g, h])
    check([g, h], res, orders)


def test_batch_workload_full(ctx):
    """4,096 graphs, N log-uniform in [16, 2048] (the batched workload)."""
    graphs = gg.batch_dense(4096)
    res, orders = run_batch(ctx, graphs)
    check(graphs, res, orders)


def test_batch_mixed_with_large_graphs(ctx):
    """Size buckets 0..8 (one-CTA kernel) and 9 (n > 4096: LexBFS CTA + grid check)
    in one call, results in input order."""
    graphs = [gg.subtree_dense(5000, 700, 1), gg.cycle(5), gg.subtree_dense(300, 50, 2),
              gg.plant_cycle(gg.subtree_dense(6000, 900, 3), 6, 3)[0], gg.empty_dense(0), gg.clique(17),
              gg.subtree_dense(4096, 600, 4), gg.subtree_dense(4097, 600, 5)]
    res, orders = run_batch(ctx, graphs)
    check(graphs, res, orders)


def test_batch_plan_replays(ctx):
    graphs = gg.batch_dense(200, seed=77) + [gg.subtree_dense(5000, 800, 9)]
    tens = [to_dev(g) for g in graphs]
    res = torch.full((len(graphs), 4), -7, dtype=torch.int32, device=DEV)
    orders = torch.full((sum(g.n for g in graphs),), -7, dtype=torch.int32, device=DEV)
    plan = B.BatchPlan(ctx, [(t, g.n) for t, g in zip(tens, graphs)], res, orders)
    for _ in range(2):
        res.fill_(-7)
        orders.fill_(-7)
        plan.run()
        torch.cuda.synchronize()
        check(graphs, res.cpu().numpy(), orders.cpu().numpy())
    # inputs may change between runs: planted cycles appear in the results
    h, _ = gg.plant_cycle(graphs[0], 5, 1)
    tens[0].copy_(to_dev(h))
    plan.run()
    torch.cuda.synchronize()
    assert tuple(res[0].cpu().tolist()) == oracle.chordal_test(h).witness
    plan.close()


def test_autotune_keeps_results(ctx):
    graphs = gg.batch_dense(300, seed=31)
    table = B.batch_autotune(ctx, [(to_dev(g), g.n) for g in graphs])
    assert len(table) == 9 and all(t in (0, 64, 128, 256, 512) for t in table)
    res, orders = run_batch(ctx, graphs)
    check(graphs, res, orders)
    B.autotune_set(ctx, [0] * 9)
    assert B.autotune_get(ctx) == [0] * 9


def test_batch_host_entry_matches_oracle(ctx):
    """cg_chordal_test_batch_host: host rows in, host results and orders out (copies inside the library)."""
    graphs = gg.batch_dense(64, seed=11) + [gg.empty_dense(0), gg.cycle(5), gg.subtree_dense(5000, 900, 4)]
    host_rows = [(torch.from_numpy(np.ascontiguousarray(g.rows).view(np.int32)).pin_memory(), g.n) for g in graphs]
    res = torch.full((len(graphs), 4), -7, dtype=torch.int32).pin_memory()
    orders = torch.full((sum(g.n for g in graphs),), -7, dtype=torch.int32).pin_memory()
    B.chordal_test_batch_host(ctx, host_rows, res, orders)
    check(graphs, res.numpy(), orders.numpy())
    # results only, from pageable numpy rows, twice in a row (the workspace is reused)
    for _ in range(2):
        res2 = np.full((len(graphs), 4), -7, dtype=np.int32)
        B.chordal_test_batch_host(ctx, [(g.rows, g.n) for g in graphs], res2)
        for k, g in enumerate(graphs):
            assert tuple(res2[k].tolist()) == oracle.chordal_test(g).witness, k


def test_batch_host_entry_full_size_pair(ctx):
    g, h, _ = gg.large_dense_pair()
    res = np.full((2, 4), -7, dtype=np.int32)
    B.chordal_test_batch_host(ctx, [(g.rows, g.n), (h.rows, h.n)], res)
    assert [tuple(r) for r in res.tolist()] == [oracle.chordal_test(g).witness, oracle.chordal_test(h).witness]


def test_batch_host_descriptors_reused_with_new_contents(ctx):
    """A HostBatch built once over pinned buffers: each call copies the buffers'
    current contents, so overwriting the rows between calls changes the results."""
    a = gg.batch_dense(40, seed=41)
    b = [gg.random_dense(g.n, 0.3, 7 * g.n + k) for k, g in enumerate(a)]   # same sizes, other graphs
    bufs = [torch.from_numpy(np.ascontiguousarray(g.rows).view(np.int32).copy()).pin_memory() for g in a]
    batch = B.HostBatch([(t, g.n) for t, g in zip(bufs, a)])
    res = torch.full((len(a), 4), -7, dtype=torch.int32).pin_memory()
    for graphs in (a, b, a):
        for t, g in zip(bufs, graphs):
            t.copy_(torch.from_numpy(np.ascontiguousarray(g.rows).view(np.int32)))
        B.chordal_test_batch_host(ctx, batch, res)
        for k, g in enumerate(graphs):
            assert tuple(res[k].tolist()) == oracle.chordal_test(g).witness, k
