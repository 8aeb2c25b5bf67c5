"""GPU parity of one multi-sweep LexBFS sweep (a caller-given tie-break rank
or LexBFS+ of a previous sweep, optional start vertex) against the CPU
oracle: order and pos bit-exact."""
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


def sweep(ctx, rows, n, kind, tb, start):
    order = torch.full((max(n, 1),), -7, dtype=torch.int32, device=DEV)
    pos = torch.full((max(n, 1),), -7, dtype=torch.int32, device=DEV)
    tbd = None if tb is None else torch.from_numpy(np.ascontiguousarray(tb, dtype=np.int32)).to(DEV)
    B.lexbfs_sweep_dense(ctx, rows, n, order, pos, kind, tbd, start)
    torch.cuda.synchronize()
    o, p = order[:n].cpu().numpy(), pos[:n].cpu().numpy()
    inv = np.empty(n, np.int32)
    inv[o] = np.arange(n)
    assert np.array_equal(p, inv)
    return o


@pytest.mark.parametrize("n", [1, 2, 33, 100, 1000, 2049, 5000])
def test_sweep_rank_and_start(ctx, n):
    for s, g in enumerate((gg.random_dense(n, 0.1, n), gg.subtree_dense(n, max(2, n // 4), n + 3))):
        rows = to_dev(g)
        rank = np.random.default_rng(n + s).permutation(n).astype(np.int32)
        for start in (-1, 0, n // 2, n - 1):
            got = sweep(ctx, rows, n, B.TIE_RANK, rank, start)
            assert np.array_equal(got, oracle.lexbfs_tiebreak(g, rank, start)), (n, s, start)
            got = sweep(ctx, rows, n, B.TIE_ID, None, start)
            assert np.array_equal(got, oracle.lexbfs_tiebreak(g, None, start)), (n, s, start)


@pytest.mark.parametrize("n", [64, 700, 3000])
def test_lexbfs_plus_chain(ctx, n):
    """Three LexBFS+ sweeps after the plain one, each fed the previous
    sweep's order (the same on both sides, checked at every sweep)."""
    g = gg.interval_graph(n, n + 11) if n < 3000 else gg.random_dense(n, 0.05, 17)
    rows = to_dev(g)
    prev = oracle.lexbfs(g)
    got_prev = sweep(ctx, rows, n, B.TIE_ID, None, -1)
    assert np.array_equal(got_prev, prev)
    for _ in range(3):
        want = oracle.lexbfs_plus(g, prev)
        got = sweep(ctx, rows, n, B.TIE_LAST_IN, got_prev, -1)
        assert np.array_equal(got, want)
        prev, got_prev = want, got


def test_sweep_large(ctx):
    g, h, _ = gg.large_dense_pair()
    rank = np.random.default_rng(3).permutation(g.n).astype(np.int32)
    for x in (g, h):
        got = sweep(ctx, to_dev(x), x.n, B.TIE_RANK, rank, 12345)
        assert np.array_equal(got, oracle.lexbfs_tiebreak(x, rank, 12345))
    t = gg.random_tree(40000, 5)               # relabelled copy in the workspace, global-state LexBFS
    rank = np.random.default_rng(4).permutation(t.n).astype(np.int32)
    got = sweep(ctx, to_dev(t), t.n, B.TIE_RANK, rank, -1)
    assert np.array_equal(got, oracle.lexbfs_tiebreak(t, rank, -1))


def test_sweep_rejects_bad_input():
    c = B.Context(0, validate=1)
    try:
        g = gg.random_dense(50, 0.2, 2)
        rows = to_dev(g)
        bad = np.arange(50, dtype=np.int32)
        bad[7] = 8
        with pytest.raises(Exception):
            sweep(c, rows, 50, B.TIE_RANK, bad, -1)
        with pytest.raises(Exception):
            sweep(c, rows, 50, B.TIE_RANK, np.arange(50, dtype=np.int32), 50)    # start out of range
        with pytest.raises(Exception):
            sweep(c, rows, 50, 7, np.arange(50, dtype=np.int32), -1)             # unknown kind
        ok = sweep(c, rows, 50, B.TIE_LAST_IN, np.arange(50, dtype=np.int32)[::-1].copy(), -1)
        assert np.array_equal(ok, oracle.lexbfs_tiebreak(g, np.arange(50, dtype=np.int32), -1))
    finally:
        c.close()


# ----------------------------------------------------------------- CSR sweeps

def sweep_csr(ctx, g, kind, tb, start):
    n = g.n
    rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr, dtype=np.int64)).to(DEV)
    col = torch.from_numpy(np.ascontiguousarray(g.col, dtype=np.int32)).to(DEV)
    if col.numel() == 0:
        col = torch.zeros(1, dtype=torch.int32, device=DEV)[:0]
    order = torch.full((max(n, 1),), -7, dtype=torch.int32, device=DEV)
    pos = torch.full((max(n, 1),), -7, dtype=torch.int32, device=DEV)
    tbd = None if tb is None else torch.from_numpy(np.ascontiguousarray(tb, dtype=np.int32)).to(DEV)
    B.lexbfs_sweep_csr(ctx, rp, col, n, order, pos, kind, tbd, start)
    torch.cuda.synchronize()
    o, p = order[:n].cpu().numpy(), pos[:n].cpu().numpy()
    inv = np.empty(n, np.int32)
    inv[o] = np.arange(n)
    assert np.array_equal(p, inv)
    return o


def hub_graph(n, seed):
    """Random sparse graph plus a vertex adjacent to everything: rows of every
    size class (<= 32, <= 4096 and longer) in the relabelled copy."""
    g = gg.random_dense(n, 8.0 / n, seed)
    rows = g.rows.copy()
    hub = n // 3
    for v in range(n):
        if v != hub:
            rows[hub, v >> 5] |= np.uint32(1 << (v & 31))
            rows[v, hub >> 5] |= np.uint32(1 << (hub & 31))
    return gg.dense_to_csr(gg.DenseGraph(n, rows))


@pytest.mark.parametrize("n", [1, 2, 40, 1000, 9000])
def test_sweep_csr_rank_and_start(ctx, n):
    graphs = [gg.dense_to_csr(gg.random_dense(n, 0.05, n)), gg.dense_to_csr(gg.subtree_dense(n, max(2, n // 4), n + 1))]
    if n >= 1000:
        graphs.append(hub_graph(n, n + 2))
    for s, g in enumerate(graphs):
        rank = np.random.default_rng(n + s).permutation(n).astype(np.int32)
        for start in (-1, n // 2):
            got = sweep_csr(ctx, g, B.TIE_RANK, rank, start)
            assert np.array_equal(got, oracle.lexbfs_tiebreak(g, rank, start)), (n, s, start)


def test_sweep_csr_plus_chain_large(ctx):
    """LexBFS+ sweeps on the N = 65,536 reversed-PEO CSR graph (a hub with a
    few thousand neighbours), each fed the previous sweep."""
    g, _, _ = gg.sparse_csr_pair(n=1 << 16)
    prev = oracle.lexbfs(g)
    got_prev = prev.astype(np.int32)
    for _ in range(2):
        want = oracle.lexbfs_plus(g, prev)
        got = sweep_csr(ctx, g, B.TIE_LAST_IN, got_prev, -1)
        assert np.array_equal(got, want)
        prev, got_prev = want, got
