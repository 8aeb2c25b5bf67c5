"""GPU parity of the dense path against the CPU oracle: the LexBFS order, the
parent array, the verdict and the witness must be identical (integer work:
bit-exact)."""
import glob
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402
from paper_1508_06329_gb300 import binding as B  # noqa: E402

from gpu_util import DEV, run_dense, to_dev  # noqa: E402

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctx():
    from paper_1508_06329_gb300 import build
    build.build()
    c = B.Context(0)
    yield c
    c.close()


def assert_parity(ctx, g, label=""):
    want = oracle.chordal_test(g)
    got_w, got_o = run_dense(ctx, g)
    assert np.array_equal(got_o, want.order), f"order differs {label} n={g.n}"
    assert got_w == want.witness, f"witness {got_w} != {want.witness} {label}"
    return want


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))))
def test_golden(ctx, path):
    rec = json.load(open(path))
    g = gg.dense_from_edges(rec["n"], rec["edges"])
    got_w, got_o = run_dense(ctx, g)
    assert got_o.tolist() == rec["order"] and list(got_w) == rec["witness"]


@pytest.mark.parametrize("k", [4, 5, 6, 31, 32, 33, 100, 1000])
def test_cycles(ctx, k):
    assert_parity(ctx, gg.cycle(k))


@pytest.mark.parametrize("n", [1, 2, 3, 32, 33, 200, 1025])
def test_cliques_paths_stars(ctx, n):
    for g in (gg.clique(n), gg.path(n), gg.star(n)):
        assert_parity(ctx, g)


def test_empty_graphs(ctx):
    for n in (0, 1, 5, 64, 1000):
        assert_parity(ctx, gg.empty_dense(n))


@pytest.mark.parametrize("n", [2, 31, 32, 33, 63, 64, 65, 100, 511, 512, 513, 1000, 1023, 1024, 1025, 1280,
                               1300, 2047, 2048, 2049, 4097, 8191])
def test_random_sizes(ctx, n):
    for s, p in enumerate((0.02, 0.1, 0.5)):
        assert_parity(ctx, gg.random_dense(n, p, 1000 * n + s), f"gnp p={p}")


@pytest.mark.parametrize("n", [50, 300, 1000, 1500, 3000, 6000])
def test_chordal_families(ctx, n):
    for s in range(2):
        g = gg.subtree_dense(n, max(2, n // 4), 7 * n + s)
        assert assert_parity(ctx, g).chordal == 1
        h, _ = gg.plant_cycle(g, 5 + s, 3 * n + s)
        assert assert_parity(ctx, h).chordal == 0
        h2, _ = gg.close_cycles_dense(g, 2 + s, 5 * n + s)
        assert assert_parity(ctx, h2).chordal == 0
    assert_parity(ctx, gg.interval_graph(min(n, 1500), n))
    assert_parity(ctx, gg.random_tree(n, n))


def test_disconnected(ctx):
    a = gg.subtree_dense(300, 50, 1)
    b = gg.cycle(9)
    edges = [(i, j) for i in range(300) for j in gg.adjacency_lists(a)[i] if i < j]
    edges += [(300 + 2 * i, 300 + 2 * ((i + 1) % 9)) for i in range(9)]  # cycle on even ids
    g = gg.dense_from_edges(320, edges)
    assert_parity(ctx, g)


@pytest.mark.parametrize("threads", [128, 256, 512, 1024])
def test_cta_sizes(threads):
    with B.Context(0, threads_override=threads) as c:
        for n in (100, 1000, 3000):
            assert_parity(c, gg.subtree_dense(n, n // 5, n + threads))
            assert_parity(c, gg.random_dense(n, 0.05, n + threads))


def test_padding_words_and_garbage_padding_bits(ctx):
    g = gg.subtree_dense(70, 15, 3)
    wide = gg.empty_dense(70, words=9)          # 3 words needed, 6 extra
    wide.rows[:, :3] = g.rows
    wide.rows[:, 3:] = 0xDEADBEEF                # words past ceil(n/32) are never read
    dirty = wide.copy()
    dirty.rows[:, 2] |= np.uint32(0xFFFFFFC0)    # bits 70..95 (padding of the last word) are masked
    want = oracle.chordal_test(g)
    for h in (wide, dirty):
        got_w, got_o = run_dense(ctx, h)
        assert np.array_equal(got_o, want.order) and got_w == want.witness


def test_padding_words_of_staged_rows(ctx):
    """Rows padded to a multiple of 4 words take the staged check, whose bulk
    copies bring in the padding word after ceil(n/32) and the padding bits of
    the last word: both must be ignored."""
    for n, t in ((70, 15), (300, 60)):
        g = gg.subtree_dense(n, t, n)
        for h in (g, gg.plant_cycle(g, 6, n)[0]):
            wn = (n + 31) // 32
            wide = gg.empty_dense(n, words=(wn + 3) // 4 * 4 + 4)
            wide.rows[:, :wn] = h.rows
            wide.rows[:, wn:] = 0xDEADBEEF
            if n % 32:
                wide.rows[:, wn - 1] |= np.uint32((0xFFFFFFFF << (n % 32)) & 0xFFFFFFFF)
            want = oracle.chordal_test(h)
            got_w, got_o = run_dense(ctx, wide)
            assert np.array_equal(got_o, want.order) and got_w == want.witness


@pytest.mark.parametrize("n", [49152, 49153])
def test_staged_check_size_limit(ctx, n):
    """The largest graph whose check stages its rows in shared memory, and the
    first one checked with the masks built from pos."""
    g = gg.subtree_dense(n, n // 2, n)
    assert assert_parity(ctx, g).chordal == 1
    h, _ = gg.plant_cycle(g, 7, n)
    assert assert_parity(ctx, h).chordal == 0


def test_small_dense_workload(ctx):
    g, h, _ = gg.small_dense_pair()
    assert assert_parity(ctx, g).chordal == 1
    assert assert_parity(ctx, h).chordal == 0


def test_large_dense_workload_full_size(ctx):
    """N=16,384, density ~0.1 (the benchmark workload): full order and witness."""
    g, h, _ = gg.large_dense_pair()
    assert assert_parity(ctx, g).chordal == 1
    assert assert_parity(ctx, h).chordal == 0


def test_wide_ids_beyond_shared_memory(ctx):
    """n > 16,384 keeps part of the state in the workspace (the split layouts)."""
    for n, t in ((16385, 2000), (20000, 3000), (40000, 20000)):
        g = gg.subtree_dense(n, t, n)
        assert_parity(ctx, g)
        h, _ = gg.plant_cycle(g, 6, n)
        assert_parity(ctx, h)


def test_lexbfs_order_entry_and_pos(ctx):
    g = gg.subtree_dense(900, 120, 77)
    rows = to_dev(g)
    order = torch.empty(900, dtype=torch.int32, device=DEV)
    pos = torch.empty(900, dtype=torch.int32, device=DEV)
    B.lexbfs_order_dense(ctx, rows, 900, order, pos)
    torch.cuda.synchronize()
    want = oracle.lexbfs(g)
    assert np.array_equal(order.cpu().numpy(), want)
    p = np.empty(900, np.int32)
    p[want] = np.arange(900)
    assert np.array_equal(pos.cpu().numpy(), p)


def test_peo_check_of_given_orders(ctx):
    """The check alone, on orders that are not LexBFS orders (witness and the
    full parent array)."""
    rs = np.random.Generator(np.random.PCG64(11))
    for n in (10, 33, 200, 1000, 2500):
        g = gg.subtree_dense(n, max(2, n // 6), n)
        for order in (rs.permutation(n), oracle.lexbfs(g)):
            order = order.astype(np.int32)
            want = oracle.peo_check(g, order)
            res = torch.empty(4, dtype=torch.int32, device=DEV)
            parent = torch.empty(n, dtype=torch.int32, device=DEV)
            B.peo_check_dense(ctx, to_dev(g), n, torch.from_numpy(order).to(DEV), res, parent)
            torch.cuda.synchronize()
            assert tuple(res.cpu().tolist()) == want.witness
            assert np.array_equal(parent.cpu().numpy(), want.parent)


@pytest.mark.parametrize("n", [8191, 8192, 8193, 16384, 20000])
def test_peo_check_multi_chunk(ctx, n):
    """Rows longer than one register chunk; random orders put parents far
    back (the mask binary search), LexBFS orders close (the probes)."""
    rs = np.random.Generator(np.random.PCG64(n))
    g = gg.random_dense(n, 0.02, n + 1)
    h = gg.subtree_dense(n, n // 8, n + 2)
    for G, order in ((g, rs.permutation(n)), (h, rs.permutation(n)), (h, oracle.lexbfs(h))):
        order = order.astype(np.int32)
        want = oracle.peo_check(G, order)
        res = torch.empty(4, dtype=torch.int32, device=DEV)
        parent = torch.empty(n, dtype=torch.int32, device=DEV)
        B.peo_check_dense(ctx, to_dev(G), n, torch.from_numpy(order).to(DEV), res, parent)
        torch.cuda.synchronize()
        assert tuple(res.cpu().tolist()) == want.witness
        assert np.array_equal(parent.cpu().numpy(), want.parent)


def test_peo_check_validates_order():
    c = B.Context(0, validate=1)
    try:
        g = gg.random_dense(100, 0.1, 3)
        rows = to_dev(g)
        res = torch.empty(4, dtype=torch.int32, device=DEV)
        bad = np.arange(100, dtype=np.int32)
        bad[5] = 6
        with pytest.raises(Exception):
            B.peo_check_dense(c, rows, 100, torch.from_numpy(bad).to(DEV), res)
        good = np.random.Generator(np.random.PCG64(1)).permutation(100).astype(np.int32)
        B.peo_check_dense(c, rows, 100, torch.from_numpy(good).to(DEV), res)
        torch.cuda.synchronize()
        assert tuple(res.cpu().tolist()) == oracle.peo_check(g, good).witness
    finally:
        c.close()


def test_host_entry(ctx):
    g, h, _ = gg.small_dense_pair()
    for G in (g, h, gg.empty_dense(0), gg.cycle(4)):
        order = np.full(max(G.n, 1), -1, np.int32)
        got = B.chordal_test_dense_host(ctx, G.rows.view(np.int32), G.n, order)
        want = oracle.chordal_test(G)
        assert got == want.witness and np.array_equal(order[:G.n], want.order)


def test_argument_errors(ctx):
    res = torch.empty(4, dtype=torch.int32, device=DEV)
    bad = B.cg_dense(-1, 0, 0)
    assert B.cg_chordal_test_dense(ctx.handle, B.ctypes.byref(bad), res.data_ptr(), None, None) == B.CG_EINVAL
    bad = B.cg_dense(100, 3, to_dev(gg.cycle(100)).data_ptr())   # words_per_row < ceil(100/32)
    assert B.cg_chordal_test_dense(ctx.handle, B.ctypes.byref(bad), res.data_ptr(), None, None) == B.CG_EINVAL
    bad = B.cg_dense(200000, 6250, 0)
    assert B.cg_chordal_test_dense(ctx.handle, B.ctypes.byref(bad), res.data_ptr(), None, None) == B.CG_EINVAL


@pytest.mark.parametrize("n", [37920, 37921, 56312, 56313, 65520, 65521])
def test_variant_size_limits(ctx, n):
    """The largest graph of each split-state layout (16-bit ids: moved counts
    and children in shared memory up to 37,920 vertices, moved counts up to
    56,312, arrival bits up to 65,520), the first one of the next, and the
    first one of the 32-bit-id variant; sparse graphs keep the oracle fast."""
    g = gg.random_tree(n, n)
    assert assert_parity(ctx, g).chordal == 1
    h = g.copy()
    # close one cycle: 0 - ... - far vertex
    h.rows[0, (n - 1) >> 5] |= np.uint32(1 << ((n - 1) & 31))
    h.rows[n - 1, 0] |= np.uint32(1)
    assert_parity(ctx, h)


@pytest.mark.gpu
def test_step_floor_probe():
    """The latency-floor probe returns positive, ordered times and rejects bad
    arguments with CG_EINVAL."""
    with B.Context(0) as ctx:
        f = B.step_floor(ctx, threads=256, iters=2048, chain_bytes=1 << 20, loads=4096)
        assert f["chain_bytes"] == 1 << 20
        assert 0 < f["barrier_pair_ns"] < 10_000
        assert 0 < f["load_ns"] < 100_000
        with pytest.raises(B.ChordalError):
            B.step_floor(ctx, threads=100)
        with pytest.raises(B.ChordalError):
            B.step_floor(ctx, chain_bytes=64)
