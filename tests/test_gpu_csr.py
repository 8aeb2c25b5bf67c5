"""GPU parity of the CSR path (sparse graphs) against the CPU oracle: order,
verdict and witness bit-exact, plus the parent array of the check."""
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

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def ctx():
    c = B.Context(0)
    yield c
    c.close()


def dev_csr(c: gg.CsrGraph):
    rp = torch.from_numpy(np.ascontiguousarray(c.row_ptr, dtype=np.int64)).to(DEV)
    col = torch.from_numpy(np.ascontiguousarray(c.col, dtype=np.int32)).to(DEV) if c.nnz else \
        torch.zeros(1, dtype=torch.int32, device=DEV)[:0]
    return rp, col


def run_csr(ctx, c: gg.CsrGraph):
    rp, col = dev_csr(c)
    res = torch.full((4,), -7, dtype=torch.int32, device=DEV)
    order = torch.full((max(c.n, 1),), -7, dtype=torch.int32, device=DEV)
    B.chordal_test_csr(ctx, rp, col, c.n, res, order)
    torch.cuda.synchronize()
    return tuple(res.cpu().tolist()), order[:c.n].cpu().numpy()


def assert_parity(ctx, c, label=""):
    want = oracle.chordal_test(c)
    got_w, got_o = run_csr(ctx, c)
    assert np.array_equal(got_o, want.order), f"order differs {label} n={c.n}"
    assert got_w == want.witness, f"{got_w} != {want.witness} {label}"
    return want


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))))
def test_golden(ctx, path):
    rec = json.load(open(path))
    c = gg.dense_to_csr(gg.dense_from_edges(rec["n"], rec["edges"]))
    got_w, got_o = run_csr(ctx, c)
    assert got_o.tolist() == rec["order"] and list(got_w) == rec["witness"]


def test_families(ctx):
    for g in (gg.cycle(4), gg.cycle(5), gg.cycle(77), gg.clique(33), gg.clique(100), gg.path(50), gg.star(70),
              gg.empty_dense(0), gg.empty_dense(1), gg.empty_dense(40), gg.random_tree(500, 3)):
        assert_parity(ctx, gg.dense_to_csr(g))


@pytest.mark.parametrize("n,p", [(40, 0.2), (100, 0.05), (300, 0.3), (1000, 0.01), (1000, 0.1), (2000, 0.05)])
def test_random(ctx, n, p):
    for s in range(2):
        assert_parity(ctx, gg.dense_to_csr(gg.random_dense(n, p, n + s)))


@pytest.mark.parametrize("n,p", [(20, 0.15), (30, 0.1), (40, 0.08), (60, 0.05), (80, 0.04), (120, 0.03)])
def test_sparse_small_random(ctx, n, p):
    """Average degree 2-3: most steps find the top class holding only the
    pivot and take the next pivot from the untouched class after it, and in
    many of these graphs a step also splits the class after that one (the
    case where the carried next class must be replaced by the new part)."""
    for s in range(30):
        assert_parity(ctx, gg.dense_to_csr(gg.random_dense(n, p, s)), f"seed {s}")


def test_long_rows_multi_chunk(ctx):
    """Rows far longer than 32 neighbours exercise the per-class carries."""
    for n, p in ((200, 0.6), (500, 0.3)):
        assert_parity(ctx, gg.dense_to_csr(gg.random_dense(n, p, 3 * n)))
    sub = gg.subtree_dense(1500, 60, 5)          # dense chordal: degrees in the hundreds
    assert assert_parity(ctx, gg.dense_to_csr(sub)).chordal == 1
    h, _ = gg.plant_cycle(sub, 7, 5)
    assert assert_parity(ctx, gg.dense_to_csr(h)).chordal == 0


@pytest.mark.parametrize("leaves", [32, 33, 4095, 4096, 4097, 9000])
def test_long_row_sort_sizes(ctx, leaves):
    """A hub row at the boundaries of the long-row step: 32 neighbours (one
    warp), 33 (the CTA), 4,096 keys (the last shared-memory sort) and longer
    rows (the tiled sort on the workspace), with a few extra edges among the
    leaves so that the hub's neighbours fall into several classes."""
    n = leaves + 1
    eu, ev = [0] * leaves, list(range(1, n))
    rng = np.random.Generator(np.random.PCG64(leaves))
    for _ in range(leaves // 3):
        a, b = sorted(rng.choice(np.arange(1, n), 2, replace=False).tolist())
        eu.append(a)
        ev.append(b)
    g = gg.csr_from_edges(n, np.array(eu, np.int64), np.array(ev, np.int64))
    assert_parity(ctx, g)
    # the same hub numbered late: its row is long when most of it is unnumbered
    perm = rng.permutation(n)
    assert_parity(ctx, gg.relabel_csr(g, perm))


@pytest.mark.parametrize("n", [10, 1000, 20000, 200000])
def test_peo_construction(ctx, n):
    g = gg.peo_csr(n, n + 1)
    assert assert_parity(ctx, g).chordal == 1
    h, pairs = gg.close_cycles_csr(g, 3, n + 2)
    r = assert_parity(ctx, h)
    if pairs:                      # tiny graphs may admit no cycle-closing edge
        assert r.chordal == 0


def test_sparse_workload_full_size(ctx):
    """N = 2^20, M = 11.0M (the sparse workload): full order and witness."""
    g, h, _ = gg.sparse_csr_pair()
    assert assert_parity(ctx, g).chordal == 1
    assert assert_parity(ctx, h).chordal == 0


def test_peo_check_csr_given_orders(ctx):
    rs = np.random.Generator(np.random.PCG64(5))
    for n in (30, 500, 5000):
        g = gg.peo_csr(n, n)
        for order in (rs.permutation(n), oracle.lexbfs(g)):
            order = order.astype(np.int32)
            want = oracle.peo_check(g, order)
            rp, col = dev_csr(g)
            res = torch.empty(4, dtype=torch.int32, device=DEV)
            parent = torch.empty(n, dtype=torch.int32, device=DEV)
            B.peo_check_csr(ctx, rp, col, n, torch.from_numpy(order).to(DEV), res, parent)
            torch.cuda.synchronize()
            assert tuple(res.cpu().tolist()) == want.witness
            assert np.array_equal(parent.cpu().numpy(), want.parent)


def test_lexbfs_order_csr_and_host_entry(ctx):
    g = gg.peo_csr(3000, 17)
    want = oracle.chordal_test(g)
    rp, col = dev_csr(g)
    order = torch.empty(3000, dtype=torch.int32, device=DEV)
    pos = torch.empty(3000, dtype=torch.int32, device=DEV)
    B.lexbfs_order_csr(ctx, rp, col, 3000, order, pos)
    torch.cuda.synchronize()
    assert np.array_equal(order.cpu().numpy(), want.order)
    assert np.array_equal(pos.cpu().numpy(), want.pos)
    ho = np.full(3000, -1, np.int32)
    assert B.chordal_test_csr_host(ctx, g.row_ptr, g.col, 3000, ho) == want.witness
    assert np.array_equal(ho, want.order)


def test_validation_rejects_malformed_csr():
    with B.Context(0, validate=1) as vctx:
        good = gg.peo_csr(200, 1)
        res = torch.empty(4, dtype=torch.int32, device=DEV)
        rp, col = dev_csr(good)
        B.chordal_test_csr(vctx, rp, col, 200, res)          # accepted
        bad_col = good.col.copy()
        r0 = slice(good.row_ptr[5], good.row_ptr[6])
        bad_col[r0] = bad_col[r0][::-1]                     # unsorted row
        for cc in (bad_col,):
            rp2, col2 = dev_csr(gg.CsrGraph(200, good.row_ptr, cc))
            with pytest.raises(B.ChordalError) as e:
                B.chordal_test_csr(vctx, rp2, col2, 200, res)
            assert e.value.status == B.CG_EINVAL
        # one-directional edge
        asym = gg.csr_from_edges(4, np.array([0, 1, 2]), np.array([1, 2, 3]))
        one_way = gg.CsrGraph(4, np.array([0, 1, 3, 5, 5], np.int64), np.array([1, 0, 2, 1, 3], np.int32))
        rp3, col3 = dev_csr(one_way)
        with pytest.raises(B.ChordalError):
            B.chordal_test_csr(vctx, rp3, col3, 4, res)
        rp4, col4 = dev_csr(asym)
        B.chordal_test_csr(vctx, rp4, col4, 4, res)
