"""Input generators: layout invariants and the workload recipes (no method
arithmetic here; verdicts on generated graphs are checked with the oracle in
test_oracle_pins.py and test_oracle_workloads.py)."""
import numpy as np
import pytest

import graphgen as gg


def check_dense_layout(g: gg.DenseGraph):
    n, w = g.n, g.words
    assert g.rows.dtype == np.uint32 and g.rows.shape == (n, w)
    bits = np.unpackbits(g.rows.view(np.uint8).reshape(n, -1), axis=1, bitorder="little")
    assert not bits[:, n:].any(), "padding bits must be zero"
    a = bits[:, :n]
    assert not np.diag(a).any(), "zero diagonal"
    assert (a == a.T).all(), "symmetric"


def check_csr_layout(c: gg.CsrGraph):
    assert c.row_ptr.dtype == np.int64 and c.col.dtype == np.int32
    assert c.row_ptr[0] == 0 and c.row_ptr[-1] == c.nnz
    for v in range(c.n):
        r = c.col[c.row_ptr[v]:c.row_ptr[v + 1]]
        assert (np.diff(r) > 0).all() and not (r == v).any()


@pytest.mark.parametrize("n,t", [(1, 1), (31, 5), (32, 5), (33, 5), (100, 10), (257, 40)])
def test_subtree_layout(n, t):
    check_dense_layout(gg.subtree_dense(n, t, 3))


def test_deterministic():
    a = gg.subtree_dense(300, 50, 99)
    b = gg.subtree_dense(300, 50, 99)
    c = gg.subtree_dense(300, 50, 100)
    assert (a.rows == b.rows).all() and not (a.rows == c.rows).all()
    assert gg.rng_stream(5, 4).tolist() == gg.rng_stream(5, 4).tolist()


def test_conversions_roundtrip():
    g = gg.subtree_dense(130, 20, 7)
    c = gg.dense_to_csr(g)
    check_csr_layout(c)
    assert (gg.csr_to_dense(c).rows == g.rows).all()
    perm = np.random.Generator(np.random.PCG64(1)).permutation(130)
    h = gg.relabel_dense(g, perm)
    check_dense_layout(h)
    assert h.num_edges() == g.num_edges()


def test_plant_cycle_is_induced_cycle():
    g = gg.subtree_dense(200, 30, 5)
    for k in range(4, 9):
        h, verts = gg.plant_cycle(g, k, 40 + k)
        check_dense_layout(h)
        sub = [[bool(h.rows[a, b >> 5] >> (b & 31) & 1) for b in verts] for a in verts]
        for i in range(k):
            for j in range(k):
                want = (j - i) % k in (1, k - 1)
                assert sub[i][j] == want


def test_peo_csr_layout_and_size():
    c = gg.peo_csr(5000, 3)
    check_csr_layout(c)
    # clique sizes U{1..20}: about 10.5 edges per vertex
    assert 9.0 < c.num_edges() / 5000 < 11.5


def test_small_dense_recipe():
    g, h, info = gg.small_dense_pair()
    assert g.n == 1000 and g.words == 32 and info["tree_nodes"] == 500
    assert 5 <= info["k"] <= 8
    check_dense_layout(g)
    check_dense_layout(h)


@pytest.mark.slow
def test_large_dense_recipe_density():
    g, h, info = gg.large_dense_pair()
    assert g.n == 16384 and g.words == 512 and g.nbytes == 32 << 20
    assert 0.09 <= g.density() <= 0.11
    assert 1 <= info["r"] <= 10 and len(info["pairs"]) == info["r"]


def test_batch_recipe():
    graphs = gg.batch_dense(64, seed=123)
    ns = [g.n for g in graphs]
    assert min(ns) >= 16 and max(ns) <= 2048
    for g in graphs[:8]:
        check_dense_layout(g)
