"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, never against the oracle itself.

* verdict: brute-force chordless-cycle enumeration on every labelled graph with
  N <= 6 and on seeded samples with N = 7..9 (chordal <=> no chordless cycle of
  length >= 4, Section 1 / Section 3.1); Maximum Cardinality Search as an
  independent verdict (Theorem 5.2); known families;
* order: LexBFS by explicit labels (Section 4.1) and the plain O(N^2)
  class-splitting form (Section 4.2) give the identical order; property LB
  holds for every triple (Lemma 4.2);
* witness: the certificate (u, p in LN(v), p rightmost, u not adjacent to p),
  v is the first vertex whose left neighbourhood is not a clique (Section 5.3),
  u is the smallest id of the violating set;
* hand-derived small cases.
"""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import reference as R


# ----------------------------------------------------------------- helpers

def adj_from_mask_graph(n, masks):
    return [[j for j in range(n) if masks[i] >> j & 1] for i in range(n)]


def has_chordless_cycle(n, masks) -> bool:
    """Brute force: some vertex set S with |S| >= 4 induces a cycle, i.e. every
    vertex of S has exactly two neighbours inside S and S is connected."""
    for S in _SUBSETS[n]:
        ok = True
        s = S
        while s:
            v = (s & -s).bit_length() - 1
            s &= s - 1
            if bin(masks[v] & S).count("1") != 2:
                ok = False
                break
        if not ok:
            continue
        start = S & -S
        seen, frontier = start, start
        while frontier:
            nxt = 0
            f = frontier
            while f:
                v = (f & -f).bit_length() - 1
                f &= f - 1
                nxt |= masks[v] & S
            frontier = nxt & ~seen
            seen |= nxt
        if seen == S:
            return True
    return False


_SUBSETS = {n: [S for S in range(1 << n) if bin(S).count("1") >= 4] for n in range(10)}


def csr_of(n, adj):
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum([len(a) for a in adj])
    col = np.array([v for a in adj for v in sorted(a)], dtype=np.int32)
    return gg.CsrGraph(n, rp, col)


def masks_of(n, edges):
    m = [0] * n
    for a, b in edges:
        m[a] |= 1 << b
        m[b] |= 1 << a
    return m


def random_graph_adj(n, p, seed):
    return gg.adjacency_lists(gg.random_dense(n, p, seed))


def witness_by_definition(adj, order):
    """(v*, p*, u*) straight from the definitions: the first order index whose
    left neighbourhood is not a clique, its rightmost left neighbour, and the
    smallest earlier neighbour other than p that is not adjacent to p."""
    i = R.first_non_simplicial(adj, order)
    if i is None:
        return (1, -1, -1, -1)
    pos = {v: k for k, v in enumerate(order)}
    v = order[i]
    left = [u for u in adj[v] if pos[u] < i]
    p = max(left, key=lambda u: pos[u])
    bad = [u for u in left if u != p and u not in set(adj[p])]
    return (0, v, p, min(bad))


# ----------------------------------------------------------------- verdict

@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 6])
def test_verdict_exhaustive_small(n):
    pairs = list(itertools.combinations(range(n), 2))
    count = 0
    for bits in range(1 << len(pairs)):
        edges = [pairs[k] for k in range(len(pairs)) if bits >> k & 1]
        masks = masks_of(n, edges)
        adj = adj_from_mask_graph(n, masks)
        res = oracle.chordal_test(csr_of(n, adj))
        assert res.chordal == (0 if has_chordless_cycle(n, masks) else 1), (n, edges)
        count += 1
    assert count == 1 << len(pairs)


@pytest.mark.parametrize("n", [7, 8, 9])
def test_verdict_sampled(n):
    rs = gg.rng_stream(1000 + n, 6000)
    for t in range(0, 6000, 2):
        p = 0.15 + 0.7 * (int(rs[t]) % 1000) / 1000.0
        g = gg.random_dense(n, p, int(rs[t + 1]))
        masks = [int(g.rows[i, 0]) for i in range(n)]
        res = oracle.chordal_test(g)
        assert res.chordal == (0 if has_chordless_cycle(n, masks) else 1)


def test_verdict_matches_mcs_theorem():
    """Theorem 5.2: the MCS order is a PEO iff the graph is chordal."""
    rs = gg.rng_stream(77, 400)
    seen = {0: 0, 1: 0}
    for t in range(200):
        n = 5 + int(rs[2 * t]) % 60
        if t % 3 == 0:
            g = gg.subtree_dense(n, max(2, n // 3), int(rs[2 * t + 1]))
        elif t % 3 == 1:
            g = gg.interval_graph(n, int(rs[2 * t + 1]), span=4 * n, max_len=6)
        else:
            g = gg.random_dense(n, 0.1 + (t % 7) / 10.0, int(rs[2 * t + 1]))
        adj = gg.adjacency_lists(g)
        mcs_chordal = R.first_non_simplicial(adj, R.mcs(adj)) is None
        res = oracle.chordal_test(g)
        assert res.chordal == int(mcs_chordal)
        seen[res.chordal] += 1
    assert seen[0] > 20 and seen[1] > 20


@pytest.mark.parametrize("k", list(range(4, 41)) + [100, 1000])
def test_cycles_not_chordal(k):
    assert oracle.chordal_test(gg.cycle(k)).chordal == 0


@pytest.mark.parametrize("n", [1, 2, 3, 10, 33, 64, 200])
def test_cliques_chordal(n):
    res = oracle.chordal_test(gg.clique(n))
    assert res.chordal == 1
    # in a clique every label is equal at every step: the order is 0..n-1
    assert res.order.tolist() == list(range(n))


@pytest.mark.parametrize("seed", range(6))
def test_trees_paths_stars_chordal(seed):
    for g in (gg.random_tree(300, seed), gg.path(97), gg.star(65)):
        assert oracle.chordal_test(g).chordal == 1


@pytest.mark.parametrize("seed", range(6))
def test_interval_and_subtree_graphs_chordal(seed):
    assert oracle.chordal_test(gg.interval_graph(400, seed)).chordal == 1
    assert oracle.chordal_test(gg.subtree_dense(700, 90, seed)).chordal == 1


def test_disconnected_and_empty():
    assert oracle.chordal_test(gg.empty_dense(0)).chordal == 1
    r = oracle.chordal_test(gg.empty_dense(5))
    assert r.chordal == 1 and r.order.tolist() == [0, 1, 2, 3, 4]
    # two C_4 components far apart in id space
    edges = [(0, 1), (1, 2), (2, 3), (3, 0), (10, 11), (11, 12), (12, 13), (13, 10)]
    g = gg.dense_from_edges(14, edges)
    r = oracle.chordal_test(g)
    assert r.chordal == 0 and (r.v, r.p, r.u) == (2, 3, 1)


# ----------------------------------------------------------------- order

@pytest.mark.parametrize("n,p", [(10, 0.3), (50, 0.1), (50, 0.5), (120, 0.05), (200, 0.2), (300, 0.03)])
def test_order_equals_explicit_labels(n, p):
    for s in range(3):
        adj = random_graph_adj(n, p, 31 * n + s)
        order = oracle.lexbfs(csr_of(n, adj)).tolist()
        assert order == R.lexbfs_labels(adj)
        assert order == R.lexbfs_classes(adj)


@pytest.mark.parametrize("seed", range(4))
def test_order_equals_explicit_labels_chordal_families(seed):
    for g in (gg.subtree_dense(150, 40, seed), gg.interval_graph(150, seed, span=300, max_len=20)):
        adj = gg.adjacency_lists(g)
        assert oracle.lexbfs(g).tolist() == R.lexbfs_labels(adj)


@pytest.mark.parametrize("n,p", [(40, 0.2), (90, 0.08), (150, 0.3), (150, 0.03)])
def test_order_has_lb_property(n, p):
    adj = random_graph_adj(n, p, 5 * n)
    order = oracle.lexbfs(csr_of(n, adj)).tolist()
    assert R.lb_violations(adj, order) == 0


def test_lb_checker_rejects_non_lexbfs_orders():
    """The LB pin itself must be able to fail: a plain BFS order that is not a
    LexBFS order, and the reverse of a LexBFS order, are rejected."""
    # path 0-1-2-3 plus 0-4, 4-3? build a graph where BFS order differs
    adj = random_graph_adj(60, 0.1, 9)
    order = oracle.lexbfs(csr_of(60, adj)).tolist()
    assert R.lb_violations(adj, order[::-1]) > 0
    swapped = order[:]
    for i in range(1, 59):
        swapped = order[:]
        swapped[i], swapped[i + 1] = swapped[i + 1], swapped[i]
        if R.lb_violations(adj, swapped) > 0:
            break
    else:
        pytest.fail("no adjacent swap broke property LB")


def test_order_min_id_tie_break():
    """Among the unnumbered vertices with the largest label the lowest id is
    taken: checked step by step with explicit labels."""
    for seed in range(5):
        n = 80
        adj = random_graph_adj(n, 0.07, 100 + seed)
        order = oracle.lexbfs(csr_of(n, adj)).tolist()
        label = {v: [] for v in range(n)}
        numbered = set()
        for i, x in enumerate(order, start=1):
            best = max(label[v] for v in range(n) if v not in numbered)
            ties = [v for v in range(n) if v not in numbered and label[v] == best]
            assert x == min(ties)
            numbered.add(x)
            for y in adj[x]:
                if y not in numbered:
                    label[y].append(n - i)


# ----------------------------------------------------------------- witness

@pytest.mark.parametrize("n,p", [(30, 0.3), (80, 0.1), (150, 0.05), (300, 0.02)])
def test_witness_is_canonical(n, p):
    for s in range(4):
        adj = random_graph_adj(n, p, 7 * n + s)
        res = oracle.chordal_test(csr_of(n, adj))
        order = res.order.tolist()
        assert res.witness == witness_by_definition(adj, order)
        if res.chordal == 0:
            pos = {v: k for k, v in enumerate(order)}
            v, pp, u = res.v, res.p, res.u
            assert pos[u] < pos[v] and pos[pp] < pos[v] and u != pp
            assert pp in adj[v] and u in adj[v] and u not in adj[pp]
            assert pos[pp] == max(pos[w] for w in adj[v] if pos[w] < pos[v])


def test_parent_array_by_definition():
    adj = random_graph_adj(120, 0.08, 4242)
    res = oracle.chordal_test(csr_of(120, adj))
    pos = res.pos
    for v in range(120):
        left = [u for u in adj[v] if pos[u] < pos[v]]
        want = max(left, key=lambda u: pos[u]) if left else -1
        assert res.parent[v] == want


def test_peo_check_of_arbitrary_order():
    """The check itself (Section 5.2) on orders that are not LexBFS orders: its
    verdict equals the definition of a perfect elimination order."""
    rs = gg.rng_stream(555, 100)
    for t in range(50):
        n = 20 + int(rs[t]) % 40
        g = gg.subtree_dense(n, max(2, n // 4), int(rs[50 + t]))
        adj = gg.adjacency_lists(g)
        perm = np.random.Generator(np.random.PCG64(t)).permutation(n).tolist()
        res = oracle.peo_check(g, perm)
        assert res.witness == witness_by_definition(adj, perm)


# ----------------------------------------------------------------- hand-derived

def test_hand_c4():
    """C_4 with edges 01, 12, 23, 30.  Step 1 numbers 0 and splits {1,2,3} into
    {1,3},{2}.  Step 2 numbers 1; its unnumbered neighbour 2 is alone in its
    class, so the classes are {3},{2}.  Order 0,1,3,2.  Vertex 2 has LN = {1,3},
    p = 3, and 1 is not adjacent to 3: witness (2, 3, 1)."""
    r = oracle.chordal_test(gg.cycle(4))
    assert r.order.tolist() == [0, 1, 3, 2]
    assert r.witness == (0, 2, 3, 1)


def test_hand_c5():
    """C_5 (01,12,23,34,40): classes after 0: {1,4},{2,3}; after 1: {4},{2},{3};
    order 0,1,4,2,3.  Vertex 3 has LN = {2,4}, p = 2, 4 not adjacent to 2."""
    r = oracle.chordal_test(gg.cycle(5))
    assert r.order.tolist() == [0, 1, 4, 2, 3]
    assert r.witness == (0, 3, 2, 4)


def test_hand_path_and_diamond():
    r = oracle.chordal_test(gg.path(4))
    assert r.order.tolist() == [0, 1, 2, 3] and r.parent.tolist() == [-1, 0, 1, 2] and r.chordal == 1
    # K_4 minus edge 03: after 0 the classes are {1,2},{3}; order 0,1,2,3
    r = oracle.chordal_test(gg.dense_from_edges(4, [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3)]))
    assert r.order.tolist() == [0, 1, 2, 3] and r.chordal == 1 and r.parent.tolist() == [-1, 0, 1, 2]


def test_planted_cycle_and_closing_edges_not_chordal():
    for s in range(5):
        g = gg.subtree_dense(300, 60, 900 + s)
        assert oracle.chordal_test(g).chordal == 1
        h, _ = gg.plant_cycle(g, 5 + s % 4, 17 + s)
        assert oracle.chordal_test(h).chordal == 0
        h2, pairs = gg.close_cycles_dense(g, 1 + s, 23 + s)
        assert len(pairs) == 1 + s and oracle.chordal_test(h2).chordal == 0


# ----------------------------------------------------------------- MCS (Section 5.1)

@pytest.mark.parametrize("n,p", [(10, 0.3), (60, 0.1), (150, 0.05), (200, 0.4)])
def test_mcs_order_equals_definition(n, p):
    """The heap-based C MCS equals the plain definition (largest count of
    numbered neighbours, lowest id among equals)."""
    for s in range(3):
        adj = random_graph_adj(n, p, 71 * n + s)
        assert oracle.mcs(csr_of(n, adj)).tolist() == R.mcs(adj)


def test_mcs_verdict_theorem_5_2():
    """Theorem 5.2: the MCS order is a PEO iff the graph is chordal (the
    verdict is checked against the LexBFS test and against brute force)."""
    rs = gg.rng_stream(808, 300)
    for t in range(150):
        n = 4 + int(rs[t]) % 60
        if t % 2:
            g = gg.subtree_dense(n, max(2, n // 3), int(rs[150 + t]))
        else:
            g = gg.random_dense(n, 0.05 + (t % 9) / 10.0, int(rs[150 + t]))
        assert oracle.chordal_test_mcs(g).chordal == oracle.chordal_test(g).chordal
    for n in range(4, 8):
        for s in range(200):
            g = gg.random_dense(n, 0.5, 9000 + 17 * n + s)
            masks = [int(g.rows[i, 0]) for i in range(n)]
            assert oracle.chordal_test_mcs(g).chordal == (0 if has_chordless_cycle(n, masks) else 1)


def test_mcs_hand_c4_and_clique():
    """C_4: 0 first; its neighbours 1 and 3 get count 1, 1 wins (lower id);
    then 2 (count 1 from 1) ties with 3 (count 1), 2 wins; order 0,1,2,3.
    A clique is visited in id order."""
    assert oracle.mcs(gg.cycle(4)).tolist() == [0, 1, 2, 3]
    assert oracle.mcs(gg.clique(9)).tolist() == list(range(9))


# ----------------------------------------------------------------- multi-sweep LexBFS (tie-break rank, start)

def _prefer(rank, start):
    pref = list(int(r) for r in rank)
    if start >= 0:
        pref[start] = -1
    return pref


@pytest.mark.parametrize("n,p", [(12, 0.3), (60, 0.1), (120, 0.05), (150, 0.4)])
def test_tiebreak_order_equals_explicit_labels(n, p):
    """A caller-given tie-break: the refinement started from the class ordered
    by rank equals explicit-label LexBFS whose ties go to the lowest rank, with
    the start vertex first."""
    for s in range(3):
        adj = random_graph_adj(n, p, 31 * n + s)
        rank = np.random.default_rng(n + s).permutation(n).astype(np.int32)
        start = -1 if s == 0 else (7 * s) % n
        g = csr_of(n, adj)
        got = oracle.lexbfs_tiebreak(g, rank, start).tolist()
        assert got == R.lexbfs_labels(adj, _prefer(rank, start))
        assert R.lb_violations(adj, got) == 0
        if start >= 0:
            assert got[0] == start
        # the dense entry agrees with the CSR one
        assert oracle.lexbfs_tiebreak(gg.csr_to_dense(g), rank, start).tolist() == got


def test_tiebreak_identity_and_relabelling():
    """rank = id gives the plain LexBFS; a LexBFS with tie-break rank equals
    the plain LexBFS of the graph relabelled by rank, mapped back."""
    g = gg.random_dense(200, 0.08, 44)
    assert np.array_equal(oracle.lexbfs_tiebreak(g), oracle.lexbfs(g))
    assert np.array_equal(oracle.lexbfs_tiebreak(g, np.arange(200, dtype=np.int32)), oracle.lexbfs(g))
    rank = np.random.default_rng(5).permutation(200).astype(np.int32)
    h = gg.relabel_dense(g, rank)            # vertex v becomes rank[v]
    inv = np.empty(200, np.int64)
    inv[rank] = np.arange(200)
    assert np.array_equal(oracle.lexbfs_tiebreak(g, rank), inv[oracle.lexbfs(h)])


def test_tiebreak_rejects_non_permutation():
    g = gg.random_dense(20, 0.2, 1)
    rank = np.arange(20, dtype=np.int32)
    rank[3] = 4
    with pytest.raises(ValueError):
        oracle.lexbfs_tiebreak(g, rank)


def test_lexbfs_plus_sweeps():
    """LexBFS+ (ties to the vertex latest in the previous sweep): its first
    vertex is the previous sweep's last one; every sweep is a LexBFS order
    (property LB), and on chordal graphs a perfect elimination order
    (Theorem 5.1), so its last vertex is simplicial."""
    for seed in range(4):
        for g in (gg.subtree_dense(90, 30, 600 + seed), gg.interval_graph(80, 700 + seed),
                  gg.random_dense(70, 0.15, 800 + seed)):
            adj = gg.adjacency_lists(g)
            prev = oracle.lexbfs(g)
            for _ in range(3):
                plus = oracle.lexbfs_plus(g, prev)
                assert plus[0] == prev[-1]
                assert R.lb_violations(adj, plus.tolist()) == 0
                res = oracle.peo_check(g, plus)
                assert res.chordal == oracle.chordal_test(g).chordal
                if res.chordal:
                    last = int(plus[-1])
                    nb = adj[last]
                    assert all(b in set(adj[a]) for a in nb for b in nb if a != b)
                prev = plus
