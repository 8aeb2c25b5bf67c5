"""The rules the dense kernels rely on, replayed on the CPU against the oracle
(host logic; no GPU, no library call).

* The search's exact parents (Section 5.2's p(v) recorded during the LexBFS
  of Section 4.2): a pivot adjacent to the previous pivot has it as parent; a
  pivot taken from the top class that lost no member shares the previous
  pivot's parent (the two had the same label); a pivot taken from the class
  after an emptied top class gets that class's last moving pivot (the pivot
  at which its members last moved: they all share one label, so one latest
  numbered neighbour).  Replayed with explicit classes in the kernels' order
  (new class before its parent class, a class that moves whole keeps its
  place), the order equals the oracle's LexBFS and every parent equals the
  definition (rightmost earlier neighbour).
* The staged check's decomposition: for position i in group b = i / 32,
  LN_v = (row_v & E_b) + (row_v & {vertices at positions 32 b .. i - 1}),
  where E_b holds the vertices numbered before position 32 b; with p excluded
  and the lowest bad id taken over both parts, the first violating position
  gives exactly the oracle's witness, for units of 16 and of 32 positions.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle


def _adj(g):
    return [set(nb) for nb in gg.adjacency_lists(g)]


def replay_exact_parents(g):
    """LexBFS by class splitting with the kernels' parent rule; returns (order, parent by position)."""
    n = g.n
    adj = _adj(g)
    classes = [[0, list(range(n))]]   # top first: [id, members in id order]
    next_id, cpar = 1, {0: -1}
    x, par_x = 0, -1
    order, par = [], []
    for i in range(n):
        order.append(x)
        par.append(par_x)
        f = classes[0]
        g_cls = classes[1] if len(classes) > 1 else None
        cpar_g = cpar[g_cls[0]] if g_cls else None   # read before this step's moves
        f[1].remove(x)
        new, moved_of = [], {}
        for c in classes:
            m = [y for y in c[1] if y in adj[x]]
            if not m:
                new.append(c)
                continue
            if len(m) == len(c[1]):      # moves whole: keeps id and place
                cpar[c[0]] = x
                new.append(c)
                moved_of[id(c)] = c
            else:                         # split: the moved part goes in front under a new id
                cn = [next_id, m]
                cpar[next_id] = x
                next_id += 1
                c[1] = [y for y in c[1] if y not in adj[x]]
                new += [cn, c]
                moved_of[id(c)] = cn
        classes = [c for c in new if c[1]]
        if i == n - 1:
            break
        if id(f) in moved_of:                      # mode 0: a moved member of f
            x, par_x = min(moved_of[id(f)][1]), x
        elif f[1]:                                 # mode 1: f lost no member
            x = min(f[1])                          # par_x unchanged: same label as x
        elif g_cls is not None and id(g_cls) in moved_of:
            x, par_x = min(moved_of[id(g_cls)][1]), x
        else:                                      # mode 2: the class after the emptied f
            x, par_x = min(g_cls[1]), cpar_g
    return np.array(order), par


def parents_by_definition(g, order):
    adj = _adj(g)
    pos = {v: i for i, v in enumerate(order)}
    out = []
    for i, v in enumerate(order):
        earlier = [u for u in adj[v] if pos[u] < i]
        out.append(max(earlier, key=lambda u: pos[u]) if earlier else -1)
    return out


def _graphs():
    out = []
    for s in range(60):
        n = 2 + (s * 7) % 70
        if s % 3 == 0:
            out.append(gg.subtree_dense(n, max(2, n // 4), 100 + s))
        elif s % 3 == 1:
            out.append(gg.random_dense(n, (0.05, 0.2, 0.5)[s % 3], 200 + s))
        else:
            out.append(gg.plant_cycle(gg.subtree_dense(max(n, 12), max(3, n // 3), 300 + s), 5, s)[0])
    return out + [gg.clique(9), gg.cycle(6), gg.path(7), gg.star(8), gg.empty_dense(5)]


@pytest.mark.parametrize("k", range(0, 65, 8))
def test_exact_parent_rule_matches_definition(k):
    for g in _graphs()[k:k + 8]:
        order, par = replay_exact_parents(g)
        assert np.array_equal(order, oracle.lexbfs(g)), g.n
        assert par == parents_by_definition(g, order), g.n


def staged_check_model(g, order, parent, unit):
    """(chordal, v, p, u) from the staged decomposition with units of `unit` positions."""
    adj = _adj(g)
    n = g.n
    for s0 in range(0, n, unit):          # units in order: the first violating position wins
        b = s0 // 32
        E = set(order[:32 * b])            # numbered before position 32 b
        for j in range(min(unit, n - s0)):
            i = s0 + j
            v, p = order[i], parent[i]
            if p < 0:
                continue
            group = set(order[32 * b:i])    # the group's own earlier positions
            bad = [u for u in adj[v] if (u in E or u in group) and u != p and u not in adj[p]]
            if bad:
                return (0, v, p, min(bad))
    return (1, -1, -1, -1)


@pytest.mark.parametrize("unit", [16, 32])
def test_staged_decomposition_matches_witness(unit):
    graphs = _graphs() + [gg.subtree_dense(300, 40, 7), gg.plant_cycle(gg.subtree_dense(300, 40, 8), 6, 3)[0]]
    for g in graphs:
        want = oracle.chordal_test(g)
        order = list(want.order)
        parent = parents_by_definition(g, order)
        assert staged_check_model(g, order, parent, unit) == want.witness, g.n
