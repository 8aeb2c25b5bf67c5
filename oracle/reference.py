"""Slow pure-Python restatements used to pin the C oracle (small graphs only).

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  Each function follows one
passage of the paper and is written for reading, not speed.  Graphs are given
as adjacency lists ``adj[v]`` (any iterable of neighbour ids).
"""
from __future__ import annotations

import numpy as np


def lexbfs_labels(adj, prefer=None) -> list[int]:
    """LexBFS with explicit string labels (Section 4.1).

    Every vertex starts with the empty label.  In step i (1-based) the vertex x
    with the lexicographically largest label is numbered, and the number n - i
    is appended to the label of each unnumbered neighbour of x (the printed
    update names label_x; it is the neighbour's label that grows).  Labels are
    compared as sequences, a proper prefix being smaller; ties go to the
    lowest vertex id, or to the lowest prefer[v] when prefer is given.
    """
    n = len(adj)
    nbrs = [set(a) for a in adj]
    label: list[list[int]] = [[] for _ in range(n)]
    numbered = [False] * n
    order = []
    for i in range(1, n + 1):
        x = max((v for v in range(n) if not numbered[v]),
                key=lambda v: (label[v], -(v if prefer is None else prefer[v])))
        numbered[x] = True
        order.append(x)
        for y in nbrs[x]:
            if not numbered[y]:
                label[y].append(n - i)
    return order


def lexbfs_classes(adj) -> list[int]:
    """LexBFS by partition refinement in its plain O(N^2) form (Section 4.2).

    The partition is an ordered list of classes, each a list kept in id order;
    every step takes the first vertex of the first class, then replaces each
    class C by C ∩ N_x followed by C \\ N_x, dropping empty parts.
    """
    n = len(adj)
    nbrs = [set(a) for a in adj]
    classes = [list(range(n))] if n else []
    order = []
    while classes:
        x = classes[0].pop(0)
        order.append(x)
        refined = []
        for c in classes:
            inside = [y for y in c if y in nbrs[x]]
            outside = [y for y in c if y not in nbrs[x]]
            if inside:
                refined.append(inside)
            if outside:
                refined.append(outside)
        classes = refined
    return order


def mcs(adj) -> list[int]:
    """Maximum Cardinality Search (Section 5.1): the label of a vertex is the
    number of its already-numbered neighbours; the largest label is taken
    next, ties to the lowest id."""
    n = len(adj)
    nbrs = [set(a) for a in adj]
    label = [0] * n
    numbered = [False] * n
    order = []
    for _ in range(n):
        x = max((v for v in range(n) if not numbered[v]), key=lambda v: (label[v], -v))
        numbered[x] = True
        order.append(x)
        for y in nbrs[x]:
            if not numbered[y]:
                label[y] += 1
    return order


def first_non_simplicial(adj, order) -> int | None:
    """Definition of a perfect elimination order (Section 3.1): each v_i must be
    simplicial among v_1..v_i, i.e. LN(v_i) is a clique.  Returns the first
    order index whose left neighbourhood is not a clique, or None."""
    nbrs = [set(a) for a in adj]
    pos = {v: i for i, v in enumerate(order)}
    for i, v in enumerate(order):
        left = [u for u in nbrs[v] if pos[u] < i]
        for a in range(len(left)):
            for b in range(a + 1, len(left)):
                if left[b] not in nbrs[left[a]]:
                    return i
    return None


def lb_violations(adj, order) -> int:
    """Count triples breaking property LB (Section 4.1): for positions
    a < b < c with ac ∈ E and ab ∉ E there must be d < a with db ∈ E and
    dc ∉ E.  An order is a LexBFS order iff the count is zero (Lemma 4.2)."""
    n = len(adj)
    if n < 3:
        return 0
    pos = np.empty(n, dtype=np.int64)
    pos[np.asarray(order)] = np.arange(n)
    A = np.zeros((n, n), dtype=bool)
    for v in range(n):
        for u in adj[v]:
            A[pos[v], pos[u]] = True
    # D[b, c] = smallest d with db ∈ E and dc ∉ E (n if none)
    cand = A[:, :, None] & ~A[:, None, :]                  # [d, b, c]
    any_d = cand.any(axis=0)
    D = np.where(any_d, cand.argmax(axis=0), n)            # [b, c]
    idx = np.arange(n)
    a = idx[:, None, None]
    b = idx[None, :, None]
    c = idx[None, None, :]
    trip = (a < b) & (b < c) & A[:, None, :] & ~A[:, :, None]   # [a, b, c]: ac ∈ E, ab ∉ E
    bad = trip & ~(D[None, :, :] < a)
    return int(bad.sum())
