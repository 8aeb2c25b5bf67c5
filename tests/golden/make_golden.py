"""Writes the small fixtures in this folder.  Calls only ``oracle/`` (and the
input generators); run from the repository root:

    python tests/golden/make_golden.py

Each fixture stores the graph as an edge list and the oracle's LexBFS order,
parent array and verdict/witness.  Hand-derived cases (C_4, C_5, P_4) are
pinned separately in tests/test_oracle_pins.py.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def edges_of(g):
    adj = gg.adjacency_lists(g)
    return [[a, b] for a in range(g.n) for b in adj[a] if a < b]


def fixtures():
    yield "c6", "cycle C_6", gg.cycle(6)
    yield "k7", "clique K_7", gg.clique(7)
    yield "subtree_n64", "subtree model N=64, 20-node tree, seed 11", gg.subtree_dense(64, 20, 11)
    g = gg.subtree_dense(100, 30, 12)
    yield "planted_c6_n100", "subtree model N=100 with planted C_6, seeds 12/13", gg.plant_cycle(g, 6, 13)[0]
    yield "closed_n90", "subtree model N=90 plus 3 cycle-closing edges, seeds 14/15", gg.close_cycles_dense(
        gg.subtree_dense(90, 25, 14), 3, 15)[0]
    yield "gnp_n70", "G(70, 0.12), seed 16", gg.random_dense(70, 0.12, 16)
    yield "ragged_n33", "subtree model N=33 (one bit past a word), seed 17", gg.subtree_dense(33, 9, 17)


def main():
    for name, desc, g in fixtures():
        r = oracle.chordal_test(g)
        rec = {
            "description": desc,
            "source": "oracle (tests/golden/make_golden.py)",
            "n": g.n,
            "edges": edges_of(g),
            "order": r.order.tolist(),
            "parent": r.parent.tolist(),
            "witness": list(r.witness),
        }
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(rec, f, separators=(",", ":"))
            f.write("\n")


if __name__ == "__main__":
    main()
