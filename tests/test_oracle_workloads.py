"""The oracle on the benchmark workloads and on the stored fixtures."""
import glob
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))))
def test_golden_fixture(path):
    rec = json.load(open(path))
    g = gg.dense_from_edges(rec["n"], rec["edges"])
    r = oracle.chordal_test(g)
    assert r.order.tolist() == rec["order"]
    assert r.parent.tolist() == rec["parent"]
    assert list(r.witness) == rec["witness"]
    # same answer through the CSR entry point
    r2 = oracle.chordal_test(gg.dense_to_csr(g))
    assert r2.order.tolist() == rec["order"] and list(r2.witness) == rec["witness"]


def test_small_dense_workload_verdicts():
    g, h, info = gg.small_dense_pair()
    assert oracle.chordal_test(g).chordal == 1
    r = oracle.chordal_test(h)
    assert r.chordal == 0
    # the witness lies on the planted cycle or next to it: v and u both
    # adjacent in h, u not adjacent to p
    assert r.u in set(gg.adjacency_lists(h)[r.v])


@pytest.mark.slow
def test_large_dense_workload_verdicts():
    g, h, _ = gg.large_dense_pair()
    assert oracle.chordal_test(g).chordal == 1
    assert oracle.chordal_test(h).chordal == 0


@pytest.mark.slow
def test_sparse_workload_verdicts():
    g, h, info = gg.sparse_csr_pair()
    assert g.n == 1 << 20 and 10_000_000 <= g.num_edges() <= 12_000_000
    assert oracle.chordal_test(g).chordal == 1
    assert oracle.chordal_test(h).chordal == 0
