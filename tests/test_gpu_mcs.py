"""GPU parity of the MCS ordering (Section 5.1) and the test built on it
(Theorem 5.2) against the CPU oracle: order and witness bit-exact."""
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


def check(ctx, g):
    rows = to_dev(g)
    res = torch.full((4,), -7, dtype=torch.int32, device=DEV)
    order = torch.full((max(g.n, 1),), -7, dtype=torch.int32, device=DEV)
    B.chordal_test_mcs_dense(ctx, rows, g.n, res, order)
    torch.cuda.synchronize()
    want = oracle.chordal_test_mcs(g)
    assert np.array_equal(order[:g.n].cpu().numpy(), want.order), g.n
    assert tuple(res.cpu().tolist()) == want.witness
    # Theorem 5.2: the same verdict as the LexBFS test
    assert want.chordal == oracle.chordal_test(g).chordal
    return want


@pytest.mark.parametrize("n", [1, 2, 5, 31, 32, 33, 100, 1000, 4096, 4097, 8000])
def test_mcs_random_and_chordal(ctx, n):
    check(ctx, gg.random_dense(n, 0.1, n))
    g = gg.subtree_dense(n, max(2, n // 5), n + 1)
    assert check(ctx, g).chordal == 1
    if n >= 8:
        check(ctx, gg.plant_cycle(g, 6, n)[0])


def test_mcs_families(ctx):
    for g in (gg.cycle(4), gg.cycle(9), gg.clique(300), gg.path(200), gg.star(100), gg.empty_dense(70),
              gg.random_tree(2000, 4), gg.interval_graph(800, 5)):
        check(ctx, g)


def test_mcs_large(ctx):
    g, h, _ = gg.large_dense_pair()
    assert check(ctx, g).chordal == 1
    assert check(ctx, h).chordal == 0
    t = gg.random_tree(40000, 8)               # 1024 threads x 2 words per thread
    check(ctx, t)


def test_mcs_order_entry(ctx):
    g = gg.subtree_dense(700, 100, 3)
    order = torch.empty(700, dtype=torch.int32, device=DEV)
    pos = torch.empty(700, dtype=torch.int32, device=DEV)
    B.mcs_order_dense(ctx, to_dev(g), 700, order, pos)
    torch.cuda.synchronize()
    want = oracle.mcs(g)
    assert np.array_equal(order.cpu().numpy(), want)
    p = np.empty(700, np.int32)
    p[want] = np.arange(700)
    assert np.array_equal(pos.cpu().numpy(), p)
