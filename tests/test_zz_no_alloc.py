"""cg_chordal_test_dense_noalloc: the dense test for callers that cannot
allocate device memory when they call (plugins in hosts that own the device
memory, allocator-free latency loops, callers without a context).  It must
return exactly what cg_chordal_test_dense returns; it is called twice in a row
on different graphs, so a stale witness key or order from the previous call
would show.  This file sorts last so that a stop-at-first-failure run has run
every other test before it."""
import ctypes

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


def _rows(g):
    return torch.from_numpy(np.ascontiguousarray(g.rows).view(np.int32)).to(DEV)


def _existing(ctx, g, rows):
    res = torch.full((4,), -9, dtype=torch.int32, device=DEV)
    order = torch.full((max(g.n, 1),), -9, dtype=torch.int32, device=DEV)
    d = B.cg_dense(g.n, g.words, rows.data_ptr())
    st = B.cg_chordal_test_dense(ctx.handle, ctypes.byref(d), res.data_ptr(), order.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    assert st == B.CG_OK, B.cg_last_error_string()
    torch.cuda.synchronize()
    return res.cpu().tolist(), order[:g.n].cpu().tolist()


def _noalloc(g, rows, with_order=True):
    res = torch.full((4,), -9, dtype=torch.int32, device=DEV)
    order = torch.full((max(g.n, 1),), -9, dtype=torch.int32, device=DEV) if with_order else None
    d = B.cg_dense(g.n, g.words, rows.data_ptr())
    st = B.cg_chordal_test_dense_noalloc(ctypes.byref(d), res.data_ptr(), None if order is None else order.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
    assert st == B.CG_OK, B.cg_last_error_string()
    torch.cuda.synchronize()
    return res.cpu().tolist(), (order[:g.n].cpu().tolist() if order is not None else None)


def test_noalloc_matches_existing_entry_two_calls_in_a_row():
    small, planted, _ = gg.small_dense_pair()
    big = gg.subtree_dense(16384, 562, 99)
    big_nc, _ = gg.close_cycles_dense(big, 3, 7)
    with B.Context(0) as ctx:
        for first, second in ((planted, small), (big, big_nc), (gg.cycle(5), gg.cycle(5))):
            rf, rs = _rows(first), _rows(second)
            want1, want2 = _existing(ctx, first, rf), _existing(ctx, second, rs)
            got1 = _noalloc(first, rf)
            got2 = _noalloc(second, rs)
            assert got1 == want1
            assert got2 == want2
        # order buffer taken from the fixed scratch when the caller passes none
        rf = _rows(planted)
        assert _noalloc(planted, rf, with_order=False)[0] == _existing(ctx, planted, rf)[0]


def test_noalloc_rejects_graphs_over_the_limit():
    big = torch.zeros((16385, 513), dtype=torch.int32, device=DEV)
    res = torch.empty(4, dtype=torch.int32, device=DEV)
    d = B.cg_dense(16385, 513, big.data_ptr())
    st = B.cg_chordal_test_dense_noalloc(ctypes.byref(d), res.data_ptr(), None, None)
    assert st == B.CG_EINVAL
    assert b"16384" in B.cg_last_error_string()


def test_noalloc_matches_the_oracle_including_empty_and_tiny_graphs():
    """Also against the oracle directly (not only the context entry), for the
    empty graph, one vertex, a ragged row length and a full-size graph."""
    g16, h16, _ = gg.large_dense_pair()
    for g in (gg.empty_dense(0), gg.empty_dense(1), gg.cycle(4), gg.random_dense(33, 0.3, 5), g16, h16):
        rows = _rows(g)
        want = oracle.chordal_test(g)
        res, order = _noalloc(g, rows)
        assert tuple(res) == want.witness
        assert order == [int(x) for x in want.order]


def test_noalloc_allocates_no_device_memory():
    """After a first call (which resolves the scratch array's address and may
    load the library's device code), further calls leave the device's free
    memory unchanged: the entry point allocates nothing."""
    g = gg.subtree_dense(16384, 562, 5)
    rows = _rows(g)
    res = torch.empty(4, dtype=torch.int32, device=DEV)
    order = torch.empty(g.n, dtype=torch.int32, device=DEV)
    d = B.cg_dense(g.n, g.words, rows.data_ptr())
    stream = torch.cuda.current_stream().cuda_stream
    assert B.cg_chordal_test_dense_noalloc(ctypes.byref(d), res.data_ptr(), order.data_ptr(), stream) == B.CG_OK
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        assert B.cg_chordal_test_dense_noalloc(ctypes.byref(d), res.data_ptr(), None, stream) == B.CG_OK
        assert B.cg_chordal_test_dense_noalloc(ctypes.byref(d), res.data_ptr(), order.data_ptr(), stream) == B.CG_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    assert tuple(res.cpu().tolist()) == oracle.chordal_test(g).witness
