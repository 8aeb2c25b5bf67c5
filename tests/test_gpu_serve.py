"""Serving queue (continuous batching): every result equals the oracle and the
same graph's result alone; admission by memory budget; back-pressure and
drain timeouts are reported on the host."""
import time

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


def to_dev(g):
    if hasattr(g, "rows"):
        return ("dense", torch.from_numpy(np.ascontiguousarray(g.rows).view(np.int32)).to(DEV), g.n)
    rp = torch.from_numpy(g.row_ptr).to(DEV)
    col = torch.from_numpy(g.col).to(DEV) if g.nnz else torch.zeros(1, dtype=torch.int32, device=DEV)[:0]
    return ("csr", (rp, col), g.n)


def submit(q, dg):
    kind, data, n = dg
    return q.submit_dense(data, n) if kind == "dense" else q.submit_csr(data[0], data[1], n)


@pytest.fixture(scope="module")
def mix():
    graphs = []
    rs = np.random.Generator(np.random.PCG64(3))
    for i in range(40):                                   # small dense, both verdicts
        n = int(rs.integers(16, 1500))
        g = gg.subtree_dense(n, max(2, n // 4), 100 + i)
        graphs.append(gg.plant_cycle(g, 5 + i % 4, i)[0] if i % 2 and n >= 8 else g)
    graphs.append(gg.subtree_dense(6000, 400, 7))          # bucket 9 (n > 4096)
    graphs.append(gg.close_cycles_dense(gg.subtree_dense(5000, 500, 8), 2, 8)[0])
    graphs.append(gg.dense_to_csr(gg.subtree_dense(9000, 600, 9)))      # CSR, expanded to bits
    graphs.append(gg.dense_to_csr(gg.plant_cycle(gg.subtree_dense(3000, 300, 10), 6, 10)[0]))
    graphs.append(gg.peo_csr(20000, 11))                   # sparse CSR: CSR kernels
    graphs.append(gg.close_cycles_csr(gg.peo_csr(15000, 12), 2, 12)[0])
    graphs.append(gg.empty_dense(0))
    graphs.append(gg.cycle(4))
    tests = [oracle.chordal_test(g) for g in graphs]
    return graphs, [t.witness for t in tests], [t.order for t in tests]


def test_mixed_stream_matches_oracle_and_alone(mix):
    """Each query's verdict, witness and LexBFS order are bit-exact, in the
    mix (batches overlapping in flight) and alone."""
    graphs, want, want_order = mix
    dev = [to_dev(g) for g in graphs]
    with B.Context(0) as ctx:
        q = B.Queue(ctx, mem_budget_bytes=1 << 30, max_inflight=4, max_batch=16, keep_orders=True)
        tickets = []
        for k, dg in enumerate(dev):       # staggered arrivals so batches overlap in flight
            tickets.append(submit(q, dg))
            if k % 7 == 0:
                time.sleep(0.0005)
        assert q.drain(int(120e9)) == B.CG_OK
        mixed = []
        for t, wo in zip(tickets, want_order):
            st, res, lat, order = q.poll(t, with_order=True)
            assert st == B.CG_OK and lat > 0
            assert np.array_equal(order, wo)
            mixed.append(res)
        assert mixed == want
        st = q.stats()
        assert st["completed"] == len(graphs) and st["batches"] >= 3
        # each graph alone through the queue
        for dg, w, wo in zip(dev, want, want_order):
            t = submit(q, dg)
            assert q.drain(int(60e9)) == B.CG_OK
            st, res, _, order = q.poll(t, with_order=True)
            assert st == B.CG_OK and res == w and np.array_equal(order, wo)
        q.close()


def test_orders_need_keep_orders(mix):
    graphs, want, _ = mix
    with B.Context(0) as ctx:
        q = B.Queue(ctx, mem_budget_bytes=64 << 20)
        t = submit(q, to_dev(graphs[0]))
        assert q.drain(int(60e9)) == B.CG_OK
        st, _, _, _ = q.poll(t, with_order=True)
        assert st == B.CG_EINVAL                            # this queue keeps no orders
        assert q.poll(t)[0:2] == (B.CG_OK, want[0])         # the ticket is still there
        q.close()


def test_csr_queries_checked_at_submit_when_validating():
    """With cfg.validate a malformed CSR query is refused at submit (it never
    reaches a kernel); well-formed ones are served."""
    c = gg.dense_to_csr(gg.subtree_dense(300, 40, 3))
    rp = torch.from_numpy(c.row_ptr).to(DEV)
    col_ok = torch.from_numpy(c.col).to(DEV)
    bad = c.col.copy()
    bad[5] = c.n                                            # a column index out of range
    col_bad = torch.from_numpy(bad).to(DEV)
    with B.Context(0, validate=1) as ctx:
        q = B.Queue(ctx, mem_budget_bytes=64 << 20)
        with pytest.raises(B.ChordalError) as e:
            q.submit_csr(rp, col_bad, c.n)
        assert e.value.status == B.CG_EINVAL
        t = q.submit_csr(rp, col_ok, c.n)
        assert q.drain(int(60e9)) == B.CG_OK
        assert q.poll(t)[0:2] == (B.CG_OK, oracle.chordal_test(c).witness)
        q.close()


def test_memory_budget_admission_and_oversize(mix):
    graphs, want, _ = mix
    big = gg.subtree_dense(16384, 562, 3)                  # 32 MiB rows, ~0.4 MiB of scratch
    with B.Context(0) as ctx:
        q = B.Queue(ctx, mem_budget_bytes=2 << 20, max_inflight=2, max_batch=64)   # 2 MiB pool
        dev = [to_dev(g) for g in graphs[:40]]
        tickets = [submit(q, dg) for dg in dev]
        assert q.drain(int(60e9)) == B.CG_OK
        assert [q.poll(t)[1] for t in tickets] == want[:40]
        assert q.stats()["batches"] > 1                    # the budget forced several batches
        # a CSR query that expands to 32 MiB of bits can never fit a 2 MiB pool
        c = to_dev(gg.dense_to_csr(big))
        t = submit(q, c)
        assert q.drain(int(60e9)) == B.CG_OK
        st, res, _ = q.poll(t)
        assert st == B.CG_ENOMEM
        q.close()


def test_back_pressure_and_drain_timeout():
    g = gg.subtree_dense(16384, 562, 5)                    # ~37 ms of GPU time
    dg = to_dev(g)
    with B.Context(0) as ctx:
        q = B.Queue(ctx, max_pending=2, max_inflight=1, max_batch=1)
        t1 = submit(q, dg)
        accepted, rejected = [t1], 0
        for _ in range(8):
            try:
                accepted.append(submit(q, dg))
            except B.ChordalError as e:
                assert e.status == B.CG_EAGAIN
                rejected += 1
        assert rejected > 0
        assert q.drain(1000) == B.CG_ETIMEOUT              # 1 us: work still in flight
        assert q.drain(int(60e9)) == B.CG_OK
        w = oracle.chordal_test(g).witness
        for t in accepted:
            st, res, _ = q.poll(t)
            assert st == B.CG_OK and res == w
        q.close()
