"""ctypes binding of libchordal.so (argument marshalling only).

Every C entry point of ``include/chordal.h`` is exposed under the same name
with the same arguments (device pointers as ints, ``cudaStream_t`` as an int
handle).  The helpers at the bottom accept torch tensors and pass their data
pointers and the current torch stream; all work runs in the library's CUDA
kernels.  There is no fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# CG_LIBCHORDAL selects another build of the library (e.g. the bounds-checking
# libchordal_debug.so); the default is the release build next to this file.
LIB_PATH = os.environ.get("CG_LIBCHORDAL") or os.path.join(HERE, "libchordal.so")
DEBUG_LIB_PATH = os.path.join(HERE, "libchordal_debug.so")

CG_OK, CG_EINVAL, CG_ENOMEM, CG_ECUDA, CG_ETIMEOUT, CG_EAGAIN = range(6)
_STATUS = {0: "CG_OK", 1: "CG_EINVAL", 2: "CG_ENOMEM", 3: "CG_ECUDA", 4: "CG_ETIMEOUT", 5: "CG_EAGAIN"}


class ChordalError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class cg_dense(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("words_per_row", ctypes.c_int32), ("rows", ctypes.c_void_p)]


class cg_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p)]


class cg_result(ctypes.Structure):
    _fields_ = [("chordal", ctypes.c_int32), ("v", ctypes.c_int32), ("p", ctypes.c_int32), ("u", ctypes.c_int32)]

    def astuple(self):
        return (self.chordal, self.v, self.p, self.u)


class cg_profile(ctypes.Structure):
    _fields_ = [("lexbfs_ms", ctypes.c_double), ("check_ms", ctypes.c_double), ("fused_ms", ctypes.c_double),
                ("batch_ms", ctypes.c_double), ("lexbfs_launches", ctypes.c_int64),
                ("check_launches", ctypes.c_int64), ("fused_launches", ctypes.c_int64),
                ("batch_calls", ctypes.c_int64), ("kernel_launches", ctypes.c_int64)]


class cg_graph_ref(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("dense", cg_dense), ("csr", cg_csr)]


class cg_queue_config(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("max_pending", ctypes.c_int32), ("max_batch_large", ctypes.c_int32),
                ("keep_orders", ctypes.c_int32)]


class cg_step_floor_info(ctypes.Structure):
    _fields_ = [("barrier_pair_ns", ctypes.c_double), ("load_ns", ctypes.c_double), ("chain_bytes", ctypes.c_int64)]


class cg_queue_info(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "completed", "pending", "inflight", "batches",
                                              "pool_free_bytes")]


CG_GRAPH_DENSE, CG_GRAPH_CSR = 0, 1


class cg_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("validate", ctypes.c_int32), ("threads_override", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64

# name -> argtypes (restype int unless noted)
SIGNATURES = {
    "cg_version": ([], ctypes.c_char_p),
    "cg_last_error_string": ([], ctypes.c_char_p),
    "cg_context_create": ([P, P], ctypes.c_int),
    "cg_context_destroy": ([P], ctypes.c_int),
    "cg_lexbfs_order_dense": ([P, P, P, P, P], ctypes.c_int),
    "cg_peo_check_dense": ([P, P, P, P, P, P], ctypes.c_int),
    "cg_chordal_test_dense": ([P, P, P, P, P], ctypes.c_int),
    "cg_chordal_test_dense_host": ([P, I32, I32, P, P, P, P], ctypes.c_int),
    "cg_chordal_test_batch": ([P, P, I32, P, P, P, P], ctypes.c_int),
    "cg_chordal_test_batch_host": ([P, P, I32, P, P, P], ctypes.c_int),
    "cg_lexbfs_sweep_dense": ([P, P, ctypes.c_int32, P, ctypes.c_int32, P, P, P], ctypes.c_int),
    "cg_lexbfs_sweep_csr": ([P, P, ctypes.c_int32, P, ctypes.c_int32, P, P, P], ctypes.c_int),
    "cg_mcs_order_dense": ([P, P, P, P, P], ctypes.c_int),
    "cg_chordal_test_mcs_dense": ([P, P, P, P, P], ctypes.c_int),
    "cg_lexbfs_order_csr": ([P, P, P, P, P], ctypes.c_int),
    "cg_peo_check_csr": ([P, P, P, P, P, P], ctypes.c_int),
    "cg_chordal_test_csr": ([P, P, P, P, P], ctypes.c_int),
    "cg_chordal_test_csr_host": ([P, I32, I64, P, P, P, P, P], ctypes.c_int),
    "cg_chordal_test_dense_noalloc": ([P, P, P, P], ctypes.c_int),
    "cg_profile_enable": ([P, I32], ctypes.c_int),
    "cg_queue_create": ([P, P, P], ctypes.c_int),
    "cg_queue_submit": ([P, P, P], ctypes.c_int),
    "cg_queue_poll": ([P, ctypes.c_uint64, P, P, P], ctypes.c_int),
    "cg_queue_drain": ([P, I64], ctypes.c_int),
    "cg_queue_stats": ([P, P], ctypes.c_int),
    "cg_queue_destroy": ([P], ctypes.c_int),
    "cg_batch_plan_create": ([P, P, I32, P, P, P, P], ctypes.c_int),
    "cg_batch_plan_run": ([P, P], ctypes.c_int),
    "cg_batch_plan_destroy": ([P], ctypes.c_int),
    "cg_batch_autotune": ([P, P, I32, P], ctypes.c_int),
    "cg_autotune_get": ([P, P, I32], ctypes.c_int),
    "cg_autotune_set": ([P, P, I32], ctypes.c_int),
    "cg_profile_read": ([P, P], ctypes.c_int),
    "cg_step_floor": ([P, I32, I32, I64, I32, P, P], ctypes.c_int),
    "cg_debug_describe": ([ctypes.c_uint64, P, I32], ctypes.c_int),
    "cg_debug_inject": ([I32], ctypes.c_int),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libchordal.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise ImportError(f"{p} is missing: build it with `python -m paper_1508_06329_gb300.build` "
                                  "(there is no CPU fallback)")
            lib = ctypes.CDLL(p)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _check(status: int):
    if status != CG_OK:
        raise ChordalError(status, load().cg_last_error_string().decode())


def _fn(name):
    def call(*args):
        return getattr(load(), name)(*args)
    call.__name__ = name
    return call


# Same names as the C ABI: raw calls returning the status code.
cg_version = _fn("cg_version")
cg_last_error_string = _fn("cg_last_error_string")
cg_context_create = _fn("cg_context_create")
cg_context_destroy = _fn("cg_context_destroy")
cg_lexbfs_order_dense = _fn("cg_lexbfs_order_dense")
cg_peo_check_dense = _fn("cg_peo_check_dense")
cg_chordal_test_dense = _fn("cg_chordal_test_dense")
cg_chordal_test_dense_host = _fn("cg_chordal_test_dense_host")
cg_chordal_test_batch = _fn("cg_chordal_test_batch")
cg_chordal_test_batch_host = _fn("cg_chordal_test_batch_host")
cg_lexbfs_sweep_dense = _fn("cg_lexbfs_sweep_dense")
cg_lexbfs_sweep_csr = _fn("cg_lexbfs_sweep_csr")
cg_mcs_order_dense = _fn("cg_mcs_order_dense")
cg_chordal_test_mcs_dense = _fn("cg_chordal_test_mcs_dense")
cg_lexbfs_order_csr = _fn("cg_lexbfs_order_csr")
cg_peo_check_csr = _fn("cg_peo_check_csr")
cg_chordal_test_csr = _fn("cg_chordal_test_csr")
cg_chordal_test_csr_host = _fn("cg_chordal_test_csr_host")
cg_chordal_test_dense_noalloc = _fn("cg_chordal_test_dense_noalloc")
cg_debug_describe = _fn("cg_debug_describe")
cg_debug_inject = _fn("cg_debug_inject")
cg_profile_enable = _fn("cg_profile_enable")
cg_queue_create = _fn("cg_queue_create")
cg_queue_submit = _fn("cg_queue_submit")
cg_queue_poll = _fn("cg_queue_poll")
cg_queue_drain = _fn("cg_queue_drain")
cg_queue_stats = _fn("cg_queue_stats")
cg_queue_destroy = _fn("cg_queue_destroy")
cg_batch_plan_create = _fn("cg_batch_plan_create")
cg_batch_plan_run = _fn("cg_batch_plan_run")
cg_batch_plan_destroy = _fn("cg_batch_plan_destroy")
cg_batch_autotune = _fn("cg_batch_autotune")
cg_autotune_get = _fn("cg_autotune_get")
cg_autotune_set = _fn("cg_autotune_set")
cg_profile_read = _fn("cg_profile_read")
cg_step_floor = _fn("cg_step_floor")


# --------------------------------------------------------------------------- torch-facing helpers

def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Context:
    """Owns a cg_context (device workspace + pinned staging)."""

    def __init__(self, device: int = 0, threads_override: int = 0, validate: int = 0):
        cfg = cg_config(device, validate, threads_override, 0)
        h = ctypes.c_void_p()
        _check(cg_context_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self.device = device

    def profile(self, enable: bool = True):
        _check(cg_profile_enable(self.handle, 1 if enable else 0))

    def read_profile(self) -> dict:
        p = cg_profile()
        _check(cg_profile_read(self.handle, ctypes.byref(p)))
        return {f: getattr(p, f) for f, _ in cg_profile._fields_}

    def close(self):
        if self.handle:
            _check(cg_context_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dense_desc(rows, n: int) -> cg_dense:
    """rows: CUDA tensor of 32-bit words, shape [n, words] (int32 or uint32)."""
    words = int(rows.shape[1]) if rows.dim() == 2 else 0
    if rows.element_size() != 4 or not rows.is_contiguous():
        raise ValueError("rows must be a contiguous tensor of 32-bit words")
    return cg_dense(n, words, _ptr(rows))


def lexbfs_order_dense(ctx: Context, rows, n: int, order, pos=None, stream=None):
    d = dense_desc(rows, n)
    _check(cg_lexbfs_order_dense(ctx.handle, ctypes.byref(d), _ptr(order), _ptr(pos), _stream(stream)))


def chordal_test_dense(ctx: Context, rows, n: int, res, order=None, stream=None):
    """res: CUDA int32 tensor [4] -> (chordal, v, p, u)."""
    d = dense_desc(rows, n)
    _check(cg_chordal_test_dense(ctx.handle, ctypes.byref(d), _ptr(res), _ptr(order), _stream(stream)))


TIE_ID, TIE_RANK, TIE_LAST_IN = 0, 1, 2


def lexbfs_sweep_dense(ctx: Context, rows, n: int, order, pos=None, kind: int = TIE_ID, tiebreak=None,
                       start: int = -1, stream=None):
    d = dense_desc(rows, n)
    _check(cg_lexbfs_sweep_dense(ctx.handle, ctypes.byref(d), kind, _ptr(tiebreak), start, _ptr(order), _ptr(pos),
                                 _stream(stream)))


def lexbfs_plus_dense(ctx: Context, rows, n: int, prev_order, order, pos=None, start: int = -1, stream=None):
    """LexBFS+ of a previous sweep: ties go to the vertex latest in prev_order."""
    lexbfs_sweep_dense(ctx, rows, n, order, pos, TIE_LAST_IN, prev_order, start, stream)


def mcs_order_dense(ctx: Context, rows, n: int, order, pos=None, stream=None):
    d = dense_desc(rows, n)
    _check(cg_mcs_order_dense(ctx.handle, ctypes.byref(d), _ptr(order), _ptr(pos), _stream(stream)))


def chordal_test_mcs_dense(ctx: Context, rows, n: int, res, order=None, stream=None):
    d = dense_desc(rows, n)
    _check(cg_chordal_test_mcs_dense(ctx.handle, ctypes.byref(d), _ptr(res), _ptr(order), _stream(stream)))


def peo_check_dense(ctx: Context, rows, n: int, order, res, parent=None, stream=None):
    d = dense_desc(rows, n)
    _check(cg_peo_check_dense(ctx.handle, ctypes.byref(d), _ptr(order), _ptr(parent), _ptr(res), _stream(stream)))


def chordal_test_dense_host(ctx: Context, rows_host, n: int, order_host=None, stream=None) -> tuple:
    """rows_host: CPU tensor/ndarray of 32-bit words [n, words] (pinned preferred)."""
    import numpy as np
    if hasattr(rows_host, "data_ptr"):
        ptr, words = int(rows_host.data_ptr()), int(rows_host.shape[1]) if rows_host.dim() == 2 else 0
        optr = 0 if order_host is None else int(order_host.data_ptr())
    else:
        a = np.ascontiguousarray(rows_host)
        ptr, words = a.ctypes.data, (a.shape[1] if a.ndim == 2 else 0)
        optr = 0 if order_host is None else order_host.ctypes.data
    out = cg_result()
    _check(cg_chordal_test_dense_host(ctx.handle, n, words, ptr, ctypes.byref(out), optr, _stream(stream)))
    return out.astuple()


def chordal_test_batch(ctx: Context, graphs, res, orders=None, order_offsets=None, stream=None):
    """graphs: list of (rows_tensor, n); res: CUDA int32 tensor [count, 4]."""
    count = len(graphs)
    arr = (cg_dense * max(count, 1))()
    for k, (rows, n) in enumerate(graphs):
        arr[k] = dense_desc(rows, n)
    offs = None
    if order_offsets is not None:
        offs = (ctypes.c_int64 * max(count, 1))(*[int(x) for x in order_offsets])
    _check(cg_chordal_test_batch(ctx.handle, arr, count, _ptr(res), _ptr(orders),
                                 offs if offs is not None else None, _stream(stream)))


class HostBatch:
    """The cg_dense descriptors of a list of host graphs, built once: repeated
    calls on the same host buffers (whose contents may change between calls)
    skip the per-graph marshalling.  graphs: list of (rows, n) with rows a CPU
    tensor or ndarray of 32-bit words [n, words] (pinned preferred)."""

    def __init__(self, graphs):
        import numpy as np
        self.count = len(graphs)
        self.arr = (cg_dense * max(self.count, 1))()
        self._keep = []   # the arrays whose addresses the descriptors hold
        for k, (rows, n) in enumerate(graphs):
            if hasattr(rows, "data_ptr"):
                ptr, words = int(rows.data_ptr()), (int(rows.shape[1]) if rows.dim() == 2 else 0)
                self._keep.append(rows)
            else:
                a = np.ascontiguousarray(rows)
                self._keep.append(a)
                ptr, words = a.ctypes.data, (a.shape[1] if a.ndim == 2 else 0)
            self.arr[k] = cg_dense(n, words, ptr if n > 0 else 0)


def chordal_test_batch_host(ctx: Context, graphs, host_res, host_orders=None, stream=None):
    """graphs: a HostBatch, or a list of (rows, n) as HostBatch takes; host_res: CPU int32
    tensor/ndarray [count, 4]; host_orders: CPU int32 [sum n] or None."""
    batch = graphs if isinstance(graphs, HostBatch) else HostBatch(graphs)

    def hptr(x):
        if x is None:
            return None
        return int(x.data_ptr()) if hasattr(x, "data_ptr") else x.ctypes.data
    _check(cg_chordal_test_batch_host(ctx.handle, batch.arr, batch.count, hptr(host_res), hptr(host_orders),
                                      _stream(stream)))


def csr_desc(row_ptr, col, n: int) -> cg_csr:
    """row_ptr: CUDA int64 tensor [n+1]; col: CUDA int32 tensor [nnz]."""
    if row_ptr.element_size() != 8 or col.element_size() != 4:
        raise ValueError("row_ptr must hold int64 and col int32")
    return cg_csr(n, int(col.numel()), _ptr(row_ptr), _ptr(col) if col.numel() else 0)


def lexbfs_order_csr(ctx: Context, row_ptr, col, n: int, order, pos=None, stream=None):
    d = csr_desc(row_ptr, col, n)
    _check(cg_lexbfs_order_csr(ctx.handle, ctypes.byref(d), _ptr(order), _ptr(pos), _stream(stream)))


def lexbfs_sweep_csr(ctx: Context, row_ptr, col, n: int, order, pos=None, kind: int = TIE_ID, tiebreak=None,
                     start: int = -1, stream=None):
    d = csr_desc(row_ptr, col, n)
    _check(cg_lexbfs_sweep_csr(ctx.handle, ctypes.byref(d), kind, _ptr(tiebreak), start, _ptr(order), _ptr(pos),
                               _stream(stream)))


def lexbfs_plus_csr(ctx: Context, row_ptr, col, n: int, prev_order, order, pos=None, start: int = -1, stream=None):
    """LexBFS+ of a previous sweep on a CSR graph."""
    lexbfs_sweep_csr(ctx, row_ptr, col, n, order, pos, TIE_LAST_IN, prev_order, start, stream)


def chordal_test_csr(ctx: Context, row_ptr, col, n: int, res, order=None, stream=None):
    d = csr_desc(row_ptr, col, n)
    _check(cg_chordal_test_csr(ctx.handle, ctypes.byref(d), _ptr(res), _ptr(order), _stream(stream)))


def peo_check_csr(ctx: Context, row_ptr, col, n: int, order, res, parent=None, stream=None):
    d = csr_desc(row_ptr, col, n)
    _check(cg_peo_check_csr(ctx.handle, ctypes.byref(d), _ptr(order), _ptr(parent), _ptr(res), _stream(stream)))


def chordal_test_csr_host(ctx: Context, row_ptr, col, n: int, order_host=None, stream=None) -> tuple:
    """row_ptr / col: host numpy arrays (int64 / int32) or CPU tensors."""
    import numpy as np

    def hp(a):
        if a is None:
            return 0
        return int(a.data_ptr()) if hasattr(a, "data_ptr") else np.ascontiguousarray(a).ctypes.data
    nnz = int(col.numel() if hasattr(col, "numel") else col.shape[0])
    out = cg_result()
    _check(cg_chordal_test_csr_host(ctx.handle, n, nnz, hp(row_ptr), hp(col) if nnz else 0, ctypes.byref(out),
                                    hp(order_host), _stream(stream)))
    return out.astuple()


def _dense_array(graphs):
    arr = (cg_dense * max(len(graphs), 1))()
    for k, (rows, n) in enumerate(graphs):
        arr[k] = dense_desc(rows, n)
    return arr


class BatchPlan:
    """A captured batch (cg_batch_plan): run() replays one CUDA graph."""

    def __init__(self, ctx: Context, graphs, res, orders=None, order_offsets=None):
        self.ctx = ctx
        self._keep = (graphs, res, orders)
        arr = _dense_array(graphs)
        offs = None
        if order_offsets is not None:
            offs = (ctypes.c_int64 * max(len(graphs), 1))(*[int(x) for x in order_offsets])
        h = ctypes.c_void_p()
        _check(cg_batch_plan_create(ctx.handle, arr, len(graphs), _ptr(res), _ptr(orders), offs, ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None):
        _check(cg_batch_plan_run(self.handle, _stream(stream)))

    def close(self):
        if self.handle:
            _check(cg_batch_plan_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_autotune(ctx: Context, graphs, stream=None) -> list:
    arr = _dense_array(graphs)
    _check(cg_batch_autotune(ctx.handle, arr, len(graphs), _stream(stream)))
    return autotune_get(ctx)


def autotune_get(ctx: Context) -> list:
    buf = (ctypes.c_int32 * 9)()
    _check(cg_autotune_get(ctx.handle, buf, 9))
    return list(buf)


def autotune_set(ctx: Context, table) -> None:
    buf = (ctypes.c_int32 * 9)(*[int(x) for x in table][:9])
    _check(cg_autotune_set(ctx.handle, buf, 9))


def step_floor(ctx: Context, threads: int = 1024, iters: int = 16384, chain_bytes: int = 32 << 20,
               loads: int = 100000, stream=None) -> dict:
    """Latency floors of one LexBFS step (cg_step_floor): ns per pair of CTA
    barriers and ns per dependent load over a chain of `chain_bytes`."""
    out = cg_step_floor_info()
    _check(cg_step_floor(ctx.handle, threads, iters, chain_bytes, loads, _stream(stream), ctypes.byref(out)))
    return {f: getattr(out, f) for f, _ in cg_step_floor_info._fields_}


class Queue:
    """Continuous-batching request queue (cg_queue_*).  Graph tensors passed to
    submit_* must stay alive until their ticket completes (kept here)."""

    def __init__(self, ctx: Context, mem_budget_bytes: int = 0, max_inflight: int = 0, max_batch: int = 0,
                 max_pending: int = 0, max_batch_large: int = 0, keep_orders: bool = False):
        cfg = cg_queue_config(mem_budget_bytes, max_inflight, max_batch, max_pending, max_batch_large,
                              1 if keep_orders else 0)
        self.keep_orders = keep_orders
        h = ctypes.c_void_p()
        _check(cg_queue_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def _submit(self, ref, keep, n: int) -> int:
        t = ctypes.c_uint64()
        _check(cg_queue_submit(self.handle, ctypes.byref(ref), ctypes.byref(t)))
        self._keep[t.value] = (keep, n)
        return t.value

    def submit_dense(self, rows, n: int) -> int:
        ref = cg_graph_ref(CG_GRAPH_DENSE, dense_desc(rows, n), cg_csr())
        return self._submit(ref, rows, n)

    def submit_csr(self, row_ptr, col, n: int) -> int:
        ref = cg_graph_ref(CG_GRAPH_CSR, cg_dense(), csr_desc(row_ptr, col, n))
        return self._submit(ref, (row_ptr, col), n)

    def poll(self, ticket: int, with_order: bool = False):
        """(status, (chordal, v, p, u), latency_s), plus the order (numpy int32[n]) when
        with_order (the queue must keep orders); status CG_EAGAIN while pending."""
        import numpy as np
        r = cg_result()
        lat = ctypes.c_double()
        order = None
        optr = None
        if with_order:
            n = self._keep.get(ticket, (None, 0))[1]
            order = np.full(max(n, 1), -1, dtype=np.int32)
            optr = order.ctypes.data
        st = cg_queue_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(r), optr, ctypes.byref(lat))
        if st != CG_EAGAIN:
            n = self._keep.pop(ticket, (None, 0))[1]
            if order is not None:
                order = order[:n]
        if with_order:
            return st, r.astuple(), lat.value, order
        return st, r.astuple(), lat.value

    def drain(self, timeout_ns: int = -1) -> int:
        return cg_queue_drain(self.handle, timeout_ns)

    def stats(self) -> dict:
        info = cg_queue_info()
        _check(cg_queue_stats(self.handle, ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in cg_queue_info._fields_}

    def close(self):
        if self.handle:
            _check(cg_queue_destroy(self.handle))
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
