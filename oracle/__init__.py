"""CPU oracle for the parallel chordality test.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference arm may import this package.  It
shares no code with the CUDA path (``paper_1508_06329_gb300``) and never
imports it.

Contents
* ``oracle.c`` (compiled on demand to ``liboracle.so``): the O(N + M)
  partition-refinement LexBFS with the lowest-id tie-break (Section 4.2) or a
  caller-given tie-break rank and start vertex (multi-sweep LexBFS), the
  perfect-elimination check with its canonical witness (Sections 5.2-5.3), and
  Maximum Cardinality Search with the same tie-break (Section 5.1).
* ``reference.py``: slower restatements used to pin the C code — LexBFS by
  explicit labels (Section 4.1), the O(N^2) class-splitting form of Section
  4.2, Maximum Cardinality Search (Section 5.1) and the definition of a
  perfect elimination order (Section 3.1).

Result convention: ``(chordal, v, p, u)``; when chordal is 1 the witness is
(-1, -1, -1).  Otherwise v is the violating vertex with the smallest order
index, p = p(v) its rightmost earlier neighbour and u the smallest id in
(LN_v - {p}) \\ N(p).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc -O2, single thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path: str) -> ctypes.CDLL:
    """Load a build of oracle.c and declare its entry points."""
    lib = ctypes.CDLL(path)
    P, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.or_lexbfs_csr.argtypes = [i32, P, P, P]
    lib.or_lexbfs_dense.argtypes = [i32, i32, P, P]
    lib.or_peo_check_csr.argtypes = [i32, P, P, P, P, P]
    lib.or_peo_check_dense.argtypes = [i32, i32, P, P, P, P]
    lib.or_chordal_test_csr.argtypes = [i32, P, P, P, P, P]
    lib.or_chordal_test_dense.argtypes = [i32, i32, P, P, P, P]
    lib.or_lexbfs_rank_csr.argtypes = [i32, P, P, P, i32, P]
    lib.or_lexbfs_rank_dense.argtypes = [i32, i32, P, P, i32, P]
    lib.or_mcs_csr.argtypes = [i32, P, P, P]
    lib.or_mcs_dense.argtypes = [i32, i32, P, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def use_library(path: str) -> None:
    """Point the oracle at another build of oracle.c (the planted-mistake tests
    load deliberately broken copies this way, in a child process)."""
    global _lib
    with _lock:
        _lib = _bind(path)


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


@dataclass
class OracleResult:
    order: np.ndarray      # int32[n], order[i] = i-th visited vertex
    parent: np.ndarray     # int32[n], p(v) or -1
    chordal: int
    v: int
    p: int
    u: int

    @property
    def pos(self) -> np.ndarray:
        pos = np.empty_like(self.order)
        pos[self.order] = np.arange(self.order.shape[0], dtype=self.order.dtype)
        return pos

    @property
    def witness(self) -> tuple[int, int, int, int]:
        return (self.chordal, self.v, self.p, self.u)


def _is_dense(g) -> bool:
    return hasattr(g, "rows")


def _dense_args(g):
    rows = np.ascontiguousarray(g.rows, dtype=np.uint32)
    return rows, (rows.shape[1] if rows.ndim == 2 else 0)


def _csr_args(g):
    return (np.ascontiguousarray(g.row_ptr, dtype=np.int64), np.ascontiguousarray(g.col, dtype=np.int32))


def lexbfs(g) -> np.ndarray:
    """LexBFS order under the lowest-id tie-break (Section 4.2)."""
    order = np.zeros(max(g.n, 1), dtype=np.int32)
    if _is_dense(g):
        rows, words = _dense_args(g)
        rc = _load().or_lexbfs_dense(g.n, words, _p(rows), _p(order))
    else:
        rp, col = _csr_args(g)
        rc = _load().or_lexbfs_csr(g.n, _p(rp), _p(col), _p(order))
    if rc:
        raise ValueError(f"oracle lexbfs failed ({rc})")
    return order[:g.n]


def lexbfs_tiebreak(g, rank=None, start: int = -1) -> np.ndarray:
    """LexBFS whose ties go to the smallest rank[v] (a permutation of
    0..n-1; None = the vertex id), with `start` (if >= 0) numbered first: the
    sweep that multi-sweep LexBFS repeats (Section 4.2's refinement started
    from the class ordered by rank)."""
    order = np.zeros(max(g.n, 1), dtype=np.int32)
    rk = None if rank is None else np.ascontiguousarray(rank, dtype=np.int32)
    rp_ = ctypes.c_void_p(0) if rk is None else _p(rk)
    if _is_dense(g):
        rows, words = _dense_args(g)
        rc = _load().or_lexbfs_rank_dense(g.n, words, _p(rows), rp_, int(start), _p(order))
    else:
        rp, col = _csr_args(g)
        rc = _load().or_lexbfs_rank_csr(g.n, _p(rp), _p(col), rp_, int(start), _p(order))
    if rc:
        raise ValueError(f"oracle lexbfs_tiebreak failed ({rc})")
    return order[:g.n]


def lexbfs_plus(g, prev_order, start: int = -1) -> np.ndarray:
    """LexBFS+ of a previous sweep: ties go to the vertex that comes latest in
    prev_order (rank = n - 1 - position in prev_order)."""
    prev = np.asarray(prev_order, dtype=np.int64)
    rank = np.empty(g.n, dtype=np.int32)
    rank[prev] = g.n - 1 - np.arange(g.n)
    return lexbfs_tiebreak(g, rank, start)


def mcs(g) -> np.ndarray:
    """Maximum Cardinality Search order, lowest-id tie-break (Section 5.1)."""
    order = np.zeros(max(g.n, 1), dtype=np.int32)
    if _is_dense(g):
        rows, words = _dense_args(g)
        rc = _load().or_mcs_dense(g.n, words, _p(rows), _p(order))
    else:
        rp, col = _csr_args(g)
        rc = _load().or_mcs_csr(g.n, _p(rp), _p(col), _p(order))
    if rc:
        raise ValueError(f"oracle mcs failed ({rc})")
    return order[:g.n]


def chordal_test_mcs(g) -> OracleResult:
    """MCS order, then the perfect-elimination check (Theorem 5.2)."""
    return peo_check(g, mcs(g))


def peo_check(g, order) -> OracleResult:
    """Perfect-elimination check of a given order (Sections 5.2-5.3)."""
    order = np.ascontiguousarray(order, dtype=np.int32)
    parent = np.zeros(max(g.n, 1), dtype=np.int32)
    res = np.zeros(4, dtype=np.int32)
    if _is_dense(g):
        rows, words = _dense_args(g)
        rc = _load().or_peo_check_dense(g.n, words, _p(rows), _p(order), _p(parent), _p(res))
    else:
        rp, col = _csr_args(g)
        rc = _load().or_peo_check_csr(g.n, _p(rp), _p(col), _p(order), _p(parent), _p(res))
    if rc:
        raise ValueError(f"oracle peo_check failed ({rc})")
    return OracleResult(order[:g.n].copy(), parent[:g.n], *[int(x) for x in res])


def chordal_test(g) -> OracleResult:
    """LexBFS, then the perfect-elimination check: the whole test."""
    order = np.zeros(max(g.n, 1), dtype=np.int32)
    parent = np.zeros(max(g.n, 1), dtype=np.int32)
    res = np.zeros(4, dtype=np.int32)
    if _is_dense(g):
        rows, words = _dense_args(g)
        rc = _load().or_chordal_test_dense(g.n, words, _p(rows), _p(order), _p(parent), _p(res))
    else:
        rp, col = _csr_args(g)
        rc = _load().or_chordal_test_csr(g.n, _p(rp), _p(col), _p(order), _p(parent), _p(res))
    if rc:
        raise ValueError(f"oracle chordal_test failed ({rc})")
    return OracleResult(order[:g.n], parent[:g.n], *[int(x) for x in res])
