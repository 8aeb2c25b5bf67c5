"""Seeded synthetic graph inputs for the chordality test (inputs only).

This package builds graphs; it holds none of the method's arithmetic.  The CPU
oracle (``oracle/``) and the GPU path (``paper_1508_06329_gb300``) both consume
what it produces and never import each other.

The paper (Section 7) tests cliques, dense random graphs, sparse random graphs
with M = 20N, trees and "chordal random" graphs, but publishes no generator
parameters and no datasets.  The families below are seeded stand-ins with the
shapes of those workloads and of the five benchmark configurations:

* ``subtree_dense``  — intersection graph of random subtrees of a random tree
  (chordal by Gavril's theorem), the model of the N=1,000 / N=16,384 / batched
  workloads;
* ``plant_cycle``    — overwrite k vertices' induced subgraph with C_k;
* ``close_cycles_*`` — add edges uv with u, v connected in G - (N(u) ∩ N(v));
* ``peo_csr``        — chordal graph grown along a reversed perfect elimination
  order with a shuffled id permutation (the N=2^20 sparse workload);
* families: cycles, cliques, paths, stars, trees, interval graphs, G(n, p).

Dense layout: uint32 rows, ``rows[i, j >> 5] >> (j & 31) & 1`` is edge ij,
symmetric, zero diagonal, zero padding.  CSR layout: ``row_ptr`` int64[n+1],
``col`` int32, rows sorted ascending, symmetric, no loops or duplicates.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

SEED_BASE = 1508063290


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to its source (gcc, portable C)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64, u32, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
            lib.gg_subtree_dense.argtypes = [i32, i32, i32, i32, u64, P, i32]
            lib.gg_random_dense.argtypes = [i32, u32, u64, P, i32]
            lib.gg_plant_cycle_dense.argtypes = [i32, i32, P, i32, u64, P]
            lib.gg_close_cycles_dense.argtypes = [i32, i32, P, i32, u64, i32, P]
            lib.gg_peo_edges.argtypes = [i32, i32, u64, P, P, i64]
            lib.gg_peo_edges.restype = i64
            lib.gg_close_cycles_csr.argtypes = [i32, P, P, i32, u64, i32, P]
            lib.gg_stream.argtypes = [u64, P, i64]
            lib.gg_dense_to_csr.argtypes = [i32, i32, P, P, P]
            lib.gg_dense_to_csr.restype = i64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------- containers

def words_for(n: int) -> int:
    return (n + 31) // 32


@dataclass
class DenseGraph:
    n: int
    rows: np.ndarray          # uint32 [n, words]

    @property
    def words(self) -> int:
        return self.rows.shape[1] if self.rows.ndim == 2 else 0

    @property
    def nbytes(self) -> int:
        return int(self.rows.nbytes)

    def copy(self) -> "DenseGraph":
        return DenseGraph(self.n, self.rows.copy())

    def num_edges(self) -> int:
        if self.n == 0:
            return 0
        return int(np.unpackbits(self.rows.view(np.uint8)).sum()) // 2

    def density(self) -> float:
        return self.num_edges() / max(1, self.n * (self.n - 1) // 2)


@dataclass
class CsrGraph:
    n: int
    row_ptr: np.ndarray       # int64 [n+1]
    col: np.ndarray           # int32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @property
    def nbytes(self) -> int:
        return int(self.row_ptr.nbytes + self.col.nbytes)

    def num_edges(self) -> int:
        return self.nnz // 2


def empty_dense(n: int, words: int | None = None) -> DenseGraph:
    w = words_for(n) if words is None else words
    return DenseGraph(n, np.zeros((n, w), dtype=np.uint32))


def dense_from_edges(n: int, edges, words: int | None = None) -> DenseGraph:
    g = empty_dense(n, words)
    e = np.asarray(list(edges) if not isinstance(edges, np.ndarray) else edges, dtype=np.int64).reshape(-1, 2)
    if e.size:
        a, b = e[:, 0], e[:, 1]
        keep = a != b
        a, b = a[keep], b[keep]
        for x, y in ((a, b), (b, a)):
            np.bitwise_or.at(g.rows, (x, y >> 5), (np.uint32(1) << (y & 31).astype(np.uint32)))
    return g


def csr_from_edges(n: int, eu: np.ndarray, ev: np.ndarray) -> CsrGraph:
    """Symmetric CSR with sorted rows; self-loops and duplicate edges dropped."""
    eu = np.asarray(eu, dtype=np.int64)
    ev = np.asarray(ev, dtype=np.int64)
    keep = eu != ev
    key = np.concatenate([eu[keep] * n + ev[keep], ev[keep] * n + eu[keep]])
    key.sort()
    if key.size:
        key = key[np.concatenate([[True], key[1:] != key[:-1]])]
    a = key // n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(a, minlength=n))
    return CsrGraph(n, row_ptr, (key - a * n).astype(np.int32))


def dense_to_csr(g: DenseGraph) -> CsrGraph:
    n = g.n
    if n > 4096:   # large graphs: C pass (no n x n byte matrix)
        rows = np.ascontiguousarray(g.rows)
        rp = np.zeros(n + 1, dtype=np.int64)
        nnz = _load().gg_dense_to_csr(n, g.words, _ptr(rows), _ptr(rp), None)
        col = np.empty(max(nnz, 1), dtype=np.int32)
        _load().gg_dense_to_csr(n, g.words, _ptr(rows), _ptr(rp), _ptr(col))
        return CsrGraph(n, rp, col[:nnz])
    if n == 0:
        return CsrGraph(0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    bits = np.unpackbits(g.rows.view(np.uint8).reshape(n, -1), axis=1, bitorder="little")[:, :n]
    a, b = np.nonzero(bits)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(a, minlength=n))
    return CsrGraph(n, row_ptr, b.astype(np.int32))


def csr_to_dense(g: CsrGraph, words: int | None = None) -> DenseGraph:
    n = g.n
    d = empty_dense(n, words)
    if g.nnz:
        a = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.row_ptr))
        b = g.col.astype(np.int64)
        np.bitwise_or.at(d.rows, (a, b >> 5), (np.uint32(1) << (b & 31).astype(np.uint32)))
    return d


def adjacency_lists(g) -> list[list[int]]:
    c = g if isinstance(g, CsrGraph) else dense_to_csr(g)
    return [c.col[c.row_ptr[i]:c.row_ptr[i + 1]].tolist() for i in range(c.n)]


def relabel_csr(g: CsrGraph, perm: np.ndarray) -> CsrGraph:
    """Vertex i becomes perm[i]."""
    a = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    return csr_from_edges(g.n, perm[a], perm[g.col.astype(np.int64)])


def relabel_dense(g: DenseGraph, perm: np.ndarray) -> DenseGraph:
    c = relabel_csr(dense_to_csr(g), np.asarray(perm, dtype=np.int64))
    return csr_to_dense(c, g.words)


# --------------------------------------------------------------------------- generators

def rng_stream(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _load().gg_stream(ctypes.c_uint64(seed & (2**64 - 1)), _ptr(out), count)
    return out


def subtree_dense(n: int, tree_nodes: int, seed: int, smin: int = 1, smax: int = 20,
                  words: int | None = None) -> DenseGraph:
    g = empty_dense(n, words)
    rc = _load().gg_subtree_dense(n, tree_nodes, smin, smax, ctypes.c_uint64(seed), _ptr(g.rows), g.words)
    if rc != 0:
        raise ValueError("gg_subtree_dense: bad arguments")
    return g


def random_dense(n: int, p: float, seed: int) -> DenseGraph:
    g = empty_dense(n)
    pn = min(int(round(p * 2**32)), 2**32 - 1)
    _load().gg_random_dense(n, ctypes.c_uint32(pn), ctypes.c_uint64(seed), _ptr(g.rows), g.words)
    return g


def plant_cycle(g: DenseGraph, k: int, seed: int) -> tuple[DenseGraph, list[int]]:
    h = g.copy()
    verts = np.zeros(k, dtype=np.int32)
    rc = _load().gg_plant_cycle_dense(h.n, h.words, _ptr(h.rows), k, ctypes.c_uint64(seed), _ptr(verts))
    if rc != 0:
        raise ValueError("gg_plant_cycle_dense: bad arguments")
    return h, verts.tolist()


def close_cycles_dense(g: DenseGraph, r: int, seed: int, max_tries: int = 100000):
    h = g.copy()
    pairs = np.zeros(2 * max(r, 1), dtype=np.int32)
    added = _load().gg_close_cycles_dense(h.n, h.words, _ptr(h.rows), r, ctypes.c_uint64(seed), max_tries, _ptr(pairs))
    return h, [tuple(pairs[2 * j:2 * j + 2].tolist()) for j in range(added)]


def peo_csr(n: int, seed: int, smax: int = 20, permute: bool = True) -> CsrGraph:
    cap = int(n) * smax + 1
    eu = np.empty(cap, dtype=np.int32)
    ev = np.empty(cap, dtype=np.int32)
    m = _load().gg_peo_edges(n, smax, ctypes.c_uint64(seed), _ptr(eu), _ptr(ev), cap)
    if m < 0:
        raise RuntimeError("gg_peo_edges: edge buffer too small")
    eu, ev = eu[:m].astype(np.int64), ev[:m].astype(np.int64)
    if permute:
        perm = np.random.Generator(np.random.PCG64(seed ^ 0x5EED)).permutation(n).astype(np.int64)
        eu, ev = perm[eu], perm[ev]
    return csr_from_edges(n, eu, ev)


def close_cycles_csr(g: CsrGraph, r: int, seed: int, max_tries: int = 100000):
    pairs = np.zeros(2 * max(r, 1), dtype=np.int32)
    added = _load().gg_close_cycles_csr(g.n, _ptr(g.row_ptr), _ptr(g.col), r, ctypes.c_uint64(seed),
                                        max_tries, _ptr(pairs))
    pr = [tuple(pairs[2 * j:2 * j + 2].tolist()) for j in range(added)]
    if not pr:
        return g, pr
    a = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    eu = np.concatenate([a, np.array([p[0] for p in pr], np.int64)])
    ev = np.concatenate([g.col.astype(np.int64), np.array([p[1] for p in pr], np.int64)])
    return csr_from_edges(g.n, eu, ev), pr


# --------------------------------------------------------------------------- families

def cycle(k: int) -> DenseGraph:
    return dense_from_edges(k, [(i, (i + 1) % k) for i in range(k)])


def clique(n: int) -> DenseGraph:
    g = empty_dense(n)
    for i in range(n):
        for w in range(g.words):
            lo = w * 32
            hi = min(n, lo + 32)
            if hi > lo:
                g.rows[i, w] = np.uint32((1 << (hi - lo)) - 1)
        g.rows[i, i >> 5] &= ~np.uint32(1 << (i & 31))
    return g


def path(n: int) -> DenseGraph:
    return dense_from_edges(n, [(i, i + 1) for i in range(n - 1)])


def star(n: int) -> DenseGraph:
    return dense_from_edges(n, [(0, i) for i in range(1, n)])


def random_tree(n: int, seed: int) -> DenseGraph:
    r = rng_stream(seed, max(n, 1))
    edges = [(i, int(r[i] % np.uint64(i))) for i in range(1, n)]
    return dense_from_edges(n, edges)


def interval_graph(n: int, seed: int, span: int = 1000, max_len: int = 60) -> DenseGraph:
    """Intersection graph of n random closed intervals on the integer line."""
    r = rng_stream(seed, 2 * max(n, 1))
    lo = (r[:n] % np.uint64(span)).astype(np.int64)
    ln = (r[n:2 * n] % np.uint64(max_len)).astype(np.int64)
    hi = lo + ln
    edges = [(i, j) for i in range(n) for j in range(i + 1, n) if lo[i] <= hi[j] and lo[j] <= hi[i]]
    return dense_from_edges(n, edges)


# --------------------------------------------------------------------------- workloads

def log_uniform_int(u: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Map uniforms in [0,1) to integers log-uniform in [lo, hi]."""
    v = np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo)))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)


def _u01(seed: int, count: int) -> np.ndarray:
    return (rng_stream(seed, count) >> np.uint64(11)).astype(np.float64) / float(2**53)


def small_dense_pair(seed: int = SEED_BASE + 1, n: int = 1000, tree_nodes: int = 500):
    """N=1,000 workload: subtree model (500-node tree, sizes U{1..20}) and a copy
    with one planted induced C_k, k ~ U{5..8}."""
    g = subtree_dense(n, tree_nodes, seed)
    k = 5 + int(rng_stream(seed + 17, 1)[0] % np.uint64(4))
    h, verts = plant_cycle(g, k, seed + 29)
    return g, h, {"tree_nodes": tree_nodes, "k": k, "cycle": verts}


# Tree size calibrated for N=16,384 at edge density ~0.1: the seeded bisection
# ``calibrate_tree_nodes(16384, 0.10, SEED_BASE + 2)`` returns 562 nodes at
# density 0.0999 (M = 13.4M); the tests re-check the density band.
LARGE_DENSE_TREE_NODES = 562


def calibrate_tree_nodes(n: int, target: float, seed: int, lo: int = 8, hi: int = 4096) -> tuple[int, float]:
    """Smallest-error tree size for the subtree model at a target edge density
    (density decreases as the tree grows); deterministic bisection."""
    best = (lo, subtree_dense(n, lo, seed).density())
    while hi - lo > 1:
        mid = (lo + hi) // 2
        d = subtree_dense(n, mid, seed).density()
        if abs(d - target) < abs(best[1] - target):
            best = (mid, d)
        if d > target:
            lo = mid
        else:
            hi = mid
    return best


def large_dense_pair(seed: int = SEED_BASE + 2, n: int = 16384, tree_nodes: int | None = None):
    """N=16,384 workload: subtree model at density ~0.1 and a copy with
    r ~ U{1..10} cycle-closing extra edges."""
    t = tree_nodes if tree_nodes is not None else (LARGE_DENSE_TREE_NODES or calibrate_tree_nodes(n, 0.10, seed)[0])
    g = subtree_dense(n, t, seed)
    r = 1 + int(rng_stream(seed + 17, 1)[0] % np.uint64(10))
    h, pairs = close_cycles_dense(g, r, seed + 29)
    return g, h, {"tree_nodes": t, "r": r, "pairs": pairs}


def sparse_csr_pair(seed: int = SEED_BASE + 3, n: int = 1 << 20, smax: int = 20):
    """N=2^20 workload: reversed-PEO chordal graph with shuffled ids and a copy
    with 1..10 cycle-closing extra edges."""
    g = peo_csr(n, seed, smax)
    r = 1 + int(rng_stream(seed + 17, 1)[0] % np.uint64(10))
    h, pairs = close_cycles_csr(g, r, seed + 29)
    return g, h, {"smax": smax, "r": r, "pairs": pairs}


def batch_dense(count: int = 4096, seed: int = SEED_BASE + 4, nmin: int = 16, nmax: int = 2048):
    """Batched workload: N log-uniform in [nmin, nmax]; even index = subtree model
    (tree nodes = N/2, sizes U{1..20}), odd index = the same plus a planted
    induced C_k, k ~ U{5..8} (only when N >= k)."""
    ns = log_uniform_int(_u01(seed, count), nmin, nmax)
    graphs = []
    for i, n in enumerate(ns.tolist()):
        g = subtree_dense(n, max(1, n // 2), seed * 7919 + i)
        if i % 2 == 1:
            k = 5 + int(rng_stream(seed + 31 * i, 1)[0] % np.uint64(4))
            if n >= k:
                g, _ = plant_cycle(g, k, seed + 37 * i + 1)
        graphs.append(g)
    return graphs


def serve_pool_item(i: int, count: int = 64, seed: int = SEED_BASE + 5, nmin: int = 64, nmax: int = 65536,
                    dense_below: int = 8192):
    """Graph i of the serving pool (see serve_pool), built alone."""
    u = _u01(seed, 3 * count)
    ns = log_uniform_int(u[:count], nmin, nmax)
    dens = 0.01 + 0.19 * u[count:2 * count]
    n = int(ns[i])
    t = max(2, int(round(56.0 / dens[i])))
    g = subtree_dense(n, t, seed * 31 + i)
    planted = i % 2 == 1
    if planted:
        k = 5 + int(rng_stream(seed + 97 * i, 1)[0] % np.uint64(4))
        if n >= k:
            g, _ = plant_cycle(g, k, seed + 101 * i)
    info = {"n": n, "target_density": float(dens[i]), "tree_nodes": t, "planted": planted}
    return (g if n < dense_below else dense_to_csr(g)), info


def serve_pool(count: int = 64, seed: int = SEED_BASE + 5, nmin: int = 64, nmax: int = 65536,
               dense_below: int = 8192):
    """Serving pool: N log-uniform in [nmin, nmax], target edge density
    U[0.01, 0.2] (subtree model with about 56 / density tree nodes), half of
    the graphs with a planted induced C_k (k ~ U{5..8}); graphs with
    N < dense_below stay dense bit rows, larger ones are returned as CSR.
    Returns a list of (graph, info)."""
    return [serve_pool_item(i, count, seed, nmin, nmax, dense_below) for i in range(count)]
