"""CPU oracle for weighted DAWN (arxiv 2306.07872) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
and never imports it.

The arithmetic lives in ``oracle.c`` (compiled with gcc, -ffp-contract=off)
plus three pure-Python / numpy routines kept here for independence:

* :func:`dense_colmin` -- the Section 3.1 construction: the matrix A_s of
  paths from s through each k, and the column minimum, iterated densely.
* :func:`brute_force` -- minimum over all simple paths of the left-fold path
  value, by exhaustive enumeration (tiny graphs only).
* :func:`fd_grad` -- central finite differences of L = sum c_t dist[t] with
  float64 Dijkstra.

Parity unpinned: the work counters that :func:`govm` and :func:`gsvm` return
(steps, edges scanned, updates, mu) beyond mu = 1 on unit weights; the
distances, parents and gradients are pinned by the tests.

Conventions shared with the library under test: unreachable distance is
0xFFFFFFFF for uint32 weights and +inf for float32 weights; parent[v] is the
tail of v's parent edge, parent[root] = root, parent[unreachable] = -1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None

U32_INF = np.uint32(0xFFFFFFFF)
U64_INF = np.uint64(0xFFFFFFFFFFFFFFFF)
I32_INF = np.int32(0x7FFFFFFF)     # unreachable, signed int32 weights
I64_INF = np.int64(0x7FFFFFFFFFFFFFFF)


class _Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in
                ("steps", "frontier_sum", "edges_scanned", "updates", "reached", "multi_updated", "converged")]


def build(force: bool = False) -> str:
    """Compile oracle.c into an in-tree shared library."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    for name in ("govm_u32", "govm_f32", "gsvm_u32", "gsvm_f32"):
        f = getattr(lib, name)
        f.argtypes = [i32, vp, vp, vp, vp, i32, vp, ctypes.POINTER(_Stats)]
        f.restype = ctypes.c_int
    for name in ("dijkstra_u32", "dijkstra_f32"):
        f = getattr(lib, name)
        f.argtypes = [i32, vp, vp, vp, vp, i32, vp]
        f.restype = ctypes.c_int
    lib.dijkstra_f64.argtypes = [i32, vp, vp, vp, i32, vp]
    lib.dijkstra_f64.restype = ctypes.c_int
    for name in ("fw_u32", "fw_f32"):
        f = getattr(lib, name)
        f.argtypes = [i32, vp, vp, vp, vp]
        f.restype = ctypes.c_int
    for name in ("parents_u32", "parents_f32"):
        f = getattr(lib, name)
        f.argtypes = [i32, vp, vp, vp, vp, i32, vp, vp]
        f.restype = ctypes.c_int
    for name in ("cert_u32", "cert_f32"):
        f = getattr(lib, name)
        f.argtypes = [i32, vp, vp, vp, vp, i32, vp, vp, ctypes.POINTER(i64)]
        f.restype = ctypes.c_int
    lib.subtree_grad_f64.argtypes = [i32, vp, i64, vp, vp, vp, vp]
    lib.subtree_grad_f64.restype = ctypes.c_int
    lib.govm_i32.argtypes = [i32, vp, vp, vp, vp, i32, vp, ctypes.POINTER(_Stats)]
    lib.govm_i32.restype = ctypes.c_int
    lib.bellman_ford_i32.argtypes = [i32, vp, vp, vp, vp, i32, vp]
    lib.bellman_ford_i32.restype = ctypes.c_int
    lib.parents_i32.argtypes = [i32, vp, vp, vp, vp, i32, vp, vp]
    lib.parents_i32.restype = ctypes.c_int
    lib.cert_i32.argtypes = [i32, vp, vp, vp, vp, i32, vp, vp, ctypes.POINTER(i64)]
    lib.cert_i32.restype = ctypes.c_int
    _lib = lib
    return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _graph(row_ptr, col, w):
    row_ptr = _c(row_ptr, np.int32)
    col = _c(col, np.int32)
    w = np.ascontiguousarray(w)
    if w.dtype == np.uint32:
        kind = "u32"
    elif w.dtype == np.float32:
        kind = "f32"
    elif w.dtype == np.int32:
        kind = "i32"
    else:
        raise TypeError("weights must be uint32, int32 or float32")
    return row_ptr, col, w, kind


def _roots(roots):
    return _c(np.atleast_1d(roots), np.int32)


def _u64_to_u32(d: np.ndarray) -> np.ndarray:
    """uint64 exact distances -> uint32 with 0xFFFFFFFF for unreachable."""
    fin = d != U64_INF
    if np.any(d[fin] >= np.uint64(0xFFFFFFFF)):
        raise OverflowError("a shortest distance does not fit below 0xFFFFFFFF")
    out = np.full(d.shape, U32_INF, dtype=np.uint32)
    out[fin] = d[fin].astype(np.uint32)
    return out


def _i64_to_i32(d: np.ndarray) -> np.ndarray:
    """int64 exact distances -> int32 with 0x7FFFFFFF for unreachable."""
    fin = d != I64_INF
    if np.any(d[fin] >= np.int64(I32_INF)) or np.any(d[fin] < np.int64(-2 ** 31)):
        raise OverflowError("a shortest distance does not fit in int32")
    out = np.full(d.shape, I32_INF, dtype=np.int32)
    out[fin] = d[fin].astype(np.int32)
    return out


def _i32_to_i64(d: np.ndarray) -> np.ndarray:
    d = _c(d, np.int32)
    out = d.astype(np.int64)
    out[d == I32_INF] = I64_INF
    return out


def _dist_in(d, kind):
    if kind == "u32":
        return _u32_to_u64(d)
    if kind == "i32":
        return _i32_to_i64(d)
    return _c(d, np.float32)


def _u32_to_u64(d: np.ndarray) -> np.ndarray:
    d = _c(d, np.uint32)
    out = d.astype(np.uint64)
    out[d == U32_INF] = U64_INF
    return out


# --------------------------------------------------------------- algorithms

def govm(row_ptr, col, w, roots, algorithm: str = "govm"):
    """Algorithm 2 (GOVM, Section 3.4) -- or Algorithm 1 (GSVM, Section 3.2)
    with algorithm="gsvm" -- executed literally.  Returns (dist, stats)."""
    lib = _load()
    row_ptr, col, w, kind = _graph(row_ptr, col, w)
    r = _roots(roots)
    n = len(row_ptr) - 1
    st = _Stats()
    fn = getattr(lib, f"{algorithm}_{kind}")
    alpha = np.empty(n, dtype={"u32": np.uint64, "i32": np.int64, "f32": np.float32}[kind])
    rc = fn(n, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data, r.ctypes.data, len(r), alpha.ctypes.data,
            ctypes.byref(st))
    if rc not in (0, 4):
        raise MemoryError(f"{algorithm} failed")
    stats = {f: getattr(st, f) for f, _ in _Stats._fields_}
    nonroot_reached = max(stats["reached"] - len(np.unique(r)), 0)
    stats["mu"] = stats["updates"] / nonroot_reached if nonroot_reached else 0.0
    dist = _u64_to_u32(alpha) if kind == "u32" else (_i64_to_i32(alpha) if kind == "i32" else alpha)
    return dist, stats


def gsvm(row_ptr, col, w, roots):
    return govm(row_ptr, col, w, roots, algorithm="gsvm")


def dijkstra(row_ptr, col, w, roots):
    """Binary-heap Dijkstra with lazy deletion (Section 2.1); same left-fold
    path values as the GOVM iteration."""
    lib = _load()
    row_ptr, col, w, kind = _graph(row_ptr, col, w)
    r = _roots(roots)
    n = len(row_ptr) - 1
    dist = np.empty(n, dtype=np.uint64 if kind == "u32" else np.float32)
    fn = getattr(lib, f"dijkstra_{kind}")
    if fn(n, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data, r.ctypes.data, len(r), dist.ctypes.data):
        raise MemoryError("dijkstra failed")
    return _u64_to_u32(dist) if kind == "u32" else dist


def bellman_ford(row_ptr, col, w, roots):
    """Textbook Bellman-Ford (Section 2.2) for signed int32 weights; returns
    (dist, negative_cycle_reachable)."""
    lib = _load()
    row_ptr, col, w, kind = _graph(row_ptr, col, w)
    if kind != "i32":
        raise TypeError("bellman_ford expects int32 weights")
    r = _roots(roots)
    n = len(row_ptr) - 1
    dist = np.empty(n, dtype=np.int64)
    rc = lib.bellman_ford_i32(n, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data, r.ctypes.data, len(r),
                              dist.ctypes.data)
    if rc < 0:
        raise MemoryError("bellman_ford failed")
    if rc == 4:
        return None, True
    return _i64_to_i32(dist), False


def floyd_warshall(row_ptr, col, w):
    """Dense all-pairs matrix (Section 2.3).  Tiny graphs only."""
    lib = _load()
    row_ptr, col, w, kind = _graph(row_ptr, col, w)
    n = len(row_ptr) - 1
    D = np.empty((n, n), dtype=np.uint64 if kind == "u32" else np.float32)
    getattr(lib, f"fw_{kind}")(n, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data, D.ctypes.data)
    return _u64_to_u32(D) if kind == "u32" else D


def parent_edges(row_ptr, col, w, roots, dist):
    """Lowest CSR edge index e=(u->v) with fl(dist[u]+w[e]) == dist[v]; -1 for
    roots and unreachable vertices."""
    lib = _load()
    row_ptr, col, w, kind = _graph(row_ptr, col, w)
    r = _roots(roots)
    n = len(row_ptr) - 1
    d = _dist_in(dist, kind)
    pe = np.empty(n, dtype=np.int32)
    getattr(lib, f"parents_{kind}")(n, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data, r.ctypes.data, len(r),
                                    d.ctypes.data, pe.ctypes.data)
    return pe


def edge_tails(row_ptr) -> np.ndarray:
    """tail (source row) of every CSR edge."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    return np.repeat(np.arange(len(row_ptr) - 1, dtype=np.int32), np.diff(row_ptr))


def parent_vertices(row_ptr, roots, dist, parent_edge, kind: str) -> np.ndarray:
    """parent vertex: tail of the parent edge, root for roots, -1 unreachable."""
    n = len(row_ptr) - 1
    tails = edge_tails(row_ptr)
    p = np.full(n, -1, dtype=np.int32)
    has = parent_edge >= 0
    p[has] = tails[parent_edge[has]]
    p[_roots(roots)] = _roots(roots)
    return p


def sssp(row_ptr, col, w, roots, algorithm: str = "dijkstra"):
    """(dist, parent, parent_edge) for one solve with the given roots."""
    if np.asarray(w).dtype == np.int32:  # signed weights: Dijkstra does not apply
        dist, neg = bellman_ford(row_ptr, col, w, roots) if algorithm == "dijkstra" else (
            govm(row_ptr, col, w, roots)[0], False)
        if neg:
            raise ValueError("a negative cycle is reachable from the roots")
    elif algorithm == "dijkstra":
        dist = dijkstra(row_ptr, col, w, roots)
    else:
        dist, _ = govm(row_ptr, col, w, roots, algorithm=algorithm)
    pe = parent_edges(row_ptr, col, w, roots, dist)
    kind = "u32" if np.asarray(w).dtype == np.uint32 else "f32"
    return dist, parent_vertices(row_ptr, roots, dist, pe, kind), pe


CERT_CODES = {0: "ok", 1: "root has non-zero distance or a parent edge",
              2: "an edge can still be relaxed", 3: "invalid parent edge",
              4: "unreachable vertex has a parent edge", 5: "parent edges form a cycle"}


def certificate(row_ptr, col, w, roots, dist, parent_edge):
    """(code, where) of the optimality certificate; code 0 means dist is the
    exact fixpoint and parent_edge a valid shortest-path forest."""
    lib = _load()
    row_ptr, col, w, kind = _graph(row_ptr, col, w)
    r = _roots(roots)
    n = len(row_ptr) - 1
    d = _dist_in(dist, kind)
    pe = _c(parent_edge, np.int32)
    where = ctypes.c_int64(-1)
    rc = getattr(lib, f"cert_{kind}")(n, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data, r.ctypes.data,
                                      len(r), d.ctypes.data, pe.ctypes.data, ctypes.byref(where))
    if rc < 0:
        raise MemoryError("certificate failed")
    return rc, where.value


# ----------------------------------------------------------- pure Python / numpy

def dense_colmin(row_ptr, col, w, source):
    """Section 3.1: a_s starts with a_{s,s}=0; each round forms the matrix
    A_s[k, j] = a_s[k] + a[k, j] (the path from s fixed up to k, extended by
    one edge k -> j) and takes the minimum of each column together with the
    current a_s; rounds repeat until nothing changes.  Dense and O(n^2) per
    round: tiny graphs only.  float32 weights use fl32 addition; uint32 are
    exact."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col)
    w = np.asarray(w)
    n = len(row_ptr) - 1
    kind = "u32" if w.dtype == np.uint32 else "f32"
    big = np.inf
    A = np.full((n, n), big, dtype=np.float64 if kind == "u32" else np.float32)
    for u in range(n):
        for e in range(row_ptr[u], row_ptr[u + 1]):
            v = col[e]
            val = float(w[e]) if kind == "u32" else np.float32(w[e])
            if val < A[u, v]:
                A[u, v] = val
    a = np.full(n, big, dtype=A.dtype)
    a[source] = 0
    for _ in range(n + 1):
        As = a[:, None] + A            # As[k, j] = a_s[k] + a[k, j]
        new = np.minimum(a, As.min(axis=0))
        new[source] = 0                # paths back into s are never taken
        if np.array_equal(new, a):
            break
        a = new
    if kind == "u32":
        out = np.full(n, U32_INF, dtype=np.uint32)
        fin = np.isfinite(a)
        out[fin] = a[fin].astype(np.uint64).astype(np.uint32)
        return out
    return a.astype(np.float32)


def brute_force(row_ptr, col, w, source):
    """min over all simple paths s -> v of the left fold of the edge weights
    (fl32 for float32, exact for integers); tiny graphs (n <= 9) only.  With
    signed weights this is the shortest distance only when no negative cycle
    is reachable."""
    row_ptr = [int(x) for x in row_ptr]
    col = [int(x) for x in col]
    w = np.asarray(w)
    n = len(row_ptr) - 1
    f32 = w.dtype == np.float32
    best = [None] * n
    best[source] = np.float32(0) if f32 else 0

    def walk(u, val, seen):
        for e in range(row_ptr[u], row_ptr[u + 1]):
            v = col[e]
            if v in seen:
                continue
            nv = np.float32(val + w[e]) if f32 else val + int(w[e])
            if best[v] is None or nv < best[v]:
                best[v] = nv
            walk(v, nv, seen | {v})

    walk(source, best[source], {source})
    if f32:
        return np.array([np.inf if b is None else b for b in best], dtype=np.float32)
    if w.dtype == np.int32:
        return np.array([int(I32_INF) if b is None else b for b in best], dtype=np.int32)
    return np.array([0xFFFFFFFF if b is None else b for b in best], dtype=np.uint32)


def dijkstra64(row_ptr, col, w64, source):
    lib = _load()
    row_ptr = _c(row_ptr, np.int32)
    col = _c(col, np.int32)
    w64 = _c(w64, np.float64)
    n = len(row_ptr) - 1
    d = np.empty(n, dtype=np.float64)
    if lib.dijkstra_f64(n, row_ptr.ctypes.data, col.ctypes.data, w64.ctypes.data, int(source), d.ctypes.data):
        raise MemoryError("dijkstra_f64 failed")
    return d


def subtree_grad(row_ptr, col, w, source, c, dist=None, parent_edge=None):
    """float64 dL/dw for L = sum_v c[v] * dist[v]: for a tree edge e into v,
    the sum of c over v's subtree; 0 off the tree.  Uses the oracle's
    float64 distances and lowest-index parent edges."""
    lib = _load()
    row_ptr = _c(row_ptr, np.int32)
    n = len(row_ptr) - 1
    m = int(row_ptr[-1])
    w64 = np.asarray(w, dtype=np.float64)
    d64 = dijkstra64(row_ptr, col, w64, source)
    if parent_edge is None:
        if dist is None:
            dist = dijkstra(row_ptr, col, w, source)
        parent_edge = parent_edges(row_ptr, col, w, source, dist)
    order = np.argsort(-np.where(np.isfinite(d64), d64, -1.0), kind="stable").astype(np.int32)
    c = _c(c, np.float64)
    g = np.empty(m, dtype=np.float64)
    pe = _c(parent_edge, np.int32)
    if lib.subtree_grad_f64(n, row_ptr.ctypes.data, m, pe.ctypes.data, order.ctypes.data, c.ctypes.data,
                            g.ctypes.data):
        raise MemoryError("subtree_grad failed")
    return g


def _parents64(row_ptr, col, w64, d, source):
    """float64 lowest-index tight parent edge of every vertex (-1 if none)."""
    n = len(row_ptr) - 1
    col = np.asarray(col)
    tails = edge_tails(row_ptr)
    tight = np.isfinite(d[tails]) & (d[tails] + w64 == d[col]) & (col != source)
    idx = np.nonzero(tight)[0]
    pe = np.full(n, np.iinfo(np.int64).max, dtype=np.int64)
    np.minimum.at(pe, col[idx], idx)
    pe[pe == np.iinfo(np.int64).max] = -1
    return pe


def fd_grad(row_ptr, col, w, source, c, edges, h: float = 1e-3):
    """Central differences (L(w + h e_i) - L(w - h e_i)) / 2h in float64 for
    the listed edges, L = sum_v c[v] dist[v] over reachable v.  Also returns,
    per edge, whether both perturbations kept the float64 shortest-path tree
    (lowest-index tight parent edges) identical to the unperturbed one; the
    finite difference is a valid check only where it did."""
    w64 = np.asarray(w, dtype=np.float64).copy()
    c = np.asarray(c, dtype=np.float64)
    base = dijkstra64(row_ptr, col, w64, source)
    fin = np.isfinite(base)
    t0 = _parents64(row_ptr, col, w64, base, source)

    def loss(d):
        return float(np.sum(c[fin] * d[fin]))

    out = np.zeros(len(edges))
    stable = np.zeros(len(edges), dtype=bool)
    for i, e in enumerate(edges):
        wp = w64.copy()
        wp[e] += h
        wm = w64.copy()
        wm[e] -= h
        dp = dijkstra64(row_ptr, col, wp, source)
        dm = dijkstra64(row_ptr, col, wm, source)
        out[i] = (loss(dp) - loss(dm)) / (2 * h)
        stable[i] = (np.array_equal(_parents64(row_ptr, col, wp, dp, source), t0)
                     and np.array_equal(_parents64(row_ptr, col, wm, dm, source), t0))
    return out, stable


def timed_govm(row_ptr, col, w, roots_list, threads: int = 1):
    """Run the literal GOVM iteration for each root set in `roots_list` on up
    to `threads` host threads (the C call releases the GIL).  Returns
    (seconds, list of (dist, stats))."""
    from concurrent.futures import ThreadPoolExecutor
    _load()
    t0 = time.perf_counter()
    if threads <= 1:
        res = [govm(row_ptr, col, w, r) for r in roots_list]
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            res = list(ex.map(lambda r: govm(row_ptr, col, w, r), roots_list))
    return time.perf_counter() - t0, res
