"""Seeded synthetic graph workloads shared by the oracle tests, the GPU tests
and the benchmark.

This module holds none of the shortest-path arithmetic: it draws graphs and
weights from one counter-based generator (splitmix64 output function on a
(seed, stream, counter) key, implemented in ``graphgen.c``) and performs
structural bookkeeping only (CSR assembly, de-duplication, weakly connected
components, unweighted reachability) used to choose sources and targets.

The workloads stand in for the SNAP / SuiteSparse graphs of the paper's
Section 4 (Table 2, 36 general + 12 large graphs), which are not available:
power-law R-MAT graphs, Erdos-Renyi graphs, a high-diameter grid and a batch
of uneven graphs.  Weight distributions follow the paper's validation
experiment (Section 4.2: fp32 weights in [0, 2] against unit weights) and the
integer / log-uniform ranges of the workload definitions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "_graphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into an in-tree shared library (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.POINTER
    i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    vp = ctypes.c_void_p
    lib.gg_free.argtypes = [vp]
    lib.gg_draws.argtypes = [u64, u64, u64, i64, vp]
    lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int, dbl, dbl, dbl, u64, ctypes.c_int,
                            P(i32), P(i64), P(vp), P(vp)]
    lib.gg_rmat.restype = ctypes.c_int
    lib.gg_er.argtypes = [i32, i64, u64, P(i64), P(vp), P(vp)]
    lib.gg_er.restype = ctypes.c_int
    lib.gg_grid.argtypes = [i32, dbl, u64, P(i64), P(vp), P(vp), P(vp)]
    lib.gg_grid.restype = ctypes.c_int
    lib.gg_weights_u32.argtypes = [i64, ctypes.c_uint32, ctypes.c_uint32, u64, vp]
    lib.gg_weights_f32_uniform.argtypes = [i64, dbl, dbl, u64, vp]
    lib.gg_weights_f32_loguniform.argtypes = [i64, dbl, dbl, u64, vp]
    lib.gg_wcc.argtypes = [i32, vp, vp, vp]
    lib.gg_wcc.restype = i32
    lib.gg_reachable.argtypes = [i32, vp, vp, i32, vp]
    lib.gg_reachable.restype = i32
    _lib = lib
    return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _take(ptr, count: int, dtype) -> np.ndarray:
    """Copy a malloc'd C array into numpy and free it."""
    lib = _load()
    if count == 0:
        lib.gg_free(ptr)
        return np.zeros(0, dtype=dtype)
    raw = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_uint8)),
                                shape=(count * np.dtype(dtype).itemsize,))
    out = raw.view(dtype).copy()
    lib.gg_free(ptr)
    return out


# ------------------------------------------------------------------ primitives

def draws(seed: int, stream: int, count: int, ctr0: int = 0) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    if count:
        _load().gg_draws(seed, stream, ctr0, count, _ptr(out))
    return out


def uniform01(seed: int, stream: int, count: int, ctr0: int = 0) -> np.ndarray:
    return (draws(seed, stream, count, ctr0) >> np.uint64(11)).astype(np.float64) * (1.0 / 2.0 ** 53)


def below(seed: int, stream: int, count: int, bound: int, ctr0: int = 0) -> np.ndarray:
    """Integers in [0, bound) by multiply-shift of the top 32 bits."""
    x = draws(seed, stream, count, ctr0) >> np.uint64(32)
    return ((x * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)


def rmat(scale: int, edge_factor: int = 16, a=0.57, b=0.19, c=0.19, seed: int = 0, relabel: bool = True):
    lib = _load()
    n = ctypes.c_int32()
    m = ctypes.c_int64()
    rp = ctypes.c_void_p()
    cl = ctypes.c_void_p()
    rc = lib.gg_rmat(scale, edge_factor, a, b, c, seed, int(relabel), ctypes.byref(n), ctypes.byref(m),
                     ctypes.byref(rp), ctypes.byref(cl))
    if rc != 0:
        raise MemoryError("gg_rmat failed")
    return _take(rp.value, n.value + 1, np.int32), _take(cl.value, m.value, np.int32)


def erdos_renyi(n: int, M: int, seed: int = 0):
    lib = _load()
    m = ctypes.c_int64()
    rp = ctypes.c_void_p()
    cl = ctypes.c_void_p()
    rc = lib.gg_er(n, M, seed, ctypes.byref(m), ctypes.byref(rp), ctypes.byref(cl))
    if rc != 0:
        raise ValueError("gg_er failed (bad n/M or out of memory)")
    return _take(rp.value, n + 1, np.int32), _take(cl.value, m.value, np.int32)


def grid(side: int, shortcut_frac: float = 0.01, seed: int = 0):
    lib = _load()
    m = ctypes.c_int64()
    rp = ctypes.c_void_p()
    cl = ctypes.c_void_p()
    fl = ctypes.c_void_p()
    rc = lib.gg_grid(side, shortcut_frac, seed, ctypes.byref(m), ctypes.byref(rp), ctypes.byref(cl),
                     ctypes.byref(fl))
    if rc != 0:
        raise MemoryError("gg_grid failed")
    n = side * side
    return (_take(rp.value, n + 1, np.int32), _take(cl.value, m.value, np.int32),
            _take(fl.value, m.value, np.uint8).astype(bool))


def weights_u32(m: int, lo: int, hi: int, seed: int) -> np.ndarray:
    w = np.empty(m, dtype=np.uint32)
    if m:
        _load().gg_weights_u32(m, lo, hi, seed, _ptr(w))
    return w


def weights_f32_uniform(m: int, lo: float, hi: float, seed: int) -> np.ndarray:
    w = np.empty(m, dtype=np.float32)
    if m:
        _load().gg_weights_f32_uniform(m, lo, hi, seed, _ptr(w))
    return w


def weights_f32_loguniform(m: int, lo: float, hi: float, seed: int) -> np.ndarray:
    w = np.empty(m, dtype=np.float32)
    if m:
        _load().gg_weights_f32_loguniform(m, lo, hi, seed, _ptr(w))
    return w


def wcc_labels(row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    n = len(row_ptr) - 1
    label = np.empty(n, dtype=np.int32)
    _load().gg_wcc(n, _ptr(np.ascontiguousarray(row_ptr)), _ptr(np.ascontiguousarray(col)), _ptr(label))
    return label


def reachable(row_ptr: np.ndarray, col: np.ndarray, source: int) -> np.ndarray:
    n = len(row_ptr) - 1
    r = np.empty(n, dtype=np.uint8)
    _load().gg_reachable(n, _ptr(np.ascontiguousarray(row_ptr)), _ptr(np.ascontiguousarray(col)), source,
                         _ptr(r))
    return r.astype(bool)


def sample_without_replacement(pool: np.ndarray, k: int, seed: int, stream: int = 0) -> np.ndarray:
    """k distinct elements of `pool` by a partial Fisher-Yates shuffle."""
    pool = np.array(pool, copy=True)
    k = min(k, len(pool))
    if k == 0:
        return pool[:0]
    x = draws(seed, stream, k) >> np.uint64(32)
    for i in range(k):
        j = i + int((int(x[i]) * (len(pool) - i)) >> 32)
        pool[i], pool[j] = pool[j], pool[i]
    return pool[:k].copy()


# ------------------------------------------------------------------ workloads

@dataclass
class Workload:
    """A graph in CSR form with weights, sources and workload metadata."""
    name: str
    row_ptr: np.ndarray          # int32[n+1]
    col: np.ndarray              # int32[m]
    weights: np.ndarray          # uint32[m] or float32[m]
    sources: np.ndarray          # int32[k]
    e_wcc: int                   # edges inside the largest weakly connected component
    s_wcc: int                   # vertices inside the largest weakly connected component
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def m(self) -> int:
        return len(self.col)

    @property
    def wtype(self) -> str:
        return "u32" if self.weights.dtype == np.uint32 else "f32"


def largest_wcc(row_ptr: np.ndarray, col: np.ndarray):
    """(mask of vertices in the largest WCC, its vertex count, its edge count)."""
    label = wcc_labels(row_ptr, col)
    counts = np.bincount(label, minlength=len(label))
    big = int(np.argmax(counts))
    mask = label == big
    deg = np.diff(row_ptr.astype(np.int64))
    return mask, int(counts[big]), int(deg[mask].sum())


def wcc_sources(row_ptr, col, k: int, seed: int):
    """k distinct sources uniform over largest-WCC vertices with out-degree >= 1."""
    mask, s_wcc, e_wcc = largest_wcc(row_ptr, col)
    deg = np.diff(row_ptr)
    pool = np.nonzero(mask & (deg > 0))[0].astype(np.int32)
    return sample_without_replacement(pool, k, seed).astype(np.int32), s_wcc, e_wcc


def tiny_er(n: int = 1024, avg_deg: int = 8, seed: int = 0, wlo: int = 1, whi: int = 100) -> Workload:
    """Directed G(n, M=n*avg_deg) with u32 weights U[wlo, whi], source 0."""
    rp, cl = erdos_renyi(n, n * avg_deg, seed)
    w = weights_u32(len(cl), wlo, whi, seed + 1)
    _, s_wcc, e_wcc = largest_wcc(rp, cl)
    return Workload(f"er_n{n}_d{avg_deg}", rp, cl, w, np.array([0], np.int32), e_wcc, s_wcc)


def rmat_u32(scale: int, edge_factor: int = 16, nsrc: int = 64, seed: int = 0, wlo: int = 1,
             whi: int = 255) -> Workload:
    """R-MAT (.57,.19,.19,.05), relabelled, u32 weights U[wlo, whi] (seed+1),
    nsrc sources from the largest WCC with out-degree >= 1 (seed+2)."""
    rp, cl = rmat(scale, edge_factor, seed=seed, relabel=True)
    w = weights_u32(len(cl), wlo, whi, seed + 1)
    src, s_wcc, e_wcc = wcc_sources(rp, cl, nsrc, seed + 2)
    return Workload(f"rmat_s{scale}_ef{edge_factor}_u32", rp, cl, w, src, e_wcc, s_wcc)


def grid_f32(side: int = 2048, shortcut_frac: float = 0.01, nsrc: int = 16, seed: int = 0) -> Workload:
    """side^2 4-neighbour grid, fp32 log-uniform [0.1, 10] weights (seed+1),
    plus shortcut_frac * grid-edges shortcuts of weight 50 (seed), nsrc
    sources from the largest WCC (seed+2)."""
    rp, cl, sc = grid(side, shortcut_frac, seed)
    w = weights_f32_loguniform(len(cl), 0.1, 10.0, seed + 1)
    w[sc] = np.float32(50.0)
    src, s_wcc, e_wcc = wcc_sources(rp, cl, nsrc, seed + 2)
    return Workload(f"grid_{side}x{side}_f32", rp, cl, w, src, e_wcc, s_wcc,
                    extra={"shortcuts": int(sc.sum())})


def er_batch(count: int = 64, nlo: int = 1000, nhi: int = 262144, dlo: int = 4, dhi: int = 32,
             seed: int = 0) -> Workload:
    """`count` independent G(n_i, n_i*d_i) graphs, n_i log-uniform in [nlo, nhi],
    d_i uniform integer in [dlo, dhi], u32 weights U[1,255]; concatenated into
    one disjoint-union CSR.  sources[i] = node 0 of graph i."""
    u = uniform01(seed, 7, count)
    ns = np.rint(np.exp(np.log(nlo) + (np.log(nhi) - np.log(nlo)) * u)).astype(np.int64)
    ds = dlo + below(seed, 8, count, dhi - dlo + 1)
    rps, cls, offs = [], [], []
    voff = 0
    eoff = 0
    parts = []
    for i in range(count):
        rp, cl = erdos_renyi(int(ns[i]), int(ns[i] * ds[i]), seed * 1000 + 100 + i)
        rps.append(rp[:-1].astype(np.int64) + eoff)
        cls.append(cl.astype(np.int64) + voff)
        offs.append(voff)
        parts.append((int(ns[i]), len(cl)))
        voff += int(ns[i])
        eoff += len(cl)
    row_ptr = np.concatenate(rps + [np.array([eoff])]).astype(np.int32)
    col = np.concatenate(cls).astype(np.int32)
    w = weights_u32(len(col), 1, 255, seed + 1)
    src = np.array(offs, dtype=np.int32)
    _, s_wcc, e_wcc = largest_wcc(row_ptr, col)
    return Workload(f"er_batch{count}", row_ptr, col, w, src, e_wcc, s_wcc,
                    extra={"parts": parts, "offsets": np.array(offs + [voff], dtype=np.int64)})


def rmat_f32_diff(scale: int = 16, edge_factor: int = 16, ntargets: int = 256, seed: int = 0) -> Workload:
    """R-MAT without relabelling (node 0 is the main hub), fp32 weights
    U[0.5, 2.0] (seed+1), source 0, `ntargets` targets uniform among vertices
    reachable from 0 (seed+3, excluding 0) with loss coefficients c_t ~ N(0,1)
    (Box-Muller on draws of seed+3 stream 1)."""
    rp, cl = rmat(scale, edge_factor, seed=seed, relabel=False)
    w = weights_f32_uniform(len(cl), 0.5, 2.0, seed + 1)
    reach = reachable(rp, cl, 0)
    reach[0] = False
    pool = np.nonzero(reach)[0].astype(np.int32)
    targets = sample_without_replacement(pool, ntargets, seed + 3)
    u = uniform01(seed + 3, 1, 2 * len(targets))
    u1 = np.maximum(u[0::2], 1e-300)
    coef = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u[1::2])
    _, s_wcc, e_wcc = largest_wcc(rp, cl)
    return Workload(f"rmat_s{scale}_ef{edge_factor}_f32", rp, cl, w, np.array([0], np.int32), e_wcc, s_wcc,
                    extra={"targets": targets, "coef": coef})


def csr_from_edges(n: int, edges, weights, dtype=np.uint32):
    """CSR (row_ptr, col, w) from a list of (u, v) pairs and their weights.
    Edges are grouped by tail with a stable sort, so edges of one row keep
    the order in which they were listed (parallel edges and self-loops are
    kept as given)."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.asarray(weights, dtype=dtype).reshape(-1)
    order = np.argsort(edges[:, 0], kind="stable")
    e = edges[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, e[:, 0] + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return row_ptr, e[:, 1].astype(np.int32), w[order].copy()


def random_small(n: int, m: int, seed: int, kind: str = "u32", wlo=1, whi=20, self_loops=False):
    """Tiny random multigraph for exhaustive checks: m edges (u, v) drawn
    uniformly (parallel edges allowed), u32 weights U[wlo, whi] or fp32
    weights uniform in [wlo, whi]."""
    x = draws(seed, 11, 2 * m)
    u = ((x[0::2] >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
    v = ((x[1::2] >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
    edges = np.stack([u, v], 1).astype(np.int64)
    if not self_loops:
        edges = edges[edges[:, 0] != edges[:, 1]]
    k = len(edges)
    if kind == "u32":
        w = (wlo + below(seed, 12, k, whi - wlo + 1)).astype(np.uint32)
        return csr_from_edges(n, edges, w, np.uint32)
    if kind == "dyadic":
        w = ((wlo + below(seed, 12, k, (whi - wlo) * 16 + 1) / 16.0)).astype(np.float32)
        return csr_from_edges(n, edges, w, np.float32)
    w = (wlo + (whi - wlo) * uniform01(seed, 12, k)).astype(np.float32)
    return csr_from_edges(n, edges, w, np.float32)
