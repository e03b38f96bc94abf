"""Thin Python binding of libdawn (include/dawn.h).

The functions below carry the C entry points' names and only marshal
arguments (torch tensors to device pointers, the current CUDA stream) and
turn non-zero status codes into :class:`DawnError`.  Every step of the
shortest-path computation runs in the CUDA kernels of libdawn.so; there is no
CPU fallback, and importing this module without the built library fails.

On top of the raw names sit two conveniences: :class:`Graph` (owns a handle
and allocates output tensors) and :class:`DawnSSSP`, a
``torch.autograd.Function`` whose forward is the GOVM solver and whose
backward is the library's parent-tree scatter kernel.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdawn.so")

DAWN_W_U32, DAWN_W_F32, DAWN_W_I32 = 0, 1, 2
DAWN_OK, DAWN_ERR_INVALID, DAWN_ERR_OOM, DAWN_ERR_CUDA = 0, 1, 2, 3
DAWN_ERR_NOT_CONVERGED, DAWN_ERR_TIMEOUT, DAWN_ERR_BOUNDS = 4, 5, 6
DAWN_OPT_MAX_STEPS, DAWN_OPT_WAIT_LIMIT_NS, DAWN_OPT_GRID_BLOCKS, DAWN_OPT_TEST_STALL = 1, 2, 3, 4
DAWN_OPT_TRACE_STEPS = 5
DAWN_OPT_GSVM = 6
DAWN_OPT_CTAS_PER_SM, DAWN_OPT_BATCH, DAWN_OPT_TEST_FAIL_ALLOC, DAWN_OPT_SMALL_PATH = 7, 8, 9, 10
DAWN_OPT_FRONTIER = 11
DAWN_OPT_SKIP_REMARKED = 12
DAWN_FRONTIER_AUTO, DAWN_FRONTIER_QUEUE, DAWN_FRONTIER_BITMAP = 0, 1, 2
DAWN_SMALL_AUTO, DAWN_SMALL_NEVER, DAWN_SMALL_WHEN_STATE_FITS = 0, 1, 2
DAWN_TUNE_SSSP, DAWN_TUNE_MSSSP, DAWN_TUNE_ROOTS = 0, 1, 2
DAWN_WEIGHTS_ON_DEVICE, DAWN_WEIGHTS_DEFER_CHECK = 1, 2

EXPORTS = ("dawn_create_graph", "dawn_set_weights", "dawn_reserve", "dawn_sssp", "dawn_msssp", "dawn_sssp_roots",
           "dawn_sssp_backward", "dawn_status", "dawn_get_stats", "dawn_set_option", "dawn_get_trace", "dawn_graph_info",
           "dawn_status_string", "dawn_destroy", "dawn_trim_memory", "dawn_sssp_noalloc", "dawn_autotune")


class DawnError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)}")


class _Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("steps", "frontier_sum", "edges_scanned", "updates", "instances",
                                              "edges_skipped")]


class _Tuning(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("grid_blocks", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("best_ms", ctypes.c_float), ("default_ms", ctypes.c_float),
                ("small_path", ctypes.c_int32), ("frontier", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libdawn.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2306_07872_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, c_int = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int
    sig = {
        "dawn_create_graph": ([i32, i64, vp, vp, vp, c_int, c_int, vp, ctypes.POINTER(vp)], c_int),
        "dawn_set_weights": ([vp, vp, c_int, vp], c_int),
        "dawn_reserve": ([vp, i32], c_int),
        "dawn_sssp": ([vp, i32, vp, vp, vp, vp], c_int),
        "dawn_msssp": ([vp, vp, i32, vp, vp, vp], c_int),
        "dawn_sssp_roots": ([vp, vp, i32, vp, vp, vp, vp], c_int),
        "dawn_sssp_backward": ([vp, vp, vp, vp, vp], c_int),
        "dawn_status": ([vp, c_int], c_int),
        "dawn_get_stats": ([vp, ctypes.POINTER(_Stats)], c_int),
        "dawn_set_option": ([vp, c_int, i64], c_int),
        "dawn_get_trace": ([vp, vp, i32], c_int),
        "dawn_graph_info": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(c_int)], c_int),
        "dawn_status_string": ([c_int], ctypes.c_char_p),
        "dawn_destroy": ([vp], None),
        "dawn_trim_memory": ([], c_int),
        "dawn_sssp_noalloc": ([vp, i32, vp, vp, vp, vp, vp], c_int),
        "dawn_autotune": ([vp, c_int, vp, i32, i32, vp, ctypes.POINTER(_Tuning)], c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load_library().dawn_status_string(int(code)).decode()


def _check(code: int, where: str):
    if code != DAWN_OK:
        raise DawnError(code, where)


def _stream(stream) -> ctypes.c_void_p:
    """cudaStream_t of `stream`: None (torch's current stream), a
    torch.cuda.Stream, an already marshalled c_void_p or an integer handle."""
    if isinstance(stream, ctypes.c_void_p):
        return stream
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev(t: torch.Tensor | None, dtype=None, name="tensor") -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _any(t: torch.Tensor, dtype, name) -> tuple[ctypes.c_void_p, int]:
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr()), int(t.is_cuda)


# ------------------------------------------------------------- raw entry points

def dawn_create_graph(row_ptr: torch.Tensor, col_idx: torch.Tensor, weights: torch.Tensor, stream=None) -> int:
    """Create a graph from CSR tensors (CPU or CUDA, int32 / int32 / uint32 or
    float32); returns the opaque handle."""
    lib = load_library()
    n = row_ptr.numel() - 1
    m = col_idx.numel()
    if weights.dtype == torch.uint32:
        wt = DAWN_W_U32
    elif weights.dtype == torch.float32:
        wt = DAWN_W_F32
    elif weights.dtype == torch.int32:
        wt = DAWN_W_I32
    else:
        raise TypeError("weights must be torch.uint32, torch.int32 or torch.float32")
    rp, on_dev = _any(row_ptr, torch.int32, "row_ptr")
    cl, d2 = _any(col_idx, torch.int32, "col_idx")
    w, d3 = _any(weights, weights.dtype, "weights")
    if len({on_dev, d2, d3}) != 1:
        raise ValueError("row_ptr, col_idx and weights must all be on the host or all on the device")
    h = ctypes.c_void_p()
    _check(lib.dawn_create_graph(n, m, rp, cl, w, wt, on_dev, _stream(stream), ctypes.byref(h)), "dawn_create_graph")
    return h.value


def dawn_set_weights(g: int, weights: torch.Tensor, stream=None, defer_check: bool = False):
    w, on_dev = _any(weights, weights.dtype, "weights")
    flags = (DAWN_WEIGHTS_ON_DEVICE if on_dev else 0) | (DAWN_WEIGHTS_DEFER_CHECK if defer_check else 0)
    _check(load_library().dawn_set_weights(ctypes.c_void_p(g), w, flags, _stream(stream)), "dawn_set_weights")


def dawn_reserve(g: int, k: int):
    _check(load_library().dawn_reserve(ctypes.c_void_p(g), int(k)), "dawn_reserve")


def dawn_sssp(g: int, source: int, dist: torch.Tensor, parent=None, parent_edge=None, stream=None):
    _check(load_library().dawn_sssp(ctypes.c_void_p(g), int(source), _dev(dist, name="dist"),
                                    _dev(parent, torch.int32, "parent"), _dev(parent_edge, torch.int32, "parent_edge"),
                                    _stream(stream)), "dawn_sssp")


def dawn_sssp_noalloc(g: int, source: int, dist: torch.Tensor, parent=None, parent_edge=None, status_out=None,
                      stream=None):
    """dawn_sssp without any allocation: the workspace comes from the
    library's fixed 32 MiB device array (see include/dawn.h)."""
    _check(load_library().dawn_sssp_noalloc(ctypes.c_void_p(g), int(source), _dev(dist, name="dist"),
                                            _dev(parent, torch.int32, "parent"),
                                            _dev(parent_edge, torch.int32, "parent_edge"),
                                            _dev(status_out, torch.int32, "status_out"), _stream(stream)),
           "dawn_sssp_noalloc")


def dawn_msssp(g: int, sources: torch.Tensor, dist: torch.Tensor, parent=None, stream=None):
    _check(load_library().dawn_msssp(ctypes.c_void_p(g), _dev(sources, torch.int32, "sources"), sources.numel(),
                                     _dev(dist, name="dist"), _dev(parent, torch.int32, "parent"), _stream(stream)),
           "dawn_msssp")


def dawn_sssp_roots(g: int, roots: torch.Tensor, dist: torch.Tensor, parent=None, parent_edge=None, stream=None):
    _check(load_library().dawn_sssp_roots(ctypes.c_void_p(g), _dev(roots, torch.int32, "roots"), roots.numel(),
                                          _dev(dist, name="dist"), _dev(parent, torch.int32, "parent"),
                                          _dev(parent_edge, torch.int32, "parent_edge"), _stream(stream)),
           "dawn_sssp_roots")


def dawn_sssp_backward(g: int, parent_edge: torch.Tensor, grad_dist: torch.Tensor, grad_w: torch.Tensor, stream=None):
    _check(load_library().dawn_sssp_backward(ctypes.c_void_p(g), _dev(parent_edge, torch.int32, "parent_edge"),
                                             _dev(grad_dist, torch.float32, "grad_dist"),
                                             _dev(grad_w, torch.float32, "grad_w"), _stream(stream)),
           "dawn_sssp_backward")


def dawn_status(g: int, sync: bool = True) -> int:
    return int(load_library().dawn_status(ctypes.c_void_p(g), int(bool(sync))))


def dawn_get_stats(g: int) -> dict:
    st = _Stats()
    _check(load_library().dawn_get_stats(ctypes.c_void_p(g), ctypes.byref(st)), "dawn_get_stats")
    return {f: getattr(st, f) for f, _ in _Stats._fields_}


def dawn_set_option(g: int, option: int, value: int):
    _check(load_library().dawn_set_option(ctypes.c_void_p(g), int(option), int(value)), "dawn_set_option")


def dawn_autotune(g: int, mode: int, sources, reps: int = 3, stream=None) -> dict:
    """Time candidate launch configurations on `sources` (host int32 ids) and
    keep the fastest as the handle's options; returns the chosen
    configuration and its timing.  Synchronous."""
    import numpy as np
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
    tun = _Tuning()
    _check(load_library().dawn_autotune(ctypes.c_void_p(g), int(mode), ctypes.c_void_p(src.ctypes.data),
                                        int(src.size), int(reps), _stream(stream), ctypes.byref(tun)),
           "dawn_autotune")
    return {f: getattr(tun, f) for f, _ in _Tuning._fields_}


def dawn_get_trace(g: int, cap: int = 4096):
    """Per-step rows of the last solve: list of (t_ns, frontier, edges) per
    step, derived from the cumulative device trace."""
    import numpy as np
    buf = np.zeros(4 * cap, dtype=np.int64)
    rows = load_library().dawn_get_trace(ctypes.c_void_p(g), ctypes.c_void_p(buf.ctypes.data), int(cap))
    if rows < 0:
        raise DawnError(-rows, "dawn_get_trace")
    t = buf.reshape(-1, 4)[:rows]
    out = []
    for i in range(rows - 1):
        out.append((int(t[i + 1, 0] - t[i, 0]), int(t[i + 1, 1] - t[i, 1]), int(t[i + 1, 2] - t[i, 2])))
    return out


def dawn_graph_info(g: int) -> tuple[int, int, int]:
    n, m, wt = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int()
    _check(load_library().dawn_graph_info(ctypes.c_void_p(g), ctypes.byref(n), ctypes.byref(m), ctypes.byref(wt)),
           "dawn_graph_info")
    return n.value, m.value, wt.value


def dawn_status_string(code: int) -> str:
    return status_string(code)


def dawn_destroy(g: int):
    if g:
        load_library().dawn_destroy(ctypes.c_void_p(g))


def dawn_trim_memory():
    """Return the library pools' unused device memory to the devices."""
    _check(load_library().dawn_trim_memory(), "dawn_trim_memory")


# ----------------------------------------------------------------- convenience

class Graph:
    """Owns a dawn graph handle; solves return freshly allocated tensors."""

    def __init__(self, row_ptr, col_idx, weights, device="cuda", stream=None):
        def t(x, dtype):
            return x if isinstance(x, torch.Tensor) else torch.as_tensor(x, dtype=dtype)
        row_ptr = t(row_ptr, torch.int32).contiguous()
        col_idx = t(col_idx, torch.int32).contiguous()
        weights = weights if isinstance(weights, torch.Tensor) else torch.from_numpy(weights)
        weights = weights.contiguous()
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.handle = dawn_create_graph(row_ptr, col_idx, weights, stream)
        self.n, self.m, self.wtype = dawn_graph_info(self.handle)
        self.dist_dtype = {DAWN_W_U32: torch.uint32, DAWN_W_F32: torch.float32, DAWN_W_I32: torch.int32}[self.wtype]

    def close(self):
        if getattr(self, "handle", None):
            dawn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self):
        code = dawn_status(self.handle, True)
        _check(code, "solve")

    def sssp(self, source: int, parent: bool = True, parent_edge: bool = False, check: bool = True):
        dist = torch.empty(self.n, dtype=self.dist_dtype, device=self.device)
        par = torch.empty(self.n, dtype=torch.int32, device=self.device) if parent else None
        pe = torch.empty(self.n, dtype=torch.int32, device=self.device) if parent_edge else None
        dawn_sssp(self.handle, source, dist, par, pe)
        if check:
            self.check()
        return dist, par, pe

    def msssp(self, sources, parent: bool = True, check: bool = True):
        src = torch.as_tensor(sources, dtype=torch.int32, device=self.device).contiguous()
        k = src.numel()
        dist = torch.empty((k, self.n), dtype=self.dist_dtype, device=self.device)
        par = torch.empty((k, self.n), dtype=torch.int32, device=self.device) if parent else None
        dawn_msssp(self.handle, src, dist, par)
        if check:
            self.check()
        return dist, par

    def sssp_roots(self, roots, parent: bool = True, parent_edge: bool = False, check: bool = True):
        r = torch.as_tensor(roots, dtype=torch.int32, device=self.device).contiguous()
        dist = torch.empty(self.n, dtype=self.dist_dtype, device=self.device)
        par = torch.empty(self.n, dtype=torch.int32, device=self.device) if parent else None
        pe = torch.empty(self.n, dtype=torch.int32, device=self.device) if parent_edge else None
        dawn_sssp_roots(self.handle, r, dist, par, pe)
        if check:
            self.check()
        return dist, par, pe

    def stats(self) -> dict:
        return dawn_get_stats(self.handle)

    def set_option(self, option: int, value: int):
        dawn_set_option(self.handle, option, value)

    def autotune(self, sources, mode: str = "sssp", reps: int = 3, stream=None, cache: str | None = None) -> dict:
        """Pick and keep the fastest launch configuration for `sources`
        (mode "sssp": one dawn_sssp per source; "msssp": one batched solve;
        "roots": one multi-root solve).  With `cache` (a JSON file path) a
        configuration tuned before for a graph of the same shape class on
        the same GPU model is applied without timing, and a new one is
        stored there."""
        m = {"sssp": DAWN_TUNE_SSSP, "msssp": DAWN_TUNE_MSSSP, "roots": DAWN_TUNE_ROOTS}[mode]
        k = len(sources)
        key = None
        if cache is not None:
            props = torch.cuda.get_device_properties(self.device)
            key = tune_cache_key(self.n, self.m, self.wtype, mode, k, f"{props.name}/{props.multi_processor_count}")
            hit = tune_cache_load(cache).get(key)
            if hit is not None:
                self.set_option(DAWN_OPT_CTAS_PER_SM, hit["ctas_per_sm"])
                self.set_option(DAWN_OPT_GRID_BLOCKS, hit["grid_blocks"])
                self.set_option(DAWN_OPT_BATCH, hit["batch"])
                self.set_option(DAWN_OPT_SMALL_PATH, hit.get("small_path", DAWN_SMALL_AUTO))
                self.set_option(DAWN_OPT_FRONTIER, hit.get("frontier", DAWN_FRONTIER_AUTO))
                return dict(hit, cached=True)
        with torch.cuda.device(self.device):
            res = dawn_autotune(self.handle, m, sources, reps, stream)
        if key is not None:
            tune_cache_store(cache, key, res)
        return dict(res, cached=False)


def tune_cache_key(n: int, m: int, wtype: int, mode: str, k: int, gpu: str) -> str:
    """Shape class of a tuning problem: GPU model, weight type, mode and the
    binary orders of magnitude of n, m, the average degree (half steps) and
    the source count."""
    import math
    lg = lambda x: int(round(math.log2(max(x, 1))))
    deg = round(2 * math.log2(max(m, 1) / max(n, 1))) / 2 if n > 0 and m > 0 else 0
    return f"{gpu}|w{wtype}|{mode}|n2^{lg(n)}|m2^{lg(m)}|d2^{deg}|k2^{lg(k)}"


def tune_cache_load(path: str) -> dict:
    import json
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def tune_cache_store(path: str, key: str, result: dict):
    """Adds one entry; the file is replaced atomically."""
    import json
    data = tune_cache_load(path)
    data[key] = {f: result[f] for f in ("ctas_per_sm", "grid_blocks", "batch", "small_path", "frontier", "best_ms",
                                        "default_ms") if f in result}
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class DawnSSSP(torch.autograd.Function):
    """dist = DawnSSSP.apply(weights, graph, source, check=True).

    Forward: loads `weights` (float32, one per CSR edge) into the graph and
    runs the GOVM solver, saving only the parent tree.  The weights are
    validated in stream order (the solve itself refuses invalid weights);
    with check=True the forward waits once for the solve's status and raises
    DawnError on any failure, with check=False it never synchronises and the
    caller reads the status later (Graph.check).  Backward: the library's
    kernel scatters dL/ddist along the parent tree, giving dL/dw (the sum of
    dL/ddist over the subtree below each tree edge, 0 off the tree).

    With check=False nothing in forward or backward synchronises, and after
    the handle's first forward and backward nothing allocates device memory
    outside torch's allocator, so a training step that uses it can be
    captured in a CUDA graph (torch.cuda.graph) and replayed."""

    @staticmethod
    def forward(ctx, weights: torch.Tensor, graph: Graph, source: int, check: bool = True):
        if weights.dtype != torch.float32 or graph.wtype != DAWN_W_F32:
            raise TypeError("DawnSSSP needs a float32 graph and float32 weights")
        w = weights.detach()
        if not w.is_contiguous():
            w = w.contiguous()
        stream = _stream(None)
        dawn_set_weights(graph.handle, w, stream=stream, defer_check=True)
        dist = torch.empty(graph.n, dtype=torch.float32, device=w.device)
        pe = torch.empty(graph.n, dtype=torch.int32, device=w.device)
        dawn_sssp(graph.handle, source, dist, None, pe, stream)
        if check:
            graph.check()
        ctx.graph = graph
        ctx.save_for_backward(pe)
        ctx.mark_non_differentiable(pe)
        return dist

    @staticmethod
    def backward(ctx, grad_dist):
        (pe,) = ctx.saved_tensors
        g = ctx.graph
        grad_w = torch.empty(g.m, dtype=torch.float32, device=grad_dist.device)
        gd = grad_dist if grad_dist.dtype == torch.float32 and grad_dist.is_contiguous() else \
            grad_dist.contiguous().float()
        dawn_sssp_backward(g.handle, pe, gd, grad_w)
        return grad_w, None, None, None
