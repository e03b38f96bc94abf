"""Benchmark of the GOVM shortest-path solver on one GB300 (or N replicas).

Default workload (one "step"): the 64 sources of the R-MAT scale-22 graph
(a,b,c,d = .57,.19,.19,.05, edge factor 16, duplicates removed, uint32
weights U[1,255]), each solved as its own SSSP through the C ABI
(dawn_sssp: init, every GOVM step and the dist/parent output in one
persistent launch).  GTEPS = edges of the largest WCC / solve time.

Printed (rank 0, one JSON line): device-timed GTEPS over K steps, the
roofline of the persistent kernel (algorithmic bytes from the solver's own
counters / CUDA-event launch time, against the measured HBM copy bandwidth),
the end-to-end GTEPS through the C ABI from pinned host buffers (graph copy
in, solves, dist + parent copied out), the CPU oracle on a bounded sample, and
the SM clocks sampled during the timed region.  At N = 1 the same line also
carries the rest of the metric, each leg with its own clocks, roofline, L2
rule and oracle leg: grid_2048_f32 (the high-diameter grid, 16 sources),
msssp_rmat18_1024 and roots_er64 (batched forms vs a loop of the plain
solver) and diff_rmat16_f32 (forward + backward vs the plain solver), plus
the random-gather rate of the GPU (gather_ceiling).  --no-legs skips them.

Other workloads (--workload): grid (2048^2 fp32 grid with shortcuts, 16
sources), batched (R-MAT s18 with 1024 sources in msssp launches vs a loop
of single solves; 64 uneven ER graphs in one multi-root launch vs a loop),
diff (R-MAT s16 fp32: forward, forward+backward, plain solve), tiny
(ER n=1024), apsp, mu, gsvm.

L2 rule: a workload whose graph (row_ptr and the column/weight pairs) is
larger than L2 is timed back to back; a smaller one gets L2 flushed before
every timed call, outside the call's CUDA events.

--impl reference times the CPU oracle (the literal GOVM iteration) on the
host cores instead; under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
METRIC = "GTEPS and % HBM roofline for SSSP on 1 GB300; batched/backward vs plain solver"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


KERNEL_SOURCES = ("paper_2306_07872_gb300/csrc/govm_kernel.cu", "paper_2306_07872_gb300/csrc/dawn_common.cuh",
                  "paper_2306_07872_gb300/csrc/dawn_keys.cuh")
TRAFFIC_SUMMARIES = "profiles/govm_kernel_*_traffic.md"


def kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """Per-launch DRAM bytes of govm_kernel from the committed ncu summary of
    this workload, or None when there is none or it was taken on a different
    version of the kernel sources."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, TRAFFIC_SUMMARIES))):
        try:
            with open(path) as f:
                kv = dict(l.split(":", 1) for l in f.read().splitlines() if l.startswith("- ") and ":" in l)
        except OSError:
            continue
        kv = {k[2:].strip(): v.strip().strip("`") for k, v in kv.items()}
        if kv.get("workload") != workload or kv.get("kernel_source_sha256_16") != kernel_hash():
            continue
        try:
            return float(kv["dram_bytes_per_launch"])
        except (KeyError, ValueError):
            return None
    return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks, utilisation and throttle reasons
    every 200 ms.  Entering waits (up to 2 s) for the first sample, so the
    samples cover the region that follows; the summary's sm_mhz is the median
    over samples taken under load (utilisation > 0) when there are any."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, index: int):
        self.index = index
        self.p = None
        self.lines = []

    def _read(self):
        for line in self.p.stdout:
            if line.strip():
                self.lines.append(line)
                self._first.set()

    def __enter__(self):
        import threading
        self.lines = []
        self._first = threading.Event()
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
            return self
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        self._first.wait(2.0)
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.p.wait(timeout=10)
            except subprocess.TimeoutExpired:
                self.p.kill()
            self._t.join(timeout=10)

    def summary(self):
        return clocks_summary(self.lines)


def clocks_summary(lines):
    """Median SM clock under load, the maximum clock and every throttle
    reason seen, from nvidia-smi CSV lines (fields as in Clocks.Q)."""
    sm, busy, smax, reasons = [], [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for l in lines:
        f = [x.strip() for x in l.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax = float(f[2])
        except ValueError:
            continue
        try:
            if len(f) > 9 and float(f[9]) > 0:
                busy.append(sm[-1])
        except ValueError:
            pass
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
    use = busy or sm
    return {"sm_mhz": float(np.median(use)), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm),
            "samples_under_load": len(busy)}


# ------------------------------------------------------------------ L2 rule

L2_FALLBACK = 132 * 1024 * 1024  # GB300: 129 MB (in MiB units as the device reports)


def l2_bytes(device=0) -> int:
    import torch
    try:
        return int(getattr(torch.cuda.get_device_properties(device), "L2_cache_size", 0)) or L2_FALLBACK
    except Exception:
        return L2_FALLBACK


def graph_bytes(n: int, m: int) -> int:
    """Device bytes of the arrays a solve streams: row_ptr (4 (n+1)) and the
    interleaved (column, weight) pairs (8 m)."""
    return 4 * (n + 1) + 8 * m


def l2_rule(n: int, m: int, l2: int):
    """(flush, note): flush L2 before every timed call when the graph could
    stay L2-resident between calls, and the sentence that says which."""
    gb = graph_bytes(n, m)
    if gb > l2:
        return False, (f"graph larger than L2 (row_ptr + column/weight pairs {gb / 1e6:.0f} MB > L2 "
                       f"{l2 / 1e6:.0f} MB); no flush between timed calls")
    return True, (f"graph fits in L2 (row_ptr + column/weight pairs {gb / 1e6:.1f} MB <= L2 {l2 / 1e6:.0f} MB); "
                  f"L2 flushed (a {2 * l2 / 1e6:.0f} MB write) before every timed call, outside its CUDA events")


class L2Flush:
    """Writes a buffer twice the size of L2, evicting whatever a previous
    call left there."""

    def __init__(self, device=0):
        import torch
        self.buf = torch.empty(2 * l2_bytes(device) // 4, dtype=torch.int32, device=device)
        self.k = 0

    def __call__(self):
        self.k += 1
        self.buf.fill_(self.k)


def timed_calls(fn, reps: int, flush=None, warm: int = 1):
    """CUDA-event seconds of each of `reps` calls of fn on the current
    stream, after `warm` untimed calls; with `flush`, L2 is flushed before
    every call, outside the events."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in evs:
        if flush is not None:
            flush()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in evs]) / 1e3


def reps_for(fn, seconds: float, lo: int = 3, hi: int = 4000) -> int:
    """Calls of fn that fill about `seconds` of device time (one probe)."""
    t = timed_calls(fn, 1, warm=1)[0]
    return int(max(lo, min(hi, seconds / max(t, 1e-6))))


# ------------------------------------------------------------------ workloads

def shard(sources, per_rank: int, rank: int):
    """This rank's sources: a disjoint block of `per_rank` of all ranks'
    sources (weak scaling: per-GPU work is fixed as ranks are added)."""
    return sources[rank * per_rank:(rank + 1) * per_rank]


def make_workload(name: str, rank: int = 0, world: int = 1):
    import graphgen as gg
    if name.startswith("rmat") and name[4:].isdigit():
        # rmat22 is the benchmark workload; smaller scales serve profiling
        wl = gg.rmat_u32(int(name[4:]), 16, nsrc=64 * world, seed=0)
        wl.sources = shard(wl.sources, 64, rank)
        return wl
    if name == "grid":
        wl = gg.grid_f32(2048, 0.01, nsrc=16 * world, seed=0)
        wl.sources = shard(wl.sources, 16, rank)
        return wl
    if name == "tiny":
        return gg.tiny_er()
    raise ValueError(name)


def bytes_alg(st):
    """Algorithmic bytes of one solve from its counters: 16 B per frontier
    vertex (id, row_ptr pair, own distance), 12 B per scanned edge (col,
    weight, target state filter read), 12 B per strict update (8 B atomic,
    4 B queue append)."""
    return 16 * st["frontier_sum"] + 12 * st["edges_scanned"] + 12 * st["updates"]


def roofline_entry(b_alg: float, seconds: float, kernel: str, rule: str):
    """Algorithmic bytes per call over the call's CUDA-event time, against
    the measured HBM copy bandwidth."""
    peak, kind = measured_peak()
    gbs = b_alg / seconds / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "peak_kind": f"{kind} copy bandwidth", "kernel": kernel, "b_alg_per_call": b_alg, "b_alg_rule": rule}


def host_threads(units: int) -> int:
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return max(1, min(cores, 16, units))


# --------------------------------------------------------------- our solver

def run_sssp_bench(args, wl, device, world, rank, steps=None, keep_dist=True):
    """Device-timed single-source solves: `steps` (default --steps) timed
    steps of one dawn_sssp per source, after --warmup untimed steps."""
    import torch
    import paper_2306_07872_gb300 as dawn

    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream()
    steps = args.steps if steps is None else steps
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights, device=device)
    S = len(wl.sources)
    flush_needed, l2note = l2_rule(wl.n, wl.m, l2_bytes(device))
    flush = L2Flush(device) if flush_needed else None
    tuning = None
    if not args.no_tune:  # launch shape picked by the library's autotuner (untimed setup, like the upload)
        t = time.perf_counter()
        tuning = g.autotune(wl.sources[:min(8, S)], mode="sssp", reps=2)
        tuning["tune_s"] = time.perf_counter() - t
        log(f"[bench] autotune: {tuning}")
    dist = torch.empty((S, wl.n), dtype=g.dist_dtype, device=device)
    par = torch.empty((S, wl.n), dtype=torch.int32, device=device)
    srcs = [int(s) for s in wl.sources]

    def step(evs=None):
        for i, s in enumerate(srcs):
            if evs is not None:
                evs[i][0].record(stream)
            dawn.dawn_sssp(g.handle, s, dist[i], par[i], None)
            if evs is not None:
                evs[i][1].record(stream)

    # warm-up (untimed)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g.check()
    # counters of one pass (untimed): algorithmic bytes, mu, steps
    stats = []
    for s in srcs:
        dawn.dawn_sssp(g.handle, s, dist[0], par[0], None)
        stats.append(dawn.dawn_get_stats(g.handle))
    # timed region
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in srcs]
           for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with Clocks(device) as clk:
        t0.record(stream)
        for k in range(steps):
            if flush is not None:  # between timed steps, outside their events
                flush()
            step(evs[k])
        t1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    g.check()
    dist_host = dist.cpu().numpy() if (rank == 0 and not args.no_cpu and keep_dist) else None
    if flush is None:
        elapsed = t0.elapsed_time(t1) / 1e3
    else:  # each step from its first launch's start to its last launch's end
        elapsed = sum(row[0][0].elapsed_time(row[-1][1]) for row in evs) / 1e3
    elapsed = max_over_ranks(elapsed, world)
    launch_ms = np.array([[a.elapsed_time(b) for a, b in row] for row in evs])  # [K, S]
    per_src_ms = launch_ms.mean(axis=0)
    b_alg = np.array([bytes_alg(st) for st in stats], dtype=np.float64)
    achieved_gbs = float((b_alg / (per_src_ms / 1e3)).mean() / 1e9)
    achieved_gbs_total = float(b_alg.sum() / (per_src_ms.sum() / 1e3) / 1e9)
    mu = float(np.mean([st["updates"] for st in stats]))
    # the mu = 1 floor of the algorithmic bytes, from each source's reached set
    # (read off the distances of the timed run): B_min = 28 S_reach + 12 E_reach
    inf_bits = {"u32": -1, "f32": 0x7F800000, "i32": 0x7FFFFFFF}[wl.wtype]
    deg = torch.from_numpy(np.diff(wl.row_ptr).astype(np.int64)).to(device)
    s_reach = np.zeros(S)
    e_reach = np.zeros(S)
    for i in range(S):
        reach = dist[i].view(torch.int32) != inf_bits
        s_reach[i] = float(reach.sum())
        e_reach[i] = float((deg * reach).sum())
    b_min = 28.0 * s_reach + 12.0 * e_reach
    mu_gpu = np.array([st["updates"] for st in stats], dtype=np.float64) / np.maximum(s_reach - 1, 1)
    res = {
        "dist_host": dist_host,
        "tuning": tuning,
        "elapsed": elapsed,
        "gteps": S * steps * world * wl.e_wcc / elapsed / 1e9,
        "steps": steps,
        "l2": l2note,
        "flushed": flush is not None,
        "launch_ms_mean": float(launch_ms.mean()),
        "launch_ms_median": float(np.median(launch_ms)),
        "gteps_median": float(np.median(wl.e_wcc / (per_src_ms / 1e3) / 1e9)),
        "gteps_hmean": float(S / np.sum(1.0 / (wl.e_wcc / (per_src_ms / 1e3) / 1e9))),
        "achieved_gbs": achieved_gbs_total,
        "achieved_gbs_mean_of_launches": achieved_gbs,
        "b_alg_mean": float(b_alg.mean()),
        "b_min_mean": float(b_min.mean()),
        "achieved_gbs_b_min": float(b_min.sum() / (per_src_ms.sum() / 1e3) / 1e9),
        "mu_gpu": float(mu_gpu.mean()),
        "updates_mean": mu,
        "edges_scanned_mean": float(np.mean([st["edges_scanned"] for st in stats])),
        "steps_mean": float(np.mean([st["steps"] for st in stats])),
        "clocks": clk.summary(),
        "launches": S * steps,
        "frontier_sum_mean": float(np.mean([st["frontier_sum"] for st in stats])),
        "stats0": stats[0],
    }
    g.close()
    del dist, par
    torch.cuda.empty_cache()
    return res


def run_e2e(args, wl, device, world, tuning=None):
    """Same metric through the C ABI from pinned host buffers.  Every step
    copies the graph in and validates it (dawn_create_graph with host
    inputs), sets the tuned launch options, solves every source and copies
    each source's dist + parent rows back to pinned host memory.  The steps
    are pipelined the way a serving loop would run them: result copies go
    back on a second stream while the next solves run, and the next step's
    graph is uploaded on a third stream while this step's solves run."""
    import torch
    import paper_2306_07872_gb300 as dawn

    torch.cuda.set_device(device)
    rp = torch.from_numpy(wl.row_ptr).pin_memory()
    cl = torch.from_numpy(wl.col).pin_memory()
    w = torch.from_numpy(wl.weights).pin_memory()
    S = len(wl.sources)
    dist_dtype = torch.uint32 if wl.weights.dtype == np.uint32 else torch.float32
    h_dist = torch.empty((S, wl.n), dtype=dist_dtype).pin_memory()
    h_par = torch.empty((S, wl.n), dtype=torch.int32).pin_memory()
    dist = torch.empty((S, wl.n), dtype=dist_dtype, device=device)
    par = torch.empty((S, wl.n), dtype=torch.int32, device=device)
    stream = torch.cuda.current_stream()
    copy_stream = torch.cuda.Stream(device=device)
    ingest_stream = torch.cuda.Stream(device=device)
    done = [torch.cuda.Event() for _ in wl.sources]
    srcs = [int(s) for s in wl.sources]

    def ingest():
        h = dawn.dawn_create_graph(rp, cl, w, ingest_stream)  # returns once the graph is validated
        if tuning:
            dawn.dawn_set_option(h, dawn.DAWN_OPT_CTAS_PER_SM, tuning["ctas_per_sm"])
            dawn.dawn_set_option(h, dawn.DAWN_OPT_GRID_BLOCKS, tuning["grid_blocks"])
            dawn.dawn_set_option(h, dawn.DAWN_OPT_FRONTIER, tuning["frontier"])
        return h

    def solve(h):
        stream.wait_stream(ingest_stream)  # the graph's device copy is complete
        for i, s in enumerate(srcs):
            dawn.dawn_sssp(h, s, dist[i], par[i], None, stream)
            done[i].record(stream)
            copy_stream.wait_event(done[i])
            with torch.cuda.stream(copy_stream):
                h_dist[i].copy_(dist[i], non_blocking=True)
                h_par[i].copy_(par[i], non_blocking=True)
        stream.wait_stream(copy_stream)

    def finish(h):
        code = dawn.dawn_status(h, True)  # waits for the solves and the copies back
        dawn.dawn_destroy(h)
        if code:
            raise dawn.DawnError(code, "e2e solve")

    def run(steps, phases=None):
        # phases: host milliseconds of each part of a step, and device
        # milliseconds of its solves (events on the solve stream; they add
        # nothing to the stream's work)
        clock = lambda: time.perf_counter() * 1e3
        t0 = clock()
        h = ingest()
        first = clock() - t0
        rows = []
        for k in range(steps):
            t0 = clock()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            solve(h)
            ev[1].record(stream)
            t1 = clock()
            h_next = ingest() if k + 1 < steps else None  # overlaps this step's solves
            t2 = clock()
            finish(h)
            t3 = clock()
            h = h_next
            rows.append((t1 - t0, t2 - t1, t3 - t2, ev))
        if phases is not None:
            torch.cuda.synchronize()
            phases["first_ingest_ms"] = first
            phases["steps"] = [{"enqueue_ms": a, "ingest_next_ms": b, "status_and_destroy_ms": c,
                                "device_ms": ev[0].elapsed_time(ev[1]),
                                "device_gap_before_ms": rows[i - 1][3][1].elapsed_time(ev[0]) if i else None}
                               for i, (a, b, c, ev) in enumerate(rows)]

    # warm-up: the line's W steps (at least two, so that two graphs have been
    # alive at once and the library's memory pool holds what the loop needs: a
    # pool that grows maps new memory while solves run, which can stall them)
    run(max(2, args.warmup))
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 10))  # the line's K steps, at most 10
    barrier(world)
    torch.cuda.synchronize()
    phases = {}
    t = time.perf_counter()
    run(steps, phases)
    torch.cuda.synchronize()
    el = time.perf_counter() - t
    barrier(world)
    el = max_over_ranks(el, world)
    h2d = wl.row_ptr.nbytes + wl.col.nbytes + wl.weights.nbytes
    d2h = h_dist.numel() * 4 + h_par.numel() * 4
    # after the timed region: each direction's copies alone, on an idle GPU,
    # to show how much of a step the host link needs
    a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a_ev.record(stream)
    h_dist.copy_(dist, non_blocking=True)
    h_par.copy_(par, non_blocking=True)
    b_ev.record(stream)
    torch.cuda.synchronize()
    d2h_ms = a_ev.elapsed_time(b_ev)
    g_dev = [torch.empty(x.numel(), dtype=x.dtype, device=device) for x in (rp, cl, w)]
    a_ev.record(stream)
    for dst, src in zip(g_dev, (rp, cl, w)):
        dst.copy_(src, non_blocking=True)
    b_ev.record(stream)
    torch.cuda.synchronize()
    h2d_ms = a_ev.elapsed_time(b_ev)
    del g_dev
    return {"value": S * world * wl.e_wcc / (el / steps) / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps, "ms_per_step": el / steps * 1e3,
            "copies_alone_ms": {"d2h": d2h_ms, "h2d": h2d_ms, "d2h_gbs": d2h / d2h_ms / 1e6,
                                "h2d_gbs": h2d / h2d_ms / 1e6},
            # the same metric from the median step's host wall time (the first
            # step's graph upload excluded): a step that met a slow host link
            # moves the mean, not this
            "median_step_value": S * world * wl.e_wcc / (float(np.median(
                [st["enqueue_ms"] + st["ingest_next_ms"] + st["status_and_destroy_ms"] for st in phases["steps"]]))
                / 1e3) / 1e9,
            "phases": phases}


def cpu_baseline(wl, budget_s: float = 20.0, gpu_dist=None, single_core: bool = True):
    """The oracle's literal GOVM iteration (Algorithm 2) on the host cores,
    one source per thread, on a bounded sample of the sources; plus the
    single-core time of one source by Algorithm 2 and by Dijkstra.  With
    `gpu_dist` (row i = the GPU's distances from source i) every sampled
    source is also compared bit for bit with the GPU.  single_core=False
    (workloads whose one-source solve takes many seconds) skips the
    single-core probes and runs one round of one source per thread."""
    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    threads = max(1, min(cores, 16, len(wl.sources)))
    if single_core:
        # one probe solve sizes the sample to the time budget
        t, _ = oracle.timed_govm(wl.row_ptr, wl.col, wl.weights, [int(wl.sources[0])], threads=1)
        t0 = time.perf_counter()
        oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, int(wl.sources[0]))
        t_dij = time.perf_counter() - t0
        rounds = max(1, int(budget_s / max(t, 1e-3) / 2))
    else:
        rounds = 1
    nsrc = min(len(wl.sources), threads * rounds)
    sample = [int(s) for s in wl.sources[:nsrc]]
    el, res = oracle.timed_govm(wl.row_ptr, wl.col, wl.weights, sample, threads=threads)
    out = {"value": len(sample) * wl.e_wcc / el / 1e9, "unit": "GTEPS", "cores": threads, "kind": "oracle",
           "sample": f"{len(sample)} of the {len(wl.sources)} sources, literal GOVM (Algorithm 2), "
                     f"one source per thread, {threads} threads, {el:.1f} s",
           "mu_oracle": float(np.mean([r[1]["mu"] for r in res]))}
    if single_core:
        out["single_core_ms_per_source"] = {"govm_alg2": t * 1e3, "dijkstra": t_dij * 1e3}
    if gpu_dist is not None:
        same = [np.array_equal(np.asarray(r[0]).view(np.uint32), gpu_dist[i].view(np.uint32))
                for i, r in enumerate(res)]
        out["bit_exact_vs_gpu"] = {"sources_compared": len(same), "all_equal": bool(all(same))}
    if wl.n <= 2048:  # small graphs: Floyd-Warshall too (Section 3.1's all-pairs form)
        t0 = time.perf_counter()
        D = oracle.floyd_warshall(wl.row_ptr, wl.col, wl.weights)
        out["single_core_ms_floyd_warshall_all_pairs"] = (time.perf_counter() - t0) * 1e3
        if gpu_dist is not None:
            out["floyd_warshall_equal_to_gpu"] = bool(all(
                np.array_equal(np.asarray(D[int(s)]).view(np.uint32), gpu_dist[i].view(np.uint32))
                for i, s in enumerate(wl.sources)))
    return out


# ------------------------------------------------- batched and differentiable

def _time(fn, reps=3, warm=1, flush=None):
    """Mean CUDA-event seconds per call (see timed_calls)."""
    return float(timed_calls(fn, reps, flush=flush, warm=warm).mean())


ALG_RULE = "16 B per frontier vertex + 12 B per scanned edge + 12 B per update"


def leg_msssp(args, device=0):
    """Pattern 2a: the 1024 sources of an R-MAT s18 graph in batched
    launches (dawn_msssp) vs a loop of single-source solves, each arm in the
    launch shape the autotuner picks for it."""
    import torch
    import graphgen as gg
    import paper_2306_07872_gb300 as dawn
    wl = gg.rmat_u32(18, 16, nsrc=1024, seed=0)
    if args.sources:  # a smaller batch (profiling runs)
        wl.sources = wl.sources[:args.sources]
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    src = torch.from_numpy(wl.sources).cuda()
    k = len(wl.sources)
    dist = torch.empty((k, wl.n), dtype=torch.uint32, device="cuda")
    par = torch.empty((k, wl.n), dtype=torch.int32, device="cuda")
    dawn.dawn_reserve(g.handle, k)
    flush_needed, l2note = l2_rule(wl.n, wl.m, l2_bytes(device))
    flush = L2Flush(device) if flush_needed else None
    tune_batch = None if args.no_tune else g.autotune(wl.sources, mode="msssp", reps=2)
    srcs = [int(x) for x in wl.sources]

    def loop():
        for i, s_ in enumerate(srcs):
            dawn.dawn_sssp(g.handle, s_, dist[i], par[i], None)
    # the loop arm gets its own tuned launch shape; both shapes are applied
    # in turn inside the one clocked region
    tune_loop = None if args.no_tune else g.autotune(wl.sources[:8], mode="sssp", reps=2)
    def use(t):
        if t:
            dawn.dawn_set_option(g.handle, dawn.DAWN_OPT_CTAS_PER_SM, t["ctas_per_sm"])
            dawn.dawn_set_option(g.handle, dawn.DAWN_OPT_GRID_BLOCKS, t["grid_blocks"])
            dawn.dawn_set_option(g.handle, dawn.DAWN_OPT_BATCH, t["batch"])
            dawn.dawn_set_option(g.handle, dawn.DAWN_OPT_SMALL_PATH, t["small_path"])
            dawn.dawn_set_option(g.handle, dawn.DAWN_OPT_FRONTIER, t["frontier"])
    with Clocks(device) as clk:
        use(tune_batch)
        tb = timed_calls(lambda: dawn.dawn_msssp(g.handle, src, dist, par), 5, flush=flush)
        g.check()
        st = g.stats()  # summed over the launches of the last call
        rows_host = dist[:64].cpu().numpy()
        use(tune_loop)
        tl = timed_calls(loop, 3, flush=flush)
        g.check()
    t_batch, t_loop = float(tb.mean()), float(tl.mean())
    out = {"batched_s": t_batch, "loop_s": t_loop, "speedup": t_loop / t_batch,
           "gteps_batched": k * wl.e_wcc / t_batch / 1e9, "gteps_loop": k * wl.e_wcc / t_loop / 1e9,
           "edges_scanned_per_instance": st["edges_scanned"] / k, "updates_per_instance": st["updates"] / k,
           "tuning_batched": tune_batch, "tuning_loop": tune_loop, "clocks": clk.summary(), "l2": l2note,
           "config": {"workload": wl.name, "n": wl.n, "m": wl.m, "e_wcc": wl.e_wcc, "sources": k,
                      "timed_calls": {"batched": len(tb), "loop": len(tl)}},
           "roofline": roofline_entry(bytes_alg(st), t_batch, "govm_kernel (1024 instances)",
                                      ALG_RULE + ", summed over the instances")}
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_leg_sources(wl, rows_host, args.cpu_budget)
    del dist, par
    g.close()
    torch.cuda.empty_cache()
    return out


def leg_roots(args, device=0):
    """Pattern 2b: 64 uneven ER graphs solved as one multi-root forest on
    their disjoint union (dawn_sssp_roots) vs a loop of per-graph solves."""
    import torch
    import graphgen as gg
    import paper_2306_07872_gb300 as dawn
    wb = gg.er_batch(count=64, seed=0)
    gu = dawn.Graph(wb.row_ptr, wb.col, wb.weights)
    roots = torch.from_numpy(wb.sources).cuda()
    du = torch.empty(wb.n, dtype=torch.uint32, device="cuda")
    pu = torch.empty(wb.n, dtype=torch.int32, device="cuda")
    flush_needed, l2note = l2_rule(wb.n, wb.m, l2_bytes(device))
    flush = L2Flush(device) if flush_needed else None
    tune_roots = None if args.no_tune else gu.autotune(wb.sources, mode="roots", reps=2)
    offs = wb.extra["offsets"]
    parts = []
    for i in range(64):
        a, b = int(offs[i]), int(offs[i + 1])
        e0, e1 = int(wb.row_ptr[a]), int(wb.row_ptr[b])
        rp = (wb.row_ptr[a:b + 1] - e0).astype(np.int32)
        parts.append(dawn.Graph(rp, (wb.col[e0:e1] - a).astype(np.int32), wb.weights[e0:e1]))
        if not args.no_tune:
            parts[-1].autotune([0], mode="sssp", reps=1)
    outs = [(torch.empty(p_.n, dtype=torch.uint32, device="cuda"), torch.empty(p_.n, dtype=torch.int32, device="cuda"))
            for p_ in parts]

    def loop2():
        for p_, (d_, pp_) in zip(parts, outs):
            dawn.dawn_sssp(p_.handle, 0, d_, pp_, None)
    one = lambda: dawn.dawn_sssp_roots(gu.handle, roots, du, pu)
    with Clocks(device) as clk:
        tr = timed_calls(one, reps_for(one, 1.0, lo=5, hi=200), flush=flush)
        gu.check()
        st_roots = gu.stats()
        tl = timed_calls(loop2, reps_for(loop2, 1.0, lo=3, hi=100), flush=flush)
        for p_ in parts:
            p_.check()
    t_roots, t_loop2 = float(tr.mean()), float(tl.mean())
    out = {"one_launch_s": t_roots, "loop_s": t_loop2, "speedup": t_loop2 / t_roots,
           "gteps_one_launch": wb.m / t_roots / 1e9, "gteps_loop": wb.m / t_loop2 / 1e9,
           "tuning_one_launch": tune_roots, "clocks": clk.summary(), "l2": l2note,
           "config": {"workload": wb.name, "n": wb.n, "m": wb.m, "graphs": 64,
                      "gteps_edges": "all m edges of the union (every graph is solved from its root)",
                      "timed_calls": {"one_launch": len(tr), "loop": len(tl)}},
           "roofline": roofline_entry(bytes_alg(st_roots), t_roots, "govm_kernel (multi-root forest)", ALG_RULE)}
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_leg_roots(wb, du.cpu().numpy())
    for p_ in parts:
        p_.close()
    gu.close()
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    return {"msssp_rmat18_1024": leg_msssp(args), "roots_er64": leg_roots(args)}


def run_batched22(args):
    """The headline graph's sources (the first --sources of them) in batched
    dawn_msssp launches alone, without the single-solve line (profiling runs)."""
    wl = make_workload("rmat22")
    if args.sources:
        wl.sources = wl.sources[:args.sources]
    return {"msssp_rmat22": leg_c2_batched(args, wl, None)}


def leg_diff(args, device=0):
    """Pattern 3 on R-MAT s16 fp32: plain solve, forward + backward through
    the C ABI, and forward (weights loaded + solve saving the parent tree)
    and forward + backward through torch.autograd."""
    import torch
    import graphgen as gg
    import paper_2306_07872_gb300 as dawn
    wl = gg.rmat_f32_diff(scale=16, edge_factor=16, ntargets=256, seed=0)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    w = torch.from_numpy(wl.weights).cuda()
    tg = torch.from_numpy(wl.extra["targets"]).long().cuda()
    cf = torch.from_numpy(wl.extra["coef"]).float().cuda()
    dist = torch.empty(wl.n, dtype=torch.float32, device="cuda")
    pe = torch.empty(wl.n, dtype=torch.int32, device="cuda")
    grad_dist = torch.zeros(wl.n, dtype=torch.float32, device="cuda")
    grad_dist[tg] = cf
    grad_w = torch.empty(wl.m, dtype=torch.float32, device="cuda")
    flush_needed, l2note = l2_rule(wl.n, wl.m, l2_bytes(device))
    flush = L2Flush(device) if flush_needed else None
    ww = w.clone().requires_grad_(True)

    def plain():
        dawn.dawn_sssp(g.handle, 0, dist, None, pe)

    def fwd():
        return dawn.DawnSSSP.apply(w, g, 0)

    def fwd_bwd():
        ww.grad = None
        d = dawn.DawnSSSP.apply(ww, g, 0)
        (d[tg] * cf).sum().backward()

    def fwd_bwd_nosync():  # status read after the loop, not per forward
        ww.grad = None
        d = dawn.DawnSSSP.apply(ww, g, 0, False)
        (d[tg] * cf).sum().backward()

    def bwd():
        dawn.dawn_sssp_backward(g.handle, pe, grad_dist, grad_w)

    leaf = torch.zeros(wl.n, dtype=torch.float32, device="cuda", requires_grad=True)

    def loss_only():  # the same loss and its backward on a leaf tensor: PyTorch's share of an autograd step
        leaf.grad = None
        (leaf[tg] * cf).sum().backward()

    def c_abi_fwd_bwd():
        dawn.dawn_sssp(g.handle, 0, dist, None, pe)
        dawn.dawn_sssp_backward(g.handle, pe, grad_dist, grad_w)
    times = {}
    with Clocks(device) as clk:
        for name, fn in (("plain_sssp_s", plain), ("backward_kernel_s", bwd), ("c_abi_forward_backward_s", c_abi_fwd_bwd),
                         ("autograd_forward_s", fwd), ("autograd_forward_backward_s", fwd_bwd),
                         ("autograd_forward_backward_nosync_s", fwd_bwd_nosync), ("autograd_loss_only_s", loss_only)):
            times[name] = float(np.median(timed_calls(fn, reps_for(fn, 0.4, lo=20, hi=2000), flush=flush, warm=3)))
        g.check()
        # the same autograd step (no status read) captured once in a CUDA
        # graph and replayed: what a training loop that captures its step runs
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(2):
                fwd_bwd_nosync()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        ww.grad = None
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg):
            d_cap = dawn.DawnSSSP.apply(ww, g, 0, False)
            (d_cap[tg] * cf).sum().backward()
        times["autograd_forward_backward_graph_s"] = float(np.median(
            timed_calls(cg.replay, reps_for(cg.replay, 0.4, lo=20, hi=2000), flush=flush, warm=3)))
        g.check()
        grad_graph = ww.grad.detach().clone()
    dawn.dawn_sssp(g.handle, 0, dist, None, pe)
    bwd()
    g.check()
    # the replayed graph's gradient against the C ABI's (float32 sums in a
    # varying order: compared relative to the largest value)
    graph_grad_diff = float((grad_graph - grad_w).abs().max().item() / max(grad_w.abs().max().item(), 1e-30))
    tree = int((pe >= 0).sum().item())
    b_bw = 8 * wl.n + 4 * wl.m + 12 * tree
    res = dict(times)
    res.update({"c_abi_fb_over_plain": times["c_abi_forward_backward_s"] / times["plain_sssp_s"],
                "autograd_fb_over_plain": times["autograd_forward_backward_s"] / times["plain_sssp_s"],
                "autograd_fb_nosync_over_plain": times["autograd_forward_backward_nosync_s"] / times["plain_sssp_s"],
                "autograd_fb_graph_over_plain": times["autograd_forward_backward_graph_s"] / times["plain_sssp_s"],
                # the eager step less the loss's own autograd cost (a leaf tensor in place of the solver)
                "autograd_fb_nosync_less_loss_over_plain":
                    (times["autograd_forward_backward_nosync_s"] - times["autograd_loss_only_s"]) / times["plain_sssp_s"],
                "graph_grad_max_diff_over_max": graph_grad_diff,
                "timing": "median of per-call CUDA events", "clocks": clk.summary(), "l2": l2note,
                "config": {"workload": wl.name, "n": wl.n, "m": wl.m, "source": 0, "targets": len(wl.extra["targets"]),
                           "tree_edges": tree},
                "roofline": roofline_entry(
                    b_bw, times["backward_kernel_s"], "bw_count_kernel + bw_walk_kernel",
                    "8 B per vertex (dL/d dist, parent edge) + 4 B per edge (dL/dw written, zeros included) + "
                    "12 B per tree edge (tail lookup, accumulator read-modify-write)")})
    if not args.no_cpu:
        res["cpu_baseline"] = cpu_leg_diff(wl, grad_dist.cpu().numpy(), grad_w.cpu().numpy())
    g.close()
    torch.cuda.empty_cache()
    return res


def run_diff(args):
    return {"diff_rmat16_f32": leg_diff(args)}


def leg_c2_batched(args, wl, res, device=0):
    """The headline workload's sources solved in batched dawn_msssp launches,
    in the batch size the autotuner picks, against the line's own single
    solves (`res`): the metric's batched-vs-plain comparison on the C2 graph.
    Distances are compared bit for bit with the line's single solves, which
    the line's cpu_baseline compares with the oracle."""
    import torch
    import paper_2306_07872_gb300 as dawn
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights, device=device)
    k = len(wl.sources)
    src = torch.from_numpy(wl.sources).to(device)
    dist = torch.empty((k, wl.n), dtype=torch.uint32, device=device)
    par = torch.empty((k, wl.n), dtype=torch.int32, device=device)
    tune = None if args.no_tune else g.autotune(wl.sources, mode="msssp", reps=2)
    flush_needed, l2note = l2_rule(wl.n, wl.m, l2_bytes(device))
    flush = L2Flush(device) if flush_needed else None
    with Clocks(device) as clk:
        tb = timed_calls(lambda: dawn.dawn_msssp(g.handle, src, dist, par), max(1, min(args.steps, 5)), flush=flush)
        g.check()
    st = g.stats()
    t_batch = float(tb.mean())
    t_single = res["launch_ms_mean"] / 1e3 * k if res else float("nan")  # the line's single solves
    out = {"batched_s": t_batch, "single_solves_s": t_single, "speedup": t_single / t_batch,
           "gteps_batched": k * wl.e_wcc / t_batch / 1e9, "tuning": tune, "clocks": clk.summary(), "l2": l2note,
           "config": {"workload": wl.name, "n": wl.n, "m": wl.m, "e_wcc": wl.e_wcc, "sources": k,
                      "timed_calls": len(tb)},
           "roofline": roofline_entry(bytes_alg(st), t_batch, f"govm_kernel ({k} instances)",
                                      ALG_RULE + ", summed over the instances")}
    if res and res.get("dist_host") is not None:
        out["bit_exact_vs_single_solves"] = bool(np.array_equal(dist.cpu().numpy(), res["dist_host"]))
    del dist, par
    g.close()
    torch.cuda.empty_cache()
    return out


def leg_grid(args, device=0):
    """C3: the 2048^2 fp32 grid with 1 % shortcuts, 16 sources each solved as
    its own SSSP (many GOVM steps with small frontiers)."""
    wl = make_workload("grid")
    res = run_sssp_bench(args, wl, device, 1, 0, steps=min(args.steps, 5))
    out = {"gteps": res["gteps"], "gteps_median": res["gteps_median"], "launch_ms_mean": res["launch_ms_mean"],
           "steps_timed": res["steps"], "govm_steps_mean": res["steps_mean"], "mu_gpu": res["mu_gpu"],
           "edges_scanned_over_e_wcc": res["edges_scanned_mean"] / wl.e_wcc,
           "us_per_govm_step": res["launch_ms_mean"] * 1e3 / max(res["steps_mean"], 1.0),
           "clocks": res["clocks"], "l2": res["l2"], "tuning": res["tuning"],
           "config": {"workload": wl.name, "n": wl.n, "m": wl.m, "e_wcc": wl.e_wcc, "sources_per_step": len(wl.sources),
                      "timed_steps": res["steps"]},
           "roofline": {**roofline_entry(res["b_alg_mean"], res["launch_ms_mean"] / 1e3, "govm_kernel", ALG_RULE),
                        "traffic": recorded_traffic(wl.name), "frac_b_min": res["achieved_gbs_b_min"] / measured_peak()[0]}}
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(wl, args.cpu_budget, res["dist_host"], single_core=False)
    return out


def gather_ceiling(device, n_rows: int, count: int = 1 << 26):
    """Random 8-byte gathers per second by a stock torch kernel
    (index_select of int64 rows at random int32 indices) from an array of
    n_rows rows, the size of the solver's packed state: the rate of the
    random L2 requests that every scanned edge makes."""
    import torch
    x = torch.arange(n_rows, dtype=torch.int64, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(7)
    idx = torch.randint(0, n_rows, (count,), dtype=torch.int32, device=device, generator=gen)
    out = torch.empty(count, dtype=torch.int64, device=device)
    t = timed_calls(lambda: torch.index_select(x, 0, idx, out=out), 5, warm=2)
    best = float(t.min())
    return {"gathers_per_s": count / best, "array_mb": 8 * n_rows / 1e6, "count": count,
            "kernel": "torch.index_select (int64 rows, int32 indices)", "best_of": len(t),
            "note": "each gather also streams a 4 B index in and an 8 B result out"}


def cpu_leg_sources(wl, gpu_rows, budget_s: float):
    """Oracle beside the batched solve: literal Algorithm 2, one source per
    host thread, on a bounded prefix of the sources; the first rows are
    compared bit for bit with the GPU's."""
    import oracle
    threads = host_threads(len(wl.sources))
    t1, _ = oracle.timed_govm(wl.row_ptr, wl.col, wl.weights, [int(wl.sources[0])], threads=1)
    nsrc = min(len(wl.sources), threads * max(1, int(budget_s / max(t1, 1e-3) / 2)))
    sample = [int(x) for x in wl.sources[:nsrc]]
    el, res = oracle.timed_govm(wl.row_ptr, wl.col, wl.weights, sample, threads=threads)
    same = [np.array_equal(np.asarray(r[0]).view(np.uint32), gpu_rows[i].view(np.uint32))
            for i, r in enumerate(res[:len(gpu_rows)])]
    return {"value": len(sample) * wl.e_wcc / el / 1e9, "unit": "GTEPS", "cores": threads, "kind": "oracle",
            "sample": f"{len(sample)} of the {len(wl.sources)} sources, literal GOVM (Algorithm 2), one source per "
                      f"thread, {el:.1f} s",
            "bit_exact_vs_gpu": {"rows_compared": len(same), "all_equal": bool(all(same))}}


def cpu_leg_roots(wb, gpu_dist):
    """Oracle beside the multi-root solve: literal Algorithm 2 with all roots
    at once (one thread), compared bit for bit with the GPU."""
    import oracle
    t0 = time.perf_counter()
    d, _ = oracle.govm(wb.row_ptr, wb.col, wb.weights, wb.sources)
    el = time.perf_counter() - t0
    return {"value": wb.m / el / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"the whole forest ({len(wb.sources)} roots), literal GOVM (Algorithm 2), one thread, "
                      f"{el:.2f} s",
            "bit_exact_vs_gpu": bool(np.array_equal(np.asarray(d).view(np.uint32), gpu_dist.view(np.uint32)))}


def cpu_leg_diff(wl, c, gpu_grad):
    """Oracle beside forward + backward: fp32 Dijkstra, the parent rule and
    the float64 subtree gradient (one thread); the GPU gradient's largest
    error relative to the largest reference value is reported."""
    import oracle
    t0 = time.perf_counter()
    g_ref = oracle.subtree_grad(wl.row_ptr, wl.col, wl.weights, 0, c)
    el = time.perf_counter() - t0
    scale = float(np.max(np.abs(g_ref))) or 1.0
    return {"seconds": el, "cores": 1, "kind": "oracle",
            "sample": "the whole graph: fp32 Dijkstra, lowest-index parents, float64 Dijkstra and subtree sums",
            "max_abs_err_over_max_ref": float(np.max(np.abs(gpu_grad.astype(np.float64) - g_ref))) / scale}


def run_mu(args):
    """The paper's validation experiment (Section 4.2) on synthetic graphs:
    every graph is solved with all weights 1.0f and with fp32 weights
    uniform in [0, 2]; mu = path updates / (reached vertices - 1) on the GPU
    (vertices entering beta per step).  With unit weights mu is exactly 1;
    the difference is the share of paths that GOVM had to update.  Unless
    --no-cpu is given, the line's cpu_baseline holds mu of the literal
    Algorithm 2 (the oracle) for the first source of each graph."""
    import torch
    import graphgen as gg
    import paper_2306_07872_gb300 as dawn
    graphs = {
        "rmat_s18": lambda: gg.rmat(18, 16, seed=0, relabel=True),
        "er_n262144_d16": lambda: gg.erdos_renyi(1 << 18, 16 << 18, seed=3),
        "grid_512": lambda: gg.grid(512, 0.01, seed=1)[:2],
    }
    out, cases = {}, []
    for name, make in graphs.items():
        rp, cl = make()
        src, _, e_wcc = gg.wcc_sources(rp, cl, 4, seed=5)
        res = {}
        for wname, w in (("unit", np.ones(len(cl), np.float32)),
                         ("u02", gg.weights_f32_uniform(len(cl), 0.0, 2.0, seed=9))):
            g = dawn.Graph(rp, cl, w)
            mus, times = [], []
            for s_ in src:
                dist, _, _ = g.sssp(int(s_), parent=False)
                t = _time(lambda: g.sssp(int(s_), parent=False, check=False), reps=3, warm=1)
                st = g.stats()
                reached = int(torch.isfinite(dist).sum().item())
                mus.append(st["updates"] / max(reached - 1, 1))
                times.append(t)
            res[wname] = {"mu_gpu": float(np.mean(mus)), "solve_ms": 1e3 * float(np.mean(times))}
            cases.append((name, wname, rp, cl, w, int(src[0])))
            g.close()
        res["updated_path_ratio_gpu"] = res["u02"]["mu_gpu"] - 1.0
        res["time_ratio_u02_over_unit"] = res["u02"]["solve_ms"] / res["unit"]["solve_ms"]
        out[name] = res
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline_mu(cases)
    return out


def cpu_baseline_mu(cases):
    """CPU leg of the mu experiment: the oracle's literal Algorithm 2 (one
    thread, in-place alpha) on each (graph, weights, source) case, giving its
    own mu and time.  Algorithm 2 updates alpha in place and the GPU reads it
    in place across concurrent tiles, so the two mu values differ; only the
    fixpoint is shared."""
    import oracle
    out = {"kind": "oracle", "cores": 1, "sample": "first WCC source of each graph and weight set, literal "
           "GOVM (Algorithm 2), one thread"}
    for name, wname, rp, cl, w, s in cases:
        t0 = time.perf_counter()
        _, ost = oracle.govm(rp, cl, w, s)
        out.setdefault(name, {})[wname] = {"mu_oracle_alg2": ost["mu"],
                                           "solve_ms": (time.perf_counter() - t0) * 1e3}
    for name in {c[0] for c in cases}:
        out[name]["updated_path_ratio_oracle"] = out[name]["u02"]["mu_oracle_alg2"] - 1.0
    return out


def run_apsp(args):
    """APSP as repeated SSSP (Section 3.4): every vertex of an R-MAT scale-14
    graph is a source, solved by one dawn_msssp call in the launch shape the
    autotuner picks; the paper's work bound is mu * S_wcc * E_wcc edge
    relaxations."""
    import torch
    import graphgen as gg
    import paper_2306_07872_gb300 as dawn
    scale = 14
    rp, cl = gg.rmat(scale, 16, seed=0, relabel=True)
    w = gg.weights_u32(len(cl), 1, 255, seed=1)
    _, s_wcc, e_wcc = gg.largest_wcc(rp, cl)
    n = len(rp) - 1
    g = dawn.Graph(rp, cl, w)
    src = torch.arange(n, dtype=torch.int32, device="cuda")
    dist = torch.empty((n, n), dtype=torch.uint32, device="cuda")
    tuning = None if args.no_tune else g.autotune(np.arange(n, dtype=np.int32), mode="msssp", reps=1)
    flush_needed, l2note = l2_rule(n, len(cl), l2_bytes(0))
    with Clocks(0) as clk:
        t = _time(lambda: dawn.dawn_msssp(g.handle, src, dist, None), reps=3, warm=1,
                  flush=L2Flush(0) if flush_needed else None)
    g.check()
    st = g.stats()  # summed over all launches of the call
    scanned = st["edges_scanned"]
    g.close()
    small = bool(tuning) and tuning.get("small_path") == dawn.DAWN_SMALL_WHEN_STATE_FITS
    if small:  # state, bitmap and frontier live in shared memory: only the CSR and the output cross the SM
        b_dev = 8 * st["frontier_sum"] + 8 * scanned + 4 * n * n
        rule = ("small-graph kernel: 8 B per frontier vertex (row_ptr pair) + 8 B per scanned edge (column and "
                "weight) + 4 B of dist per vertex and source; the solver state stays in shared memory and the "
                "2.2 MB CSR in L2, so HBM is not the bound")
    else:
        b_dev = bytes_alg(st)
        rule = "16 B per frontier vertex + 12 B per scanned edge + 12 B per update, summed over the sources"
    return {"apsp_rmat14": {"n": n, "m": len(cl), "s_wcc": s_wcc, "e_wcc": e_wcc, "seconds": t,
                            "gteps": n * e_wcc / t / 1e9, "edges_scanned": scanned,
                            "mu_work": scanned / (s_wcc * e_wcc), "tuning": tuning, "clocks": clk.summary(),
                            "l2": l2note,
                            "roofline": roofline_entry(b_dev, t, "govm_small_kernel" if small else "govm_kernel",
                                                       rule)}}


def run_gsvm(args):
    """Ablation of GOVM's frontier (Section 3.4) against GSVM (Algorithm 1,
    Section 3.2), both on the GPU: time, steps and edges relaxed per solve."""
    import graphgen as gg
    import paper_2306_07872_gb300 as dawn
    out = {}
    for name, wl in (("rmat_s20", gg.rmat_u32(20, 16, nsrc=4, seed=0)), ("grid_512", gg.grid_f32(512, 0.01, nsrc=4, seed=0))):
        g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
        res = {}
        for alg, flag in (("govm", 0), ("gsvm", 1)):
            g.set_option(dawn.DAWN_OPT_GSVM, flag)
            ts, st = [], []
            for s_ in wl.sources:
                ts.append(_time(lambda: g.sssp(int(s_), parent=False, check=False), reps=3, warm=1))
                g.check()
                st.append(g.stats())
            res[alg] = {"solve_ms": 1e3 * float(np.mean(ts)), "steps": float(np.mean([x["steps"] for x in st])),
                        "edges_scanned": float(np.mean([x["edges_scanned"] for x in st]))}
        res["work_ratio_gsvm_over_govm"] = res["gsvm"]["edges_scanned"] / res["govm"]["edges_scanned"]
        res["time_ratio_gsvm_over_govm"] = res["gsvm"]["solve_ms"] / res["govm"]["solve_ms"]
        out[name] = res
        g.close()
    return out


# ----------------------------------------------------------------- plumbing

def barrier(world):
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as tdist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if tdist.get_backend() == "nccl" else "cpu")
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def init_dist(world, local):
    if world > 1:
        import torch
        import torch.distributed as tdist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        tdist.init_process_group(backend)


def main_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    wl = make_workload(args.workload if (args.workload.startswith("rmat") or args.workload in ("grid", "tiny"))
                       else "rmat22")
    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    threads = max(1, min(cores, 16))
    t, _ = oracle.timed_govm(wl.row_ptr, wl.col, wl.weights, [int(wl.sources[0])], threads=1)
    per_step = max(1, min(len(wl.sources), threads * max(1, int(4.0 / max(t, 1e-3)))))  # about 4 s per thread
    step_sources = [int(s) for s in wl.sources[:per_step]]
    for _ in range(args.warmup):
        oracle.timed_govm(wl.row_ptr, wl.col, wl.weights, step_sources[:threads], threads=threads)
    total = 0.0
    for _ in range(args.steps):
        el, _ = oracle.timed_govm(wl.row_ptr, wl.col, wl.weights, step_sources, threads=threads)
        total += el
    value = args.steps * len(step_sources) * wl.e_wcc / total / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": wl.wtype, "data": "synthetic",
            # the workload of the GPU arm's line, key for key; what one timed step of
            # this arm solves is the sample below
            "config": {"workload": wl.name, "n": wl.n, "m": wl.m, "e_wcc": wl.e_wcc, "s_wcc": wl.s_wcc,
                       "sources_per_step": len(wl.sources) * args.gpus, "parallelism": f"replicas{args.gpus}",
                       "l2": l2_rule(wl.n, wl.m, l2_bytes(0))[1]},
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": threads, "kind": "oracle",
                             "sample": f"{len(step_sources)} of the workload's {len(wl.sources)} sources per step, "
                                       f"literal GOVM (Algorithm 2), one source per thread"},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main_ours(args):
    world, rank, local = dist_env()
    init_dist(world, local)
    device = local
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the solver has no CPU path)")
    if args.workload.startswith("rmat") or args.workload in ("grid", "tiny"):
        t = time.time()
        wl = make_workload(args.workload, rank, world)
        if args.sources:
            wl.sources = wl.sources[:args.sources]
        log(f"[bench] {wl.name}: n={wl.n} m={wl.m} e_wcc={wl.e_wcc} sources={len(wl.sources)} "
            f"(generated in {time.time() - t:.1f} s)")
        res = run_sssp_bench(args, wl, device, world, rank)
        log(f"[bench] device: {res['gteps']:.2f} GTEPS, {res['launch_ms_mean']:.3f} ms/launch, "
            f"B_alg {res['b_alg_mean'] / 1e9:.3f} GB, {res['achieved_gbs']:.0f} GB/s, steps {res['steps_mean']:.1f}")
        e2e = run_e2e(args, wl, device, world, res["tuning"]) if not args.no_e2e else None
        cpu = cpu_baseline(wl, args.cpu_budget, res["dist_host"]) if (rank == 0 and not args.no_cpu) else None
        if rank != 0:
            return
        peak, peak_kind = measured_peak()
        line = {
            "metric": METRIC, "value": res["gteps"], "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["elapsed"] / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": wl.wtype, "data": "synthetic",
            "config": {"workload": wl.name, "n": wl.n, "m": wl.m, "e_wcc": wl.e_wcc, "s_wcc": wl.s_wcc,
                       "sources_per_step": len(wl.sources) * world, "parallelism": f"replicas{world}",
                       "l2": res["l2"]},
            "roofline": {"bound": "hbm", "achieved": res["achieved_gbs"], "peak": peak, "unit": "GB/s",
                         "frac": res["achieved_gbs"] / peak, "traffic": recorded_traffic(wl.name),
                         "peak_kind": f"{peak_kind} copy bandwidth", "kernel": "govm_kernel",
                         "b_alg_per_launch": res["b_alg_mean"], "launch_ms": res["launch_ms_mean"],
                         "frac_of_8000": res["achieved_gbs"] / 8000.0,
                         "b_min_per_launch": res["b_min_mean"],
                         "frac_b_min": res["achieved_gbs_b_min"] / peak},
            "gather_ceiling": None,
            "gteps_median": res["gteps_median"], "gteps_hmean_per_launch": res["gteps_hmean"],
            "solver": {"steps_mean": res["steps_mean"], "updates_mean": res["updates_mean"], "mu_gpu": res["mu_gpu"],
                       "edges_scanned_mean": res["edges_scanned_mean"],
                       "edges_scanned_over_e_wcc": res["edges_scanned_mean"] / wl.e_wcc},
            "e2e": e2e, "gpu_launches": res["launches"], "clocks": res["clocks"], "cpu_baseline": cpu,
            "tuning": res["tuning"],
        }
        if world == 1 and not args.no_legs:
            # the random-gather rate of this GPU, and the rate of state reads
            # (one per scanned edge, one per frontier vertex) the solver made
            gc = gather_ceiling(device, wl.n)
            req = (res["edges_scanned_mean"] + res["frontier_sum_mean"]) / (res["launch_ms_mean"] / 1e3)
            line["gather_ceiling"] = gc
            line["roofline"]["state_reads_per_s"] = req
            line["roofline"]["frac_of_gather_ceiling"] = req / gc["gathers_per_s"]
        if world == 1 and args.workload == "rmat22" and not args.no_legs:
            # the rest of the metric: high-diameter, batched and
            # differentiable forms beside the plain solver, each with its own
            # clocks, roofline and oracle leg
            t = time.time()
            line["msssp_rmat22_64"] = leg_c2_batched(args, wl, res, device)
            log(f"[bench] leg msssp_rmat22_64 done in {time.time() - t:.1f} s")
            for key, fn in (("grid_2048_f32", leg_grid), ("msssp_rmat18_1024", leg_msssp),
                            ("roots_er64", leg_roots), ("diff_rmat16_f32", leg_diff)):
                t = time.time()
                line[key] = fn(args, device)
                log(f"[bench] leg {key} done in {time.time() - t:.1f} s")
        print(json.dumps(line), flush=True)
    elif args.workload in ("batched", "batched22", "diff", "mu", "apsp", "gsvm"):
        if world > 1 and rank != 0:
            return
        res = {"batched": run_batched, "batched22": run_batched22, "diff": run_diff, "mu": run_mu,
               "apsp": run_apsp, "gsvm": run_gsvm}[args.workload](args)
        print(json.dumps({"workload": args.workload, "results": res}), flush=True)
    else:
        raise SystemExit(f"unknown workload {args.workload}")


def build_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat22")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch shape (no autotuning)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--sources", type=int, default=0, help="limit sources per step (profiling runs)")
    ap.add_argument("--no-legs", action="store_true",
                    help="only the R-MAT s22 line: skip the grid, batched and backward legs and the gather ceiling")
    return ap


def main():
    args = build_parser().parse_args()
    if args.warmup < 3:
        log("[bench] warm-up raised to 3 steps")
        args.warmup = 3
    if args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
