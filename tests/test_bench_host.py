"""Host logic of bench.py on CPU (no GPU): the reference arm's JSON line,
the algorithmic-byte and roofline arithmetic, the lookup of committed ncu
traffic by kernel-source hash, and the oracle legs that sit beside the GPU
results."""
import json
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import bench
import graphgen as gg
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "2",
                        "--warmup", "3"], cwd=ROOT, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "GTEPS" and line["higher_is_better"] is True
    assert line["metric"] == bench.METRIC and line["steps"] == 2 and line["warmup"] == 3
    assert line["value"] > 0 and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == gg.tiny_er().name


def test_bytes_alg_and_roofline_arithmetic():
    st = {"frontier_sum": 10, "edges_scanned": 100, "updates": 7}
    assert bench.bytes_alg(st) == 16 * 10 + 12 * 100 + 12 * 7
    r = bench.roofline_entry(2e9, 1e-3, "k", "rule")
    peak, kind = bench.measured_peak()
    assert r["achieved"] == pytest.approx(2000.0) and r["peak"] == peak
    assert r["frac"] == pytest.approx(2000.0 / peak) and r["unit"] == "GB/s" and kind in r["peak_kind"]


def test_recorded_traffic_follows_the_kernel_source_hash(monkeypatch):
    # each committed summary applies to the kernel sources it names, and
    # only to those
    summaries = {"rmat_s22_ef16_u32": "govm_kernel_rmat22_traffic.md", "grid_2048x2048_f32": "govm_kernel_grid2048_traffic.md"}
    for workload, fname in summaries.items():
        with open(os.path.join(ROOT, "profiles", fname)) as f:
            text = f.read()
        rec_hash = re.search(r"kernel_source_sha256_16: `?([0-9a-f]{16})", text).group(1)
        rec_bytes = float(re.search(r"dram_bytes_per_launch: `?([0-9.e+]+)", text).group(1))
        current = bench.kernel_hash()
        assert bench.recorded_traffic(workload) == (pytest.approx(rec_bytes) if rec_hash == current else None)
        monkeypatch.setattr(bench, "kernel_hash", lambda: rec_hash)
        assert bench.recorded_traffic(workload) == pytest.approx(rec_bytes)
        monkeypatch.setattr(bench, "kernel_hash", lambda: "0123456789abcdef")
        assert bench.recorded_traffic(workload) is None
        monkeypatch.undo()
    assert bench.recorded_traffic("no_such_workload") is None


def test_oracle_legs_beside_batched_and_backward_results():
    wl = gg.rmat_u32(11, 16, nsrc=16, seed=1)
    rows = np.stack([oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, int(s)) for s in wl.sources[:4]])
    out = bench.cpu_leg_sources(wl, rows, 0.5)
    assert out["bit_exact_vs_gpu"] == {"rows_compared": 4, "all_equal": True}
    bad = rows.copy()
    bad[2, int(np.argmax(bad[2] != 0xFFFFFFFF))] ^= 1  # one flipped bit in a reached distance
    assert bench.cpu_leg_sources(wl, bad, 0.5)["bit_exact_vs_gpu"]["all_equal"] is False

    wb = gg.er_batch(count=4, nlo=100, nhi=800, dlo=2, dhi=6, seed=2)
    d = oracle.dijkstra(wb.row_ptr, wb.col, wb.weights, wb.sources)
    assert bench.cpu_leg_roots(wb, d)["bit_exact_vs_gpu"] is True

    wd = gg.rmat_f32_diff(scale=9, edge_factor=8, ntargets=16, seed=0)
    c = np.zeros(wd.n, np.float32)
    c[wd.extra["targets"]] = wd.extra["coef"]
    g = oracle.subtree_grad(wd.row_ptr, wd.col, wd.weights, 0, c).astype(np.float32)
    assert bench.cpu_leg_diff(wd, c, g)["max_abs_err_over_max_ref"] < 1e-6


def _bench_commands(text):
    """Argument lists of every `python bench.py ...` command quoted in a
    profile summary (continuation lines joined, redirections and pipes cut)."""
    import shlex
    joined = text.replace("\\\n", " ")
    out = []
    for line in joined.splitlines():
        i = line.find("python bench.py")
        if i < 0:
            continue
        rest = line[i + len("python bench.py"):]
        for stop in ("&&", ">", "|", "#", "`"):
            rest = rest.split(stop)[0]
        out.append(shlex.split(rest))
    return out


def test_profile_commands_run_committed_files_with_current_flags():
    known = {"grid", "tiny", "batched", "batched22", "diff", "mu", "apsp", "gsvm"}
    pdir = os.path.join(ROOT, "profiles")
    files = sorted(f for f in os.listdir(pdir) if f.endswith(".md"))
    assert files
    for f in files:
        with open(os.path.join(pdir, f)) as fh:
            text = fh.read()
        cmds = _bench_commands(text)
        assert cmds, f"{f} quotes no bench.py command"
        for argv in cmds:
            args = bench.build_parser().parse_args(argv)
            w = args.workload
            assert w in known or (w.startswith("rmat") and w[4:].isdigit()), (f, w)
        ncu_lines = [l for l in text.replace("\\\n", " ").splitlines() if re.search(r"(^|&&)\s*ncu\s", l.strip())]
        for line in ncu_lines:
            assert "--clock-control none" in line, (f, line)


def test_l2_rule_and_clock_summary():
    l2 = 132 * 2 ** 20
    flush, note = bench.l2_rule(1024, 8192, l2)  # the tiny ER graph: 69 KB
    assert flush and "fits in L2" in note and "0.1 MB" in note
    flush, note = bench.l2_rule(1 << 22, 65_243_778, l2)  # R-MAT s22: 539 MB
    assert not flush and "larger than L2" in note and "539 MB" in note
    assert bench.graph_bytes(10, 7) == 4 * 11 + 8 * 7
    lines = ["0, 1500, 2070, 300.1, 0x0, Not Active, Not Active, Not Active, Not Active, 0",
             "0, 2070, 2070, 900.5, 0x4, Not Active, Not Active, Not Active, Active, 100",
             "0, 2060, 2070, 901.0, 0x0, Not Active, Not Active, Not Active, Not Active, 97"]
    s = bench.clocks_summary(lines)
    assert s["sm_mhz"] == 2065 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["samples_under_load"] == 2 and s["reasons"] == ["sw_power_cap"]
    assert bench.clocks_summary([])["reasons"] == ["unsampled"]
    # the older nine-field form (no utilisation) still parses
    assert bench.clocks_summary([l.rsplit(",", 1)[0] for l in lines])["sm_mhz"] == 2060
