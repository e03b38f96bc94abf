"""Planted mistakes in the oracle must be caught by its pins (no GPU).

Each mutant below is one plausible slip in ``oracle/oracle.c`` or
``oracle/__init__.py``: a flipped or loosened comparison, a dropped term,
guard or reset, a wrong index or operand.  For every mutant the test copies
the oracle package into a temporary directory, applies that one change, and
runs the independent pins of ``tests/test_oracle.py`` (closed forms, scipy /
networkx routines, exhaustive search, the paper's unit-weight properties,
planted certificate mistakes) against the copy in a fresh interpreter.  At
least one pin must fail.  The unmodified copy must pass, so a failure is the
mutant's doing.

The stored values under ``tests/golden`` are left out on purpose: they were
written by the oracle itself, so they would flag any change at all, right or
wrong, and say nothing about whether the pins are independent.
"""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C, PY = "oracle.c", "__init__.py"

# (name, file, text to replace, replacement, which occurrence (0-based) or
# None when the text must be unique)
MUTANTS = [
    # Algorithm 2 (GOVM), Section 3.4
    ("govm_u32: relaxation test loosened to >=", C,
     "if (alpha[index] > alpha[j] + value && !is_root[index]) {\n            alpha[index] = alpha[j] + value;\n"
     "            beta[index] = 1;",
     "if (alpha[index] >= alpha[j] + value && !is_root[index]) {\n            alpha[index] = alpha[j] + value;\n"
     "            beta[index] = 1;", 0),
    ("govm_u32: improved vertex not marked in beta", C,
     "            alpha[index] = alpha[j] + value;\n            beta[index] = 1;\n",
     "            alpha[index] = alpha[j] + value;\n", 0),
    ("govm_u32: beta not cleared after delta <= beta", C,
     "    memset(beta, 0, (size_t)n);     /* beta <= 0 */\n", "", None),
    ("govm_u32: the last edge of every row skipped", C,
     "        st->frontier_sum++;\n        for (int32_t e = start; e < end; ++e) {\n          int32_t index = col[e];\n"
     "          uint64_t value = w[e];",
     "        st->frontier_sum++;\n        for (int32_t e = start; e < end - 1; ++e) {\n          int32_t index = col[e];\n"
     "          uint64_t value = w[e];", 0),
    ("govm_u32: roots not put in the first frontier", C,
     "for (int32_t i = 0; i < k; ++i) { alpha[roots[i]] = 0; delta[roots[i]] = 1; }",
     "for (int32_t i = 0; i < k; ++i) { alpha[roots[i]] = 0; }", 0),
    ("govm_u32: candidate uses the target's distance", C,
     "if (alpha[index] > alpha[j] + value && !is_root[index]) {\n            alpha[index] = alpha[j] + value;\n"
     "            beta[index] = 1;",
     "if (alpha[index] > alpha[j] + value && !is_root[index]) {\n            alpha[index] = alpha[index] + value;\n"
     "            beta[index] = 1;", 0),
    ("govm_u32: update counter also counts scanned edges", C,
     "          uint64_t value = w[e];\n          st->edges_scanned++;\n",
     "          uint64_t value = w[e];\n          st->edges_scanned++;\n          st->updates++;\n", 0),
    ("govm_u32: stops one step early", C,
     "    if (!ptr) { st->converged = 1; break; }\n    memcpy(delta, beta, (size_t)n); /* delta <= beta */",
     "    if (!ptr || step == 3) { st->converged = 1; break; }\n    memcpy(delta, beta, (size_t)n); /* delta <= beta */",
     None),
    ("govm_f32: comparison operands swapped", C,
     "          float cand = alpha[j] + value;\n          if (alpha[index] > cand && !is_root[index]) {",
     "          float cand = alpha[j] + value;\n          if (cand > alpha[index] && !is_root[index]) {",
     None),
    ("govm_f32: candidate summed in double without rounding to float", C,
     "          float cand = alpha[j] + value;\n          if (alpha[index] > cand && !is_root[index]) {\n"
     "            alpha[index] = cand;",
     "          double cand = (double)alpha[j] + (double)value;\n"
     "          if ((double)alpha[index] > cand && !is_root[index]) {\n            alpha[index] = (float)cand;",
     None),
    # Algorithm 1 (GSVM), Section 3.2
    ("gsvm_u32: single sweep instead of iterating to the fixpoint", C,
     "              count[index]++;\n              st->updates++;\n              ptr = 1;\n            }\n          }\n        }\n      }\n    }\n"
     "    if (!ptr) { st->converged = 1; break; }",
     "              count[index]++;\n              st->updates++;\n              ptr = 1;\n            }\n          }\n        }\n      }\n    }\n"
     "    if (1) { st->converged = 1; break; }", 0),
    ("gsvm_f32: source guard dropped and scan limited to unreached rows", C,
     "      if (alpha[j] != INFINITY) {\n        int32_t start = row_ptr[j], end = row_ptr[j + 1];",
     "      if (alpha[j] == 0.0f) {\n        int32_t start = row_ptr[j], end = row_ptr[j + 1];", None),
    # Dijkstra (Section 2.1), shared heap
    ("heap_pop: sift-down follows the larger child", C,
     "if (l < h->size && h->a[l].key < ck) { c = l; ck = h->a[l].key; }",
     "if (l < h->size && h->a[l].key > ck) { c = l; ck = h->a[l].key; }", None),
    ("heap_push: sift-up compares the wrong way", C,
     "    if (h->a[p].key <= key) break;", "    if (h->a[p].key >= key) break;", None),
    ("dijkstra_u32: relaxation into a settled vertex's neighbours skipped", C,
     "      uint64_t cand = dist[u] + w[e];\n      if (cand < dist[v]) {",
     "      uint64_t cand = dist[u] + w[e];\n      if (cand < dist[v] && e == row_ptr[u]) {", None),
    ("dijkstra_u32: distance sum truncated to 32 bits", C,
     "      uint64_t cand = dist[u] + w[e];\n      if (cand < dist[v]) {",
     "      uint64_t cand = (uint32_t)(dist[u] + w[e]);\n      if (cand < dist[v]) {", None),
    ("dijkstra_f64: source guard dropped into a heap keyed on the wrong value", C,
     "      double cand = dist[u] + w[e];\n      if (cand < dist[v]) {\n        dist[v] = cand;\n"
     "        rc |= heap_push(&h, cand, v);",
     "      double cand = dist[u] + w[e];\n      if (cand < dist[v]) {\n        dist[v] = cand;\n"
     "        rc |= heap_push(&h, w[e], v);", None),
    # Floyd-Warshall (Section 2.3)
    ("fw_u32: parallel edges keep the last one, not the lightest", C,
     "      if (col[e] != u && w[e] < D[(int64_t)u * n + col[e]]) D[(int64_t)u * n + col[e]] = w[e];\n"
     "  for (int32_t kk = 0; kk < n; ++kk)\n    for (int32_t i = 0; i < n; ++i) {\n      uint64_t dik",
     "      if (col[e] != u) D[(int64_t)u * n + col[e]] = w[e];\n"
     "  for (int32_t kk = 0; kk < n; ++kk)\n    for (int32_t i = 0; i < n; ++i) {\n      uint64_t dik", None),
    ("fw_u32: transposed intermediate term", C,
     "        uint64_t dkj = D[(int64_t)kk * n + j];", "        uint64_t dkj = D[(int64_t)j * n + kk];", None),
    ("fw_f32: pivot loop runs one short", C,
     "  for (int32_t kk = 0; kk < n; ++kk)\n    for (int32_t i = 0; i < n; ++i) {\n      float dik",
     "  for (int32_t kk = 0; kk < n - 1; ++kk)\n    for (int32_t i = 0; i < n; ++i) {\n      float dik", None),
    # Parent rule (lowest edge index) and the certificate
    ("parents_u32: last matching edge wins", C,
     "      if (is_root[v] || parent_edge[v] != -1) continue;\n      if (dist[u] + w[e] == dist[v]) parent_edge[v] = e;",
     "      if (is_root[v]) continue;\n      if (dist[u] + w[e] == dist[v]) parent_edge[v] = e;", 0),
    ("parents_f32: tolerance instead of exact equality", C,
     "      float s = dist[u] + w[e];\n      if (s == dist[v]) parent_edge[v] = e;",
     "      float s = dist[u] + w[e];\n      if (s <= dist[v] * 1.001f) parent_edge[v] = e;", None),
    ("cert_u32: edge-relaxation check dropped", C,
     "      if (!is_root[col[e]] && dist[u] + w[e] < dist[col[e]]) { rc = 2; *where = e; break; }",
     "      if (0) { rc = 2; *where = e; break; }", 0),
    ("cert_u32: parent edge tightness not checked", C,
     "    if (!finite[lo] || dist[lo] + w[e] != dist[v]) { rc = 3; *where = v; }",
     "    if (!finite[lo]) { rc = 3; *where = v; }", 0),
    ("cert_u32: root distance not checked", C,
     "    if (is_root[v] && (dist[v] != 0 || parent_edge[v] != -1)) { rc = 1; *where = v; }",
     "    if (is_root[v] && parent_edge[v] != -1) { rc = 1; *where = v; }", 0),
    ("cert_tree: cycles in the parent edges accepted", C,
     "    if (!is_root[v] && state[v] == 1) { rc = 5; *where = v; }", "", None),
    ("cert_f32: unreachable vertex with a parent edge accepted", C,
     "    if (!finite[v]) { if (e != -1) { rc = 4; *where = v; } continue; }",
     "    if (!finite[v]) { continue; }", 1),
    # Gradient of L = sum_t c_t dist[t]
    ("subtree_grad: subtree sums not passed to the parent", C,
     "    grad_w[e] = acc[v];\n    acc[lo] += acc[v];", "    grad_w[e] = acc[v];\n    acc[lo] = acc[v];", None),
    ("subtree_grad: edge gets the vertex's own weight only", C,
     "    grad_w[e] = acc[v];\n    acc[lo] += acc[v];", "    grad_w[e] = c[v];\n    acc[lo] += acc[v];", None),
    # Signed weights
    ("govm_i32: source guard dropped", C,
     "          int64_t value = w[e];\n          st->edges_scanned++;\n          if (alpha[index] > alpha[j] + value && !is_root[index]) {",
     "          int64_t value = w[e];\n          st->edges_scanned++;\n          if (alpha[index] > alpha[j] + value) {", None),
    ("bellman_ford_i32: negative-cycle round dropped", C,
     "      if (!is_root[col[e]] && dist[u] + w[e] < dist[col[e]]) { rc = 4; break; }",
     "      if (0) { rc = 4; break; }", None),
    ("bellman_ford_i32: one round short", C,
     "  for (int32_t round = 0; round < n - 1; ++round) {", "  for (int32_t round = 0; round < n - 2; ++round) {",
     None),
    ("gsvm_u32: relaxation test loosened to >=", C,
     "            if (alpha[index] > alpha[j] + value && !is_root[index]) {\n              alpha[index] = alpha[j] + value;\n"
     "              count[index]++;",
     "            if (alpha[index] >= alpha[j] + value && !is_root[index]) {\n              alpha[index] = alpha[j] + value;\n"
     "              count[index]++;", None),
    ("govm_i32: relaxation test loosened to >=", C,
     "          int64_t value = w[e];\n          st->edges_scanned++;\n          if (alpha[index] > alpha[j] + value && !is_root[index]) {",
     "          int64_t value = w[e];\n          st->edges_scanned++;\n          if (alpha[index] >= alpha[j] + value && !is_root[index]) {",
     None),
    ("parents_i32: last matching edge wins", C,
     "      if (is_root[v] || parent_edge[v] != -1) continue;\n      if (dist[u] + w[e] == dist[v]) parent_edge[v] = e;",
     "      if (is_root[v]) continue;\n      if (dist[u] + w[e] == dist[v]) parent_edge[v] = e;", 1),
    ("cert_i32: edge-relaxation check dropped", C,
     "      if (!is_root[col[e]] && dist[u] + w[e] < dist[col[e]]) { rc = 2; *where = e; break; }",
     "      if (0) { rc = 2; *where = e; break; }", 1),
    ("cert_i32: parent edge tightness not checked", C,
     "    if (!finite[lo] || dist[lo] + w[e] != dist[v]) { rc = 3; *where = v; }",
     "    if (!finite[lo]) { rc = 3; *where = v; }", 1),
    # Pure Python / numpy routines of the oracle
    ("_u64_to_u32: distances past the sentinel silently truncated", PY,
     "    if np.any(d[fin] >= np.uint64(0xFFFFFFFF)):\n        raise OverflowError(\"a shortest distance does not fit below 0xFFFFFFFF\")",
     "    if False:\n        raise OverflowError(\"a shortest distance does not fit below 0xFFFFFFFF\")", None),
    ("_i64_to_i32: negative overflow not checked", PY,
     " or np.any(d[fin] < np.int64(-2 ** 31)):", ":", None),
    ("edge_tails: tails shifted by one row", PY,
     "    return np.repeat(np.arange(len(row_ptr) - 1, dtype=np.int32), np.diff(row_ptr))",
     "    return np.repeat(np.arange(1, len(row_ptr), dtype=np.int32) % (len(row_ptr) - 1), np.diff(row_ptr))", None),
    ("dense_colmin: transposed operand in A_s[k, j] = a_s[k] + a[k, j]", PY,
     "        As = a[:, None] + A", "        As = a[None, :] + A", None),
    ("brute_force: path value folded in double, not fp32", PY,
     "            nv = np.float32(val + w[e]) if f32 else val + int(w[e])",
     "            nv = float(val) + float(w[e]) if f32 else val + int(w[e])", None),
    ("brute_force: keeps the longest path", PY,
     "            if best[v] is None or nv < best[v]:", "            if best[v] is None or nv > best[v]:", None),
    ("parent_vertices: parent edge index returned as the parent vertex", PY,
     "    p[has] = tails[parent_edge[has]]", "    p[has] = parent_edge[has]", None),
    ("subtree_grad: vertices visited parents first", PY,
     "    order = np.argsort(-np.where(np.isfinite(d64), d64, -1.0), kind=\"stable\").astype(np.int32)",
     "    order = np.argsort(np.where(np.isfinite(d64), d64, -1.0), kind=\"stable\").astype(np.int32)", None),
    ("fd_grad: one-sided step in the central difference", PY,
     "        out[i] = (loss(dp) - loss(dm)) / (2 * h)", "        out[i] = (loss(dp) - loss(dm)) / h", None),
    ("fd_grad: both perturbations in the same direction", PY,
     "        wm[e] -= h", "        wm[e] += h", None),
]


def _apply(src: str, old: str, new: str, occurrence):
    count = src.count(old)
    if occurrence is None:
        assert count == 1, f"mutation site must be unique, found {count}"
        return src.replace(old, new)
    assert count > occurrence, f"mutation site occurrence {occurrence} not found ({count})"
    i = -1
    for _ in range(occurrence + 1):
        i = src.index(old, i + 1)
    return src[:i] + new + src[i + len(old):]


def run_pins(mutant):
    """Run tests/test_oracle.py against a copy of the oracle with `mutant`
    applied (None: no change).  Returns (exit code, output)."""
    tmp = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(tmp, "oracle"),
                        ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
        os.symlink(os.path.join(ROOT, "graphgen"), os.path.join(tmp, "graphgen"))
        os.makedirs(os.path.join(tmp, "tests"))
        for f in ("__init__.py", "conftest.py", "test_oracle.py"):
            shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(tmp, "tests", f))
        if mutant is not None:
            _, fname, old, new, occ = mutant
            path = os.path.join(tmp, "oracle", fname)
            with open(path) as f:
                src = f.read()
            with open(path, "w") as f:
                f.write(_apply(src, old, new, occ))
        env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
        p = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle.py", "-x", "-q", "-p", "no:cacheprovider"],
                           cwd=tmp, env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True, timeout=600)
        return p.returncode, p.stdout
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


@pytest.fixture(scope="module")
def outcomes():
    import graphgen
    graphgen.build()  # the copies share the generator library: build it once, before they start
    workers = max(1, min(8, (os.cpu_count() or 1)))
    with ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(run_pins, [None] + MUTANTS))
    return res[0], dict(zip([m[0] for m in MUTANTS], res[1:]))


def test_mutation_sites_exist():
    for name, fname, old, new, occ in MUTANTS:
        with open(os.path.join(ROOT, "oracle", fname)) as f:
            _apply(f.read(), old, new, occ)


def test_unmodified_copy_passes_the_pins(outcomes):
    rc, out = outcomes[0]
    assert rc == 0, out[-2000:]


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(outcomes, name):
    rc, out = outcomes[1][name]
    assert rc == 1, f"the pins did not catch '{name}' (pytest exit {rc}):\n{out[-1500:]}"
