"""Pins for the CPU oracle (no GPU).

Each test ties an oracle routine to something other than itself: closed
forms, library routines (scipy, networkx), exhaustive enumeration, the
paper's stated properties (unit weights give mu = 1, Section 4.2; GOVM equals
the Floyd-Warshall recurrence, Section 3.1), and planted mistakes that the
certificate must reject.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

scipy_csgraph = pytest.importorskip("scipy.sparse.csgraph")
import scipy.sparse as sp  # noqa: E402

INF32 = np.uint32(0xFFFFFFFF)


def scipy_dist(row_ptr, col, w, source):
    """scipy Dijkstra in float64 (exact for integer weights); parallel edges
    are reduced to their minimum first because scipy's csr sums duplicates."""
    n = len(row_ptr) - 1
    tails = oracle.edge_tails(row_ptr)
    best = {}
    for u, v, x in zip(tails, col, np.asarray(w, dtype=np.float64)):
        if u == v:
            continue
        key = (int(u), int(v))
        if key not in best or x < best[key]:
            best[key] = x
    if best:
        uu, vv = zip(*best.keys())
        A = sp.csr_matrix((list(best.values()), (uu, vv)), shape=(n, n))
    else:
        A = sp.csr_matrix((n, n))
    return scipy_csgraph.dijkstra(A, directed=True, indices=source)


def as_float(d):
    d = np.asarray(d)
    if d.dtype == np.uint32:
        out = d.astype(np.float64)
        out[d == INF32] = np.inf
        return out
    return d.astype(np.float64)


ALL = ("govm", "gsvm", "dijkstra")


def run(alg, rp, cl, w, roots):
    if alg == "dijkstra":
        return oracle.dijkstra(rp, cl, w, roots)
    return oracle.govm(rp, cl, w, roots, algorithm=alg)[0]


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("alg", ALL)
def test_path_graph_prefix_sums(alg):
    # 0 -> 1 -> ... -> 9, dist[k] = w0 + ... + w_{k-1}
    ws = [3, 1, 4, 1, 5, 9, 2, 6, 5]
    rp, cl, w = gg.csr_from_edges(10, [(i, i + 1) for i in range(9)], ws)
    d = run(alg, rp, cl, w, 0)
    assert d.tolist() == [0] + list(np.cumsum(ws))


def test_path_graph_step_and_work_counts():
    # 0 -> 1 -> ... -> 9.  Algorithm 2 expands one new vertex per step (9
    # steps that change a path, then one that changes nothing): 9 edges
    # scanned, 9 updates.  Algorithm 1 sweeps the reached vertices in id
    # order with alpha updated in place, so its first sweep reaches the whole
    # path and its second changes nothing: 2 steps, 9 + 9 edges scanned.
    ws = [3, 1, 4, 1, 5, 9, 2, 6, 5]
    rp, cl, w = gg.csr_from_edges(10, [(i, i + 1) for i in range(9)], ws)
    _, st = oracle.govm(rp, cl, w, 0)
    assert (st["steps"], st["edges_scanned"], st["updates"], st["converged"]) == (10, 9, 9, 1)
    _, st = oracle.gsvm(rp, cl, w, 0)
    assert (st["steps"], st["edges_scanned"], st["updates"], st["converged"]) == (2, 18, 9, 1)


@pytest.mark.parametrize("alg", ("govm", "gsvm"))
@pytest.mark.parametrize("kind", ("u32", "f32"))
def test_iterations_stop_when_a_step_changes_nothing(alg, kind):
    # both algorithms end by their "no path changed" test, long before the
    # step cap n; a step that changes nothing scans every edge it would scan
    # again, so a run that never stops would hit the cap
    rp, cl, w = gg.random_small(300, 2400, 5, kind=kind, wlo=1, whi=20)
    _, st = oracle.govm(rp, cl, w, 0, algorithm=alg)
    assert st["converged"] == 1 and st["steps"] < 300 // 2


@pytest.mark.parametrize("alg", ALL)
def test_complete_graph_squared_weights(alg):
    # edges i -> j (i < j) with weight (j - i)^2: unit steps win, dist[j] = j.
    n = 12
    edges = [(i, j) for i in range(n) for j in range(i + 1, n)]
    rp, cl, w = gg.csr_from_edges(n, edges, [(j - i) ** 2 for i, j in edges])
    d = run(alg, rp, cl, w, 0)
    assert d.tolist() == list(range(n))


def test_complete_graph_needs_path_updates():
    # the direct edges are found first and then improved: mu > 1 (Section 3.4)
    n = 12
    edges = [(i, j) for i in range(n) for j in range(i + 1, n)]
    rp, cl, w = gg.csr_from_edges(n, edges, [(j - i) ** 2 for i, j in edges])
    _, st = oracle.govm(rp, cl, w, 0)
    assert st["updates"] > n - 1 and st["mu"] > 1.0
    # GSVM rescans every reached vertex each step: more edges examined
    _, st_gsvm = oracle.gsvm(rp, cl, w, 0)
    assert st_gsvm["edges_scanned"] > st["edges_scanned"]


@pytest.mark.parametrize("alg", ALL)
def test_unreachable_and_isolated(alg):
    # component {0,1,2}; vertices 3,4 unreachable (4 -> 3 edge only)
    rp, cl, w = gg.csr_from_edges(5, [(0, 1), (1, 2), (4, 3)], [7, 8, 1])
    d = run(alg, rp, cl, w, 0)
    assert d.tolist() == [0, 7, 15, int(INF32), int(INF32)]
    # source with out-degree 0
    d = run(alg, rp, cl, w, 2)
    assert d.tolist() == [int(INF32), int(INF32), 0, int(INF32), int(INF32)]


@pytest.mark.parametrize("alg", ALL)
def test_single_vertex_and_no_edges(alg):
    rp = np.array([0, 0], np.int32)
    cl = np.zeros(0, np.int32)
    assert run(alg, rp, cl, np.zeros(0, np.uint32), 0).tolist() == [0]
    assert np.isposinf(run(alg, np.zeros(4, np.int32), cl, np.zeros(0, np.float32), 1)[[0, 2]]).all()


@pytest.mark.parametrize("alg", ALL)
def test_edges_into_source_ignored(alg):
    # the source guard: a zero-weight edge back into the source
    rp, cl, w = gg.csr_from_edges(3, [(0, 1), (1, 0), (1, 2)], [0, 0, 5])
    d = run(alg, rp, cl, w, 0)
    assert d.tolist() == [0, 0, 5]
    pe = oracle.parent_edges(rp, cl, w, 0, d)
    assert pe[0] == -1


@pytest.mark.parametrize("alg", ALL)
def test_self_loops_and_parallel_edges(alg):
    # parallel edges 0->1 with weights 9, 4, 6 and a self-loop on 1
    rp, cl, w = gg.csr_from_edges(3, [(0, 1), (0, 1), (0, 1), (1, 1), (1, 2)], [9, 4, 6, 0, 1])
    d = run(alg, rp, cl, w, 0)
    assert d.tolist() == [0, 4, 5]
    pe = oracle.parent_edges(rp, cl, w, 0, d)
    assert pe.tolist() == [-1, 1, 4]


def test_large_uint32_weights_no_overflow():
    # distances up to 3 * (2^30 - 1) < 2^32 - 1 stay exact
    big = (1 << 30) - 1
    rp, cl, w = gg.csr_from_edges(4, [(0, 1), (1, 2), (2, 3)], [big, big, big])
    for alg in ALL:
        assert run(alg, rp, cl, w, 0).tolist() == [0, big, 2 * big, 3 * big]
    # a distance that does not fit below the 0xFFFFFFFF sentinel is reported
    rp, cl, w = gg.csr_from_edges(3, [(0, 1), (1, 2)], [0xFFFFFFFE, 0xFFFFFFFE])
    with pytest.raises(OverflowError):
        oracle.dijkstra(rp, cl, w, 0)


# ------------------------------------------------------------ fp32 semantics

@pytest.mark.parametrize("alg", ALL)
def test_fp32_left_fold_rounding(alg):
    # Path A: 2^24, then +1, +1: fl32 gives 2^24 after each +1 (ties to
    # even), so A's value is 2^24.  Path B: one edge of 2^24 + 2.  In exact
    # arithmetic both are 2^24 + 2; under fl32 left folds A is shorter.
    t24 = np.float32(2.0 ** 24)
    rp, cl, w = gg.csr_from_edges(4, [(0, 1), (1, 2), (2, 3), (0, 3)],
                                  [t24, 1.0, 1.0, t24 + np.float32(2.0)], np.float32)
    d = run(alg, rp, cl, w, 0)
    assert d[3] == t24 and d[2] == t24
    assert oracle.brute_force(rp, cl, w, 0)[3] == t24


@pytest.mark.parametrize("alg", ("govm", "gsvm"))
def test_fp32_candidate_rounding_to_current_distance_is_no_update(alg):
    # 0->2 (2^24), 0->1 (0.5), 1->2 (2^24 - 1).  The path through 1 sums to
    # 2^24 - 0.5 exactly, which rounds (ties to even) to 2^24 = dist[2]: in
    # fp32 it is not an improvement, so the run makes exactly two updates
    # (vertices 1 and 2 in step 1) and stops after step 2.
    rp, cl, w = gg.csr_from_edges(3, [(0, 2), (0, 1), (1, 2)], [2.0 ** 24, 0.5, 2.0 ** 24 - 1], np.float32)
    d, st = oracle.govm(rp, cl, w, 0, algorithm=alg)
    assert d.tolist() == [0.0, 0.5, 2.0 ** 24]
    assert st["updates"] == 2 and st["steps"] == 2 and st["converged"] == 1


@pytest.mark.parametrize("seed", range(30))
def test_fp32_brute_force_small(seed):
    # random fp32 weights (not dyadic): exact min over simple paths of the
    # fl32 left fold, by exhaustive enumeration
    n = 7
    rp, cl, w = gg.random_small(n, 18, seed, kind="f32", wlo=0.1, whi=10.0)
    bf = oracle.brute_force(rp, cl, w, 0)
    for alg in ALL:
        assert np.array_equal(run(alg, rp, cl, w, 0), bf), alg
    assert np.array_equal(oracle.dense_colmin(rp, cl, w, 0), bf)


@pytest.mark.parametrize("seed", range(30))
def test_u32_brute_force_small(seed):
    n = 8
    rp, cl, w = gg.random_small(n, 20, seed, kind="u32", wlo=0, whi=9, self_loops=True)
    bf = oracle.brute_force(rp, cl, w, 0)
    for alg in ALL:
        assert np.array_equal(run(alg, rp, cl, w, 0), bf), alg
    assert np.array_equal(oracle.dense_colmin(rp, cl, w, 0), bf)


# --------------------------------------------------------- library routines

@pytest.mark.parametrize("seed", range(8))
def test_u32_against_scipy(seed):
    rp, cl, w = gg.random_small(300, 2400, seed, kind="u32", wlo=1, whi=100)
    ref = scipy_dist(rp, cl, w, 5)
    for alg in ALL:
        assert np.array_equal(as_float(run(alg, rp, cl, w, 5)), ref), alg


@pytest.mark.parametrize("seed", range(4))
def test_u32_against_networkx(seed):
    nx = pytest.importorskip("networkx")
    rp, cl, w = gg.random_small(120, 700, seed, kind="u32", wlo=1, whi=50)
    G = nx.DiGraph()
    G.add_nodes_from(range(120))
    tails = oracle.edge_tails(rp)
    for u, v, x in zip(tails, cl, w):
        if u != v and (not G.has_edge(u, v) or G[u][v]["weight"] > int(x)):
            G.add_edge(int(u), int(v), weight=int(x))
    ref = nx.single_source_bellman_ford_path_length(G, 3)
    d = oracle.govm(rp, cl, w, 3)[0]
    for v in range(120):
        assert (d[v] == INF32) if v not in ref else (int(d[v]) == ref[v])


@pytest.mark.parametrize("seed", range(4))
def test_dyadic_fp32_against_scipy_and_fw(seed):
    # multiples of 1/16 below 2^20: every partial sum is exact in fp32, so
    # float64 scipy, Floyd-Warshall and the fl32 folds must all agree
    rp, cl, w = gg.random_small(64, 400, seed, kind="dyadic", wlo=0, whi=8)
    ref = scipy_dist(rp, cl, w, 0)
    D = oracle.floyd_warshall(rp, cl, w)
    for alg in ALL:
        d = run(alg, rp, cl, w, 0)
        assert np.array_equal(d.astype(np.float64), ref), alg
        assert np.array_equal(d, D[0]), alg


def test_fp32_close_to_float64():
    rp, cl, w = gg.random_small(500, 4000, 3, kind="f32", wlo=0.1, whi=10.0)
    ref = scipy_dist(rp, cl, w, 0)
    d = oracle.govm(rp, cl, w, 0)[0].astype(np.float64)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(d))
    assert np.allclose(d[fin], ref[fin], rtol=1e-5, atol=0)


def test_tiny_er_all_methods_agree():
    # the tiny workload: ER n=1024, m=8192, u32 U[1,100], source 0
    wl = gg.tiny_er()
    D = oracle.floyd_warshall(wl.row_ptr, wl.col, wl.weights)
    ref = scipy_dist(wl.row_ptr, wl.col, wl.weights, 0)
    for alg in ALL:
        d = run(alg, wl.row_ptr, wl.col, wl.weights, 0)
        assert np.array_equal(d, D[0]) and np.array_equal(as_float(d), ref)


def test_floyd_warshall_rows_equal_sssp():
    rp, cl, w = gg.random_small(40, 200, 9, kind="u32", wlo=1, whi=30)
    D = oracle.floyd_warshall(rp, cl, w)
    for s in range(40):
        assert np.array_equal(D[s], oracle.dijkstra(rp, cl, w, s))


# ------------------------------------------------------------- unit weights

@pytest.mark.parametrize("seed", range(3))
def test_unit_weights_are_bfs_levels_and_mu_is_one(seed):
    # Section 4.2: with unit weights every path is found once and never
    # changes (mu = 1); the distances are BFS levels.
    wl = gg.rmat_u32(12, 8, nsrc=1, seed=seed, wlo=1, whi=1)
    s = int(wl.sources[0])
    n = wl.n
    A = sp.csr_matrix((np.ones(wl.m), wl.col, wl.row_ptr), shape=(n, n))
    levels = scipy_csgraph.shortest_path(A, directed=True, unweighted=True, indices=s)
    d, st = oracle.govm(wl.row_ptr, wl.col, wl.weights, s)
    assert np.array_equal(as_float(d), levels)
    assert st["updates"] == st["reached"] - 1 and st["multi_updated"] == 0 and st["mu"] == 1.0
    # one step per BFS level plus the final step that changes nothing
    assert st["steps"] == int(levels[np.isfinite(levels)].max()) + 1
    # each reached vertex enters delta exactly once (at its own level), so the
    # work counters are closed forms: its out-edges are scanned once
    outdeg = np.diff(wl.row_ptr)
    fin = np.isfinite(levels)
    assert st["edges_scanned"] == int(outdeg[fin].sum())
    assert st["frontier_sum"] == int((outdeg[fin] > 0).sum())
    # with weights in [1, 255] paths do change: mu > 1
    wl2 = gg.rmat_u32(12, 8, nsrc=1, seed=seed)
    _, st2 = oracle.govm(wl2.row_ptr, wl2.col, wl2.weights, s)
    assert st2["mu"] > 1.0


# ---------------------------------------------------------------- multi-root

def test_multi_root_equals_per_component_solves():
    wl = gg.er_batch(count=5, nlo=50, nhi=400, dlo=2, dhi=6, seed=4)
    offs = wl.extra["offsets"]
    d_all = oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, wl.sources)
    d_govm = oracle.govm(wl.row_ptr, wl.col, wl.weights, wl.sources)[0]
    assert np.array_equal(d_all, d_govm)
    for i in range(5):
        d_one = oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, int(wl.sources[i]))
        sl = slice(int(offs[i]), int(offs[i + 1]))
        assert np.array_equal(d_all[sl], d_one[sl])
        assert np.all(d_one[: int(offs[i])] == INF32) and np.all(d_one[int(offs[i + 1]):] == INF32)


# ------------------------------------------------------------------ parents

def test_parent_rule_lowest_edge_index():
    # 0->1 (2), 0->2 (1), 2->1 (1): both edges into 1 are tight (dist 2);
    # the lower CSR index (edge 0, from vertex 0) is the parent.
    rp, cl, w = gg.csr_from_edges(3, [(0, 1), (0, 2), (2, 1)], [2, 1, 1])
    d = oracle.dijkstra(rp, cl, w, 0)
    pe = oracle.parent_edges(rp, cl, w, 0, d)
    assert d.tolist() == [0, 2, 1] and pe.tolist() == [-1, 0, 1]
    p = oracle.parent_vertices(rp, 0, d, pe, "u32")
    assert p.tolist() == [0, 0, 0]


def test_parent_rule_fp32_needs_exact_equality():
    # 0->1 (1), 0->2 (1), 1->3 (100 + 2^-17), 2->3 (100).  dist[3] = 101 via
    # vertex 2; the lower-indexed edge from 1 offers 101 + 2^-17, one ulp
    # above, so it is not tight and not the parent; the certificate rejects
    # it as a parent edge (code 3).
    w13 = np.nextafter(np.float32(100), np.float32(200))
    assert float(w13) == 100 + 2.0 ** -17
    rp, cl, w = gg.csr_from_edges(4, [(0, 1), (0, 2), (1, 3), (2, 3)], [1, 1, w13, 100], np.float32)
    d = oracle.dijkstra(rp, cl, w, 0)
    assert d.tolist() == [0, 1, 1, 101]
    pe = oracle.parent_edges(rp, cl, w, 0, d)
    assert pe.tolist() == [-1, 0, 1, 3]
    assert oracle.certificate(rp, cl, w, 0, d, pe) == (0, -1)
    bad = pe.copy()
    bad[3] = 2
    assert oracle.certificate(rp, cl, w, 0, d, bad) == (3, 3)


def test_zero_weight_tie_can_make_parent_cycle():
    # 1->2 (0), 2->1 (0), 5->1 (1), 5->2 (1), source 5: the lowest tight edge
    # into 1 comes from 2 and into 2 from 1.  The rule is a definition; the
    # certificate reports the cycle (code 5).
    rp, cl, w = gg.csr_from_edges(6, [(1, 2), (2, 1), (5, 1), (5, 2)], [0, 0, 1, 1])
    d = oracle.dijkstra(rp, cl, w, 5)
    pe = oracle.parent_edges(rp, cl, w, 5, d)
    assert pe[1] == 1 and pe[2] == 0
    assert oracle.certificate(rp, cl, w, 5, d, pe)[0] == 5


@pytest.mark.parametrize("kind", ["u32", "f32"])
def test_certificate_accepts_oracle_and_rejects_planted_mistakes(kind):
    if kind == "u32":
        rp, cl, w = gg.random_small(200, 1500, 21, kind="u32", wlo=1, whi=40)
    else:
        rp, cl, w = gg.random_small(200, 1500, 21, kind="f32", wlo=0.5, whi=2.0)
    d = oracle.dijkstra(rp, cl, w, 0)
    pe = oracle.parent_edges(rp, cl, w, 0, d)
    assert oracle.certificate(rp, cl, w, 0, d, pe) == (0, -1)
    reach = np.nonzero((pe >= 0))[0]
    v = int(reach[len(reach) // 2])
    # distance too large by one unit: the parent edge no longer matches
    bad = d.copy()
    bad[v] = bad[v] + (1 if kind == "u32" else np.float32(0.25))
    assert oracle.certificate(rp, cl, w, 0, bad, pe)[0] in (2, 3)
    # distance too small: its parent edge is not tight
    bad = d.copy()
    bad[v] = bad[v] - (1 if kind == "u32" else np.float32(0.25))
    assert oracle.certificate(rp, cl, w, 0, bad, pe)[0] in (2, 3)
    # parent edge pointing at a non-tight in-edge
    tails = oracle.edge_tails(rp)
    ins = [e for e in range(len(cl)) if cl[e] == v and e != pe[v]]
    if ins:
        badpe = pe.copy()
        badpe[v] = ins[0]
        tight = bool((d[tails[ins[0]]] + w[ins[0]]) == d[v])
        assert oracle.certificate(rp, cl, w, 0, d, badpe)[0] == (0 if tight else 3)
    # unreachable marked reachable / source distance changed
    bad = d.copy()
    bad[0] = 1 if kind == "u32" else np.float32(1)
    assert oracle.certificate(rp, cl, w, 0, bad, pe)[0] == 1
    # a planted transposition: distances of the reversed graph
    rp_t, cl_t, w_t = gg.csr_from_edges(200, np.stack([cl, tails], 1), w, w.dtype)
    d_t = oracle.dijkstra(rp_t, cl_t, w_t, 0)
    pe_t = oracle.parent_edges(rp, cl, w, 0, d_t)
    assert oracle.certificate(rp, cl, w, 0, d_t, pe_t)[0] != 0


@pytest.mark.parametrize("kind", ["u32", "f32"])
def test_certificate_rejects_a_consistent_tree_that_misses_a_shorter_edge(kind):
    # Solve on the graph without one tree edge e*: the result is a valid
    # tree with tight parent edges in the full graph too, but e* offers a
    # shorter path, which only the edge check (code 2) can see.
    if kind == "u32":
        rp, cl, w = gg.random_small(200, 1500, 21, kind="u32", wlo=1, whi=40)
    else:
        rp, cl, w = gg.random_small(200, 1500, 21, kind="f32", wlo=0.5, whi=2.0)
    d = oracle.dijkstra(rp, cl, w, 0)
    pe = oracle.parent_edges(rp, cl, w, 0, d)
    tails = oracle.edge_tails(rp)
    for e_star in sorted(int(e) for e in pe[pe >= 0]):
        keep = np.ones(len(cl), bool)
        keep[e_star] = False
        rp2, cl2, w2 = gg.csr_from_edges(200, np.stack([tails[keep], cl[keep]], 1), w[keep], w.dtype)
        d2 = oracle.dijkstra(rp2, cl2, w2, 0)
        if np.array_equal(d2, d):
            continue  # an equally short path remains
        pe2 = oracle.parent_edges(rp2, cl2, w2, 0, d2)
        full = np.nonzero(keep)[0]  # edge index in the reduced graph -> index in the full graph
        pe2_full = np.where(pe2 >= 0, full[np.maximum(pe2, 0)], -1).astype(np.int32)
        assert oracle.certificate(rp2, cl2, w2, 0, d2, pe2)[0] == 0
        code, where = oracle.certificate(rp, cl, w, 0, d2, pe2_full)
        assert code == 2
        assert (d2[tails[where]] + w[where]) < d2[cl[where]]
        return
    pytest.fail("no tree edge whose removal lengthens a path")


@pytest.mark.parametrize("kind", ["u32", "f32"])
def test_certificate_rejects_a_parent_edge_on_an_unreachable_vertex(kind):
    # 0->1; vertex 2 is reached only from the unreachable vertex 3 (edge 3->2)
    rp, cl, w = gg.csr_from_edges(4, [(0, 1), (3, 2)], [1, 1], np.uint32 if kind == "u32" else np.float32)
    d = oracle.dijkstra(rp, cl, w, 0)
    pe = oracle.parent_edges(rp, cl, w, 0, d)
    assert pe.tolist() == [-1, 0, -1, -1]
    assert oracle.certificate(rp, cl, w, 0, d, pe) == (0, -1)
    bad = pe.copy()
    bad[2] = 1
    assert oracle.certificate(rp, cl, w, 0, d, bad) == (4, 2)


def test_certificate_on_workload_sources():
    wl = gg.rmat_u32(14, 16, nsrc=3, seed=5)
    for s in wl.sources:
        d, p, pe = oracle.sssp(wl.row_ptr, wl.col, wl.weights, int(s))
        assert oracle.certificate(wl.row_ptr, wl.col, wl.weights, int(s), d, pe)[0] == 0
        assert p[s] == s and np.all((p == -1) == (d == INF32))


# ----------------------------------------------------------------- gradient

def test_gradient_closed_form_on_path():
    # dist[k] = w_0 + ... + w_{k-1}; L = sum c_k dist[k]
    # => dL/dw_i = sum_{k > i} c_k
    n = 6
    rp, cl, w = gg.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)], [1.5] * (n - 1), np.float32)
    c = np.array([0.3, -1.0, 2.0, 0.5, -0.25, 1.0])
    g = oracle.subtree_grad(rp, cl, w, 0, c)
    assert np.allclose(g, [c[i + 1:].sum() for i in range(n - 1)], rtol=0, atol=1e-12)


def test_gradient_closed_form_on_tree_and_off_tree_zero():
    # 0->1 (1), 0->2 (1), 1->3 (1), 1->4 (1), 2->4 (5) [off tree]
    rp, cl, w = gg.csr_from_edges(5, [(0, 1), (0, 2), (1, 3), (1, 4), (2, 4)], [1, 1, 1, 1, 5], np.float32)
    c = np.array([0.0, 1.0, 2.0, 4.0, 8.0])
    g = oracle.subtree_grad(rp, cl, w, 0, c)
    assert g.tolist() == [1 + 4 + 8, 2, 4, 8, 0]


def test_gradient_against_finite_differences():
    wl = gg.rmat_f32_diff(scale=10, edge_factor=8, ntargets=64, seed=1)
    n = wl.n
    c = np.zeros(n)
    c[wl.extra["targets"]] = wl.extra["coef"]
    g = oracle.subtree_grad(wl.row_ptr, wl.col, wl.weights, 0, c)
    on_tree = np.nonzero(g)[0][:40]
    fd, stable = oracle.fd_grad(wl.row_ptr, wl.col, wl.weights, 0, c, on_tree, h=1e-3)
    assert stable.sum() >= 30
    assert np.allclose(fd[stable], g[on_tree][stable], rtol=1e-6, atol=1e-9)
    off = np.nonzero(g == 0)[0][:20]
    fd0, stable0 = oracle.fd_grad(wl.row_ptr, wl.col, wl.weights, 0, c, off, h=1e-3)
    assert np.allclose(fd0[stable0], 0.0, atol=1e-9)


# -------------------------------------------------------------- generators

def test_generators_shapes():
    wl = gg.tiny_er()
    tails = oracle.edge_tails(wl.row_ptr)
    keys = tails.astype(np.int64) * wl.n + wl.col
    assert wl.n == 1024 and wl.m == 8192 and len(np.unique(keys)) == 8192 and np.all(tails != wl.col)
    assert wl.weights.min() >= 1 and wl.weights.max() <= 100
    rp, cl, sc = gg.grid(16, 0.01, 0)
    assert len(cl) == 4 * 16 * 15 + int(0.01 * 4 * 16 * 15)
    assert gg.tiny_er().weights.tobytes() == wl.weights.tobytes()  # deterministic


# ------------------------------------------------------------ signed weights

def potential_reweighted(n, m, seed, pmax=50):
    """Random graph with non-negative u32 weights w and potentials p; the
    reweighted int32 weights w + p[u] - p[v] are often negative but create no
    negative cycle (every cycle keeps its original, non-negative length)."""
    rp, cl, w = gg.random_small(n, m, seed, kind="u32", wlo=0, whi=30, self_loops=True)
    p = gg.below(seed, 21, n, 2 * pmax + 1) - pmax
    tails = oracle.edge_tails(rp)
    w2 = (w.astype(np.int64) + p[tails] - p[cl]).astype(np.int32)
    return rp, cl, w, w2, p


@pytest.mark.parametrize("seed", range(6))
def test_signed_weights_potential_closed_form(seed):
    # path lengths under w + p[u] - p[v] telescope: dist'(v) = dist(v) + p[s] - p[v];
    # the tight (parent) edges are the same set
    rp, cl, w, w2, p = potential_reweighted(150, 900, seed)
    assert (w2 < 0).any()
    s = 3
    d = oracle.dijkstra(rp, cl, w, s)
    fin = d != INF32
    expect = d.astype(np.int64)[fin] + p[s] - p[np.nonzero(fin)[0]]
    for algo in ("govm", "bellman_ford"):
        if algo == "govm":
            d2, st = oracle.govm(rp, cl, w2, s)
            assert st["converged"] == 1
        else:
            d2, neg = oracle.bellman_ford(rp, cl, w2, s)
            assert not neg
        assert np.array_equal(d2 == oracle.I32_INF, ~fin)
        assert np.array_equal(d2[fin].astype(np.int64), expect)
    pe = oracle.parent_edges(rp, cl, w, s, d)
    pe2 = oracle.parent_edges(rp, cl, w2, s, d2)
    assert np.array_equal(pe, pe2)
    assert oracle.certificate(rp, cl, w2, s, d2, pe2)[0] == 0


@pytest.mark.parametrize("seed", range(3))
def test_signed_weights_against_scipy_bellman_ford(seed):
    rp, cl, w, w2, p = potential_reweighted(200, 1200, seed + 10)
    n = len(rp) - 1
    tails = oracle.edge_tails(rp)
    best = {}
    for u, v, x in zip(tails, cl, w2.astype(np.float64)):
        if u == v:
            continue
        if (u, v) not in best or x < best[(u, v)]:
            best[(u, v)] = x
    uu, vv = zip(*best.keys())
    A = sp.csr_matrix((list(best.values()), (uu, vv)), shape=(n, n))
    ref = scipy_csgraph.bellman_ford(A, directed=True, indices=0)
    d2 = oracle.govm(rp, cl, w2, 0)[0]
    got = d2.astype(np.float64)
    got[d2 == oracle.I32_INF] = np.inf
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("seed", range(10))
def test_signed_weights_brute_force_small(seed):
    rp, cl, w, w2, p = potential_reweighted(7, 16, seed + 30, pmax=9)
    assert np.array_equal(oracle.govm(rp, cl, w2, 0)[0], oracle.brute_force(rp, cl, w2, 0))


def test_negative_cycle_reported():
    # 0 -> 1 -> 2 -> 1 with w(1,2) + w(2,1) = -1: reachable negative cycle
    rp, cl, w = gg.csr_from_edges(4, [(0, 1), (1, 2), (2, 1), (2, 3)], np.array([4, 2, -3, 1], np.int32), np.int32)
    d, st = oracle.govm(rp, cl, w, 0)
    assert st["converged"] == 0 and st["steps"] == 4  # the step cap n of Algorithm 2
    assert oracle.bellman_ford(rp, cl, w, 0)[1] is True
    # a negative cycle that is not reachable does not matter
    assert oracle.bellman_ford(rp, cl, w, 3)[1] is False
    d3, st3 = oracle.govm(rp, cl, w, 3)
    assert st3["converged"] == 1 and d3.tolist() == [int(oracle.I32_INF)] * 3 + [0]


def test_negative_cycle_through_the_source_is_excluded_by_the_guard():
    # 0->1 (1), 1->0 (-5), 1->2 (2): the cycle 0->1->0 has length -4 but only
    # re-enters the source, whose distance the source guard keeps
    # at 0 (Algorithm 2); so dist = [0, 1, 3] and the run converges.
    rp, cl, w = gg.csr_from_edges(3, [(0, 1), (1, 0), (1, 2)], np.array([1, -5, 2], np.int32), np.int32)
    d, st = oracle.govm(rp, cl, w, 0)
    assert d.tolist() == [0, 1, 3] and st["converged"] == 1 and st["updates"] == 2
    d_bf, neg = oracle.bellman_ford(rp, cl, w, 0)
    assert not neg and d_bf.tolist() == [0, 1, 3]


def test_bellman_ford_path_against_csr_order_needs_n_minus_1_rounds():
    # edges i+1 -> i, source n-1: a round visits tails in increasing order, so
    # each round extends the known path by one edge and the last vertex needs
    # all n - 1 rounds; dist[i] is the suffix sum of the weights.
    ws = np.array([3, -1, 4, 1, -5, 9, 2], np.int32)
    n = len(ws) + 1
    rp, cl, w = gg.csr_from_edges(n, [(i + 1, i) for i in range(n - 1)], ws, np.int32)
    expect = [int(ws[i:].sum()) for i in range(n - 1)] + [0]
    d_bf, neg = oracle.bellman_ford(rp, cl, w, n - 1)
    assert not neg and d_bf.tolist() == expect
    d, st = oracle.govm(rp, cl, w, n - 1)
    assert d.tolist() == expect and st["steps"] == n


def test_signed_certificate_rejects_planted_mistakes():
    # int32 weights with negative edges (potential reweighting, no negative
    # cycle): the certificate accepts the oracle's result and rejects a
    # non-tight parent edge (code 3) and a consistent tree that misses a
    # shorter edge (code 2)
    rp, cl, w, w2, p = potential_reweighted(120, 800, 3)
    d, neg = oracle.bellman_ford(rp, cl, w2, 0)
    assert not neg
    pe = oracle.parent_edges(rp, cl, w2, 0, d)
    assert oracle.certificate(rp, cl, w2, 0, d, pe) == (0, -1)
    tails = oracle.edge_tails(rp)
    fin = d != oracle.I32_INF
    # a reached vertex with an in-edge that is not tight
    cand = [e for e in range(len(cl)) if pe[cl[e]] >= 0 and e != pe[cl[e]] and fin[tails[e]]
            and int(d[tails[e]]) + int(w2[e]) != int(d[cl[e]])]
    assert cand
    bad = pe.copy()
    bad[cl[cand[0]]] = cand[0]
    assert oracle.certificate(rp, cl, w2, 0, d, bad) == (3, int(cl[cand[0]]))
    # drop a tree edge whose removal lengthens some path
    for e_star in sorted(int(e) for e in pe[pe >= 0]):
        keep = np.ones(len(cl), bool)
        keep[e_star] = False
        rp2, cl2, w22 = gg.csr_from_edges(len(rp) - 1, np.stack([tails[keep], cl[keep]], 1), w2[keep], np.int32)
        d2, neg2 = oracle.bellman_ford(rp2, cl2, w22, 0)
        if neg2 or np.array_equal(d2, d):
            continue
        pe2 = oracle.parent_edges(rp2, cl2, w22, 0, d2)
        full = np.nonzero(keep)[0]
        pe2_full = np.where(pe2 >= 0, full[np.maximum(pe2, 0)], -1).astype(np.int32)
        assert oracle.certificate(rp2, cl2, w22, 0, d2, pe2) == (0, -1)
        assert oracle.certificate(rp, cl, w2, 0, d2, pe2_full)[0] == 2
        return
    pytest.fail("no tree edge whose removal lengthens a path")


def test_signed_distance_outside_int32_is_reported():
    # path sums of -2^30 three times reach -3 * 2^30 < -2^31: the oracle works
    # in int64 and refuses to hand back a value that int32 cannot hold
    rp, cl, w = gg.csr_from_edges(4, [(0, 1), (1, 2), (2, 3)], np.full(3, -(1 << 30), np.int32), np.int32)
    with pytest.raises(OverflowError):
        oracle.bellman_ford(rp, cl, w, 0)
    with pytest.raises(OverflowError):
        oracle.govm(rp, cl, w, 0)
    # two steps still fit: -2^31 is the smallest int32
    rp, cl, w = gg.csr_from_edges(3, [(0, 1), (1, 2)], np.full(2, -(1 << 30), np.int32), np.int32)
    assert oracle.bellman_ford(rp, cl, w, 0)[0].tolist() == [0, -(1 << 30), -(1 << 31)]
