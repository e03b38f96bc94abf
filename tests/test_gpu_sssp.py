"""GPU parity of the GOVM solver (libdawn, sm_103a) against the CPU oracle.

Distances must be bit-exact (uint32 and float32: the (min, fl(+)) fixpoint is
order independent for non-negative weights), parents must follow the
lowest-edge-index rule exactly, and at full workload sizes every source's
output must pass the oracle's optimality certificate.
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

INF32 = np.uint32(0xFFFFFFFF)


@pytest.fixture(scope="module")
def dawn():
    import paper_2306_07872_gb300 as pkg
    pkg.load_library()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return pkg


# parity tests run on both kernels: the small-graph one (graphs that fit
# on-chip; others fall back to the persistent kernel) and the persistent one
@pytest.fixture(params=["auto", "persistent"])
def Graph(dawn, request):
    def make(*args):
        g = dawn.Graph(*args)
        if request.param == "persistent":
            g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)
        return g
    return make


def bits(a):
    a = np.asarray(a)
    return a.view(np.uint32) if a.dtype in (np.float32, np.uint32, np.int32) else a


def solve(g, s):
    d, p, pe = g.sssp(s, parent=True, parent_edge=True)
    return d.cpu().numpy(), p.cpu().numpy(), pe.cpu().numpy()


def assert_exact(rp, cl, w, s, d, p, pe):
    d_ref, p_ref, pe_ref = oracle.sssp(rp, cl, w, s)
    bad = np.nonzero(bits(d) != bits(d_ref))[0]
    assert len(bad) == 0, f"dist differs at {bad[:10]}: gpu {d[bad[:5]]} oracle {d_ref[bad[:5]]}"
    assert np.array_equal(pe, pe_ref), f"parent_edge differs at {np.nonzero(pe != pe_ref)[0][:10]}"
    assert np.array_equal(p, p_ref)


# ------------------------------------------------------------ tiny workload

def test_tiny_er_source0_exact_and_fw(dawn, Graph):
    wl = gg.tiny_er()
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    d, p, pe = solve(g, 0)
    assert_exact(wl.row_ptr, wl.col, wl.weights, 0, d, p, pe)
    D = oracle.floyd_warshall(wl.row_ptr, wl.col, wl.weights)
    assert np.array_equal(d, D[0])


def test_tiny_er_many_sources(dawn, Graph):
    wl = gg.tiny_er()
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    D = oracle.floyd_warshall(wl.row_ptr, wl.col, wl.weights)
    for s in range(0, 1024, 37):
        d, p, pe = solve(g, s)
        assert np.array_equal(d, D[s]), s
        assert_exact(wl.row_ptr, wl.col, wl.weights, s, d, p, pe)


# ------------------------------------------------- several tiles, ragged tails

@pytest.mark.parametrize("scale,ef,seed", [(10, 4, 1), (12, 8, 2), (14, 16, 3)])
def test_rmat_u32_exact(dawn, Graph, scale, ef, seed):
    wl = gg.rmat_u32(scale, ef, nsrc=4, seed=seed)
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    for s in wl.sources:
        d, p, pe = solve(g, int(s))
        assert_exact(wl.row_ptr, wl.col, wl.weights, int(s), d, p, pe)


@pytest.mark.parametrize("side,seed", [(32, 0), (100, 1), (257, 2)])
def test_grid_f32_exact(dawn, Graph, side, seed):
    wl = gg.grid_f32(side, 0.01, nsrc=3, seed=seed)
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    for s in wl.sources:
        d, p, pe = solve(g, int(s))
        assert_exact(wl.row_ptr, wl.col, wl.weights, int(s), d, p, pe)


def test_rmat_f32_exact(dawn, Graph):
    wl = gg.rmat_f32_diff(scale=13, edge_factor=16, ntargets=8, seed=2)
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    d, p, pe = solve(g, 0)
    assert_exact(wl.row_ptr, wl.col, wl.weights, 0, d, p, pe)


def test_rmat_f32_weights_down_to_zero_exact(dawn, Graph):
    # the paper's comparative weights (Section 4.2): fp32 uniform in [0, 2];
    # tiny weights make fl(d + w) == d ties, which the parent rule resolves
    rp, cl = gg.rmat(12, 16, seed=4)
    w = gg.weights_f32_uniform(len(cl), 0.0, 2.0, seed=8)
    w[::97] = np.float32(0.0)
    g = Graph(rp, cl, w)
    src, _, _ = gg.wcc_sources(rp, cl, 3, seed=2)
    for s in src:
        d, p, pe = solve(g, int(s))
        assert_exact(rp, cl, w, int(s), d, p, pe)


@pytest.mark.parametrize("kind", ["rmat_u32", "grid_f32"])
def test_gsvm_option_same_result_more_work(dawn, kind):
    # Algorithm 1 (GSVM) rescans every reached vertex each step; GOVM
    # (Algorithm 2) only the vertices that changed: same fixpoint, less work
    wl = gg.rmat_u32(12, 16, nsrc=2, seed=5) if kind == "rmat_u32" else gg.grid_f32(64, 0.01, nsrc=2, seed=5)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    for s in wl.sources:
        govm = solve(g, int(s))
        st_govm = g.stats()
        g.set_option(dawn.DAWN_OPT_GSVM, 1)
        gsvm = solve(g, int(s))
        st_gsvm = g.stats()
        g.set_option(dawn.DAWN_OPT_GSVM, 0)
        for a, b in zip(govm, gsvm):
            assert np.array_equal(a, b)
        assert_exact(wl.row_ptr, wl.col, wl.weights, int(s), *gsvm)
        assert st_gsvm["edges_scanned"] > st_govm["edges_scanned"]
        _, ost = oracle.gsvm(wl.row_ptr, wl.col, wl.weights, int(s))
        assert st_gsvm["steps"] >= 2 and ost["converged"] == 1


def test_unit_weights_bfs_and_mu_one(dawn, Graph):
    # Section 4.2: unit weights find every path once (mu = 1)
    wl = gg.rmat_u32(13, 8, nsrc=2, seed=7, wlo=1, whi=1)
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    for s in wl.sources:
        d, p, pe = solve(g, int(s))
        assert_exact(wl.row_ptr, wl.col, wl.weights, int(s), d, p, pe)
        st = g.stats()
        reached = int((d != INF32).sum())
        assert st["updates"] == reached - 1


def test_hub_rows_span_many_tiles(dawn, Graph):
    # a star with 5000 leaves (20 tiles in one row) feeding a path, plus
    # leaves with parallel edges and self-loops
    n = 6000
    edges, ws = [], []
    for v in range(1, 5001):
        edges.append((0, v)); ws.append(1 + (v * 7919) % 97)
    for v in range(5000, 5999):
        edges.append((v, v + 1)); ws.append(3)
    for v in range(1, 200):
        edges.append((v, 5000)); ws.append(1)
        edges.append((v, v)); ws.append(0)
        edges.append((v, 5000)); ws.append(2)
    rp, cl, w = gg.csr_from_edges(n, edges, ws)
    g = Graph(rp, cl, w)
    d, p, pe = solve(g, 0)
    assert_exact(rp, cl, w, 0, d, p, pe)


def test_hub_lowered_in_every_step(dawn, Graph):
    # A hub of 6000 out-edges (47 tiles) is reached first by a heavy edge and
    # then, one step later each time, by paths with more hops and less
    # weight, so it is lowered in every step while its own tiles are being
    # expanded: tiles of one step may read different keys.  A vertex is left
    # out of the next frontier only when every tile used its current key.
    L, fan = 30, 6000
    n = 2 + L + fan + 1
    hub, sink = 1, n - 1
    edges, ws = [], []
    chain = list(range(2, 2 + L))
    prev = 0
    for i, a in enumerate(chain):
        edges.append((prev, a)); ws.append(1)
        edges.append((a, hub)); ws.append(5000 - 150 * i)
        prev = a
    edges.append((0, hub)); ws.append(6000)
    leaves = range(2 + L, 2 + L + fan)
    for j, v in enumerate(leaves):
        edges.append((hub, v)); ws.append(1 + (j * 7919) % 251)
        if j % 3 == 0:
            edges.append((v, sink)); ws.append(1 + j % 13)
        if j % 5 == 0 and j + 1 < fan:
            edges.append((v, v + 1)); ws.append(2)
    rp, cl, w = gg.csr_from_edges(n, edges, ws)
    g = Graph(rp, cl, w)
    for s in (0, 2, 2 + L // 2):
        assert_exact(rp, cl, w, s, *solve(g, s))
    wf = w.astype(np.float32) * np.float32(0.37)
    g = Graph(rp, cl, wf)
    assert_exact(rp, cl, wf, 0, *solve(g, 0))


def test_many_degree_one_frontier(dawn, Graph):
    # binary tree (frontier of many out-degree-1/2 vertices: up to 257 entries per tile)
    n = 1 << 15
    edges = [(v, c) for v in range(n) for c in (2 * v + 1, 2 * v + 2) if c < n]
    ws = [(a * 31 + b * 17) % 50 + 1 for a, b in edges]
    rp, cl, w = gg.csr_from_edges(n, edges, ws)
    g = Graph(rp, cl, w)
    d, p, pe = solve(g, 0)
    assert_exact(rp, cl, w, 0, d, p, pe)


# ----------------------------------------------------------------- edge cases

def test_edge_cases(dawn, Graph):
    # n = 1, m = 0
    g = Graph(np.array([0, 0], np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    d, p, pe = solve(g, 0)
    assert d.tolist() == [0] and p.tolist() == [0] and pe.tolist() == [-1]
    # source with out-degree 0, unreachable parts, zero weight into the source
    rp, cl, w = gg.csr_from_edges(5, [(0, 1), (1, 0), (1, 2), (4, 3)], [0, 0, 5, 1])
    g = Graph(rp, cl, w)
    for s in range(5):
        assert_exact(rp, cl, w, s, *solve(g, s))
    # fp32 left-fold rounding: 2^24 + 1 + 1 beats 2^24 + 2
    t24 = np.float32(2.0 ** 24)
    rp, cl, w = gg.csr_from_edges(4, [(0, 1), (1, 2), (2, 3), (0, 3)], [t24, 1, 1, t24 + np.float32(2)], np.float32)
    g = Graph(rp, cl, w)
    d, p, pe = solve(g, 0)
    assert d[3] == t24 and p[3] == 2
    assert_exact(rp, cl, w, 0, d, p, pe)
    # large uint32 weights: n * max(w) just below the sentinel
    big = (0xFFFFFFFE // 4)
    rp, cl, w = gg.csr_from_edges(4, [(0, 1), (1, 2), (2, 3)], [big, big, big])
    g = Graph(rp, cl, w)
    assert_exact(rp, cl, w, 0, *solve(g, 0))
    # zero-weight ties (the parent rule may form a cycle; both sides agree)
    rp, cl, w = gg.csr_from_edges(6, [(1, 2), (2, 1), (5, 1), (5, 2)], [0, 0, 1, 1])
    g = Graph(rp, cl, w)
    assert_exact(rp, cl, w, 5, *solve(g, 5))


@pytest.mark.parametrize("seed", range(12))
def test_random_small_multigraphs(dawn, Graph, seed):
    kind = ["u32", "f32", "dyadic"][seed % 3]
    rp, cl, w = gg.random_small(60 + seed * 13, 400 + seed * 50, seed, kind=kind, wlo=0 if kind != "f32" else 0.0,
                                whi=9, self_loops=True)
    g = Graph(rp, cl, w)
    for s in (0, 3, 17):
        assert_exact(rp, cl, w, s, *solve(g, s))


# --------------------------------------------------------- errors and status

def test_invalid_inputs_rejected(dawn):
    rp = np.array([0, 2, 1, 3], np.int32)  # non-monotone
    with pytest.raises(dawn.DawnError) as e:
        dawn.Graph(rp, np.array([1, 2, 0], np.int32), np.ones(3, np.uint32))
    assert e.value.code == dawn.DAWN_ERR_INVALID
    rp = np.array([0, 1, 2], np.int32)
    with pytest.raises(dawn.DawnError):
        dawn.Graph(rp, np.array([1, 5], np.int32), np.ones(2, np.uint32))  # column out of range
    with pytest.raises(dawn.DawnError):
        dawn.Graph(rp, np.array([1, 0], np.int32), np.array([1.0, np.nan], np.float32))
    with pytest.raises(dawn.DawnError):
        dawn.Graph(rp, np.array([1, 0], np.int32), np.array([1.0, -1.0], np.float32))
    with pytest.raises(dawn.DawnError):
        dawn.Graph(rp, np.array([1, 0], np.int32), np.array([1.0, np.inf], np.float32))
    with pytest.raises(dawn.DawnError):  # 2 * 0x80000000 reaches the sentinel
        dawn.Graph(rp, np.array([1, 0], np.int32), np.array([1, 0x80000000], np.uint32))
    g = dawn.Graph(rp, np.array([1, 0], np.int32), np.ones(2, np.uint32))
    with pytest.raises(dawn.DawnError):
        g.sssp(2)
    with pytest.raises(dawn.DawnError) as e:
        g.msssp([0, 7])
    assert e.value.code == dawn.DAWN_ERR_INVALID
    d, p, _ = g.sssp(1)  # the handle stays usable
    assert d.cpu().tolist() == [1, 0]


def test_step_cap_reports_not_converged(dawn, Graph):
    rp, cl, w = gg.csr_from_edges(5, [(i, i + 1) for i in range(4)], [1, 1, 1, 1])
    g = Graph(rp, cl, w)
    g.set_option(dawn.DAWN_OPT_MAX_STEPS, 2)
    with pytest.raises(dawn.DawnError) as e:
        g.sssp(0)
    assert e.value.code == dawn.DAWN_ERR_NOT_CONVERGED
    g.set_option(dawn.DAWN_OPT_MAX_STEPS, 0)
    assert g.sssp(0)[0].cpu().tolist() == [0, 1, 2, 3, 4]


def test_bounded_wait_reports_timeout_and_context_survives(dawn):
    # block 0 waits on a flag that nothing sets; every wait is bounded, so the
    # kernel returns DAWN_ERR_TIMEOUT and the context stays usable
    wl = gg.rmat_u32(12, 8, nsrc=1, seed=1)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    g.set_option(dawn.DAWN_OPT_GRID_BLOCKS, 4)
    g.set_option(dawn.DAWN_OPT_WAIT_LIMIT_NS, 20_000_000)
    g.set_option(dawn.DAWN_OPT_TEST_STALL, 1)
    with pytest.raises(dawn.DawnError) as e:
        g.sssp(int(wl.sources[0]))
    assert e.value.code == dawn.DAWN_ERR_TIMEOUT
    g.set_option(dawn.DAWN_OPT_TEST_STALL, 0)
    g.set_option(dawn.DAWN_OPT_WAIT_LIMIT_NS, 4_000_000_000)
    d, p, pe = solve(g, int(wl.sources[0]))
    assert_exact(wl.row_ptr, wl.col, wl.weights, int(wl.sources[0]), d, p, pe)


def test_grid_sizes_agree(dawn):
    wl = gg.rmat_u32(13, 16, nsrc=1, seed=4)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    s = int(wl.sources[0])
    ref = solve(g, s)
    for blocks in (1, 3, 152, 0):
        g.set_option(dawn.DAWN_OPT_GRID_BLOCKS, blocks)
        got = solve(g, s)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), blocks


def test_host_and_device_inputs_agree(dawn, Graph):
    wl = gg.rmat_u32(11, 8, nsrc=1, seed=9)
    g1 = Graph(wl.row_ptr, wl.col, wl.weights)
    g2 = Graph(torch.from_numpy(wl.row_ptr).cuda(), torch.from_numpy(wl.col).cuda(),
                    torch.from_numpy(wl.weights).cuda())
    s = int(wl.sources[0])
    for a, b in zip(solve(g1, s), solve(g2, s)):
        assert np.array_equal(a, b)


def test_allocation_failure_reports_oom_and_handle_recovers(dawn):
    # host-side injection (no device is driven out of memory): the N-th next
    # workspace allocation fails; the call reports DAWN_ERR_OOM, frees what it
    # had, and the handle stays usable
    wl = gg.rmat_u32(11, 8, nsrc=1, seed=12)
    s = int(wl.sources[0])
    for nth in (1, 3, 5):
        g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
        g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)  # the kernel with a device workspace
        g.set_option(dawn.DAWN_OPT_TEST_FAIL_ALLOC, nth)
        with pytest.raises(dawn.DawnError) as e:
            g.sssp(s)
        assert e.value.code == dawn.DAWN_ERR_OOM
        d, p, pe = solve(g, s)
        assert_exact(wl.row_ptr, wl.col, wl.weights, s, d, p, pe)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)
    g.set_option(dawn.DAWN_OPT_TEST_FAIL_ALLOC, 1)
    with pytest.raises(dawn.DawnError) as e:
        dawn.dawn_reserve(g.handle, 8)
    assert e.value.code == dawn.DAWN_ERR_OOM
    dist, _ = g.msssp(wl.sources)
    assert np.array_equal(dist[0].cpu().numpy(), oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, s))
    with pytest.raises(dawn.DawnError):
        g.set_option(dawn.DAWN_OPT_TEST_FAIL_ALLOC, -1)
