"""GPU parity of the two frontier forms of the persistent kernel.

Queue steps compact the frontier delta into a queue cut into 128-edge
tiles; direct steps expand the marked vertices straight from the bitmap of
the previous step's marks (one device-wide barrier per step).  Both run
Algorithm 2 (Section 3.4) to the same (min, fl(+)) fixpoint, so every case
is compared with the CPU oracle bit for bit (distances) and exactly
(lowest-index parents), in each form, including forms the automatic choice
would not pick (hub rows expanded directly by one warp, light graphs in
queue form), several grid sizes (narrow bitmap chunks on small grids),
batched and multi-root solves, signed weights and the failure paths.
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

FORMS = ("queue", "bitmap")


@pytest.fixture(scope="module")
def dawn():
    import paper_2306_07872_gb300 as pkg
    pkg.load_library()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return pkg


def graph(dawn, wl_or_csr, form, grid_blocks=0):
    rp, cl, w = wl_or_csr if isinstance(wl_or_csr, tuple) else (wl_or_csr.row_ptr, wl_or_csr.col, wl_or_csr.weights)
    g = dawn.Graph(rp, cl, w)
    g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)
    g.set_option(dawn.DAWN_OPT_FRONTIER, dawn.DAWN_FRONTIER_QUEUE if form == "queue" else dawn.DAWN_FRONTIER_BITMAP)
    if grid_blocks:
        g.set_option(dawn.DAWN_OPT_GRID_BLOCKS, grid_blocks)
    return g


def bits(a):
    a = np.asarray(a)
    return a.view(np.uint32)


def exact(rp, cl, w, roots, d, p, pe):
    d_ref, p_ref, pe_ref = oracle.sssp(rp, cl, w, roots)
    bad = np.nonzero(bits(d) != bits(d_ref))[0]
    assert len(bad) == 0, f"dist differs at {bad[:10]}"
    assert np.array_equal(pe, pe_ref), f"parent_edge differs at {np.nonzero(pe != pe_ref)[0][:10]}"
    assert np.array_equal(p, p_ref)


def solve(g, s):
    d, p, pe = g.sssp(int(s), parent=True, parent_edge=True)
    return d.cpu().numpy(), p.cpu().numpy(), pe.cpu().numpy()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("grid_blocks", [0, 1, 7, 300])
def test_rmat_with_hubs_both_forms(dawn, form, grid_blocks):
    wl = gg.rmat_u32(13, 16, nsrc=2, seed=41)
    assert np.diff(wl.row_ptr).max() > 128  # hub rows: the automatic choice would take the queue
    g = graph(dawn, wl, form, grid_blocks)
    for s in wl.sources:
        exact(wl.row_ptr, wl.col, wl.weights, int(s), *solve(g, s))
        st = g.stats()
        assert st["steps"] >= 1 and st["edges_scanned"] >= st["frontier_sum"] >= 1


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("side,grid_blocks", [(37, 0), (160, 0), (160, 1), (300, 5)])
def test_grid_f32_both_forms(dawn, form, side, grid_blocks):
    wl = gg.grid_f32(side, 0.01, nsrc=2, seed=side)
    g = graph(dawn, wl, form, grid_blocks)
    for s in wl.sources:
        exact(wl.row_ptr, wl.col, wl.weights, int(s), *solve(g, s))


def test_auto_form_matches_both(dawn):
    # the automatic choice on a light graph (direct) and on a hub graph (queue)
    for wl in (gg.grid_f32(120, 0.01, nsrc=1, seed=3), gg.rmat_u32(12, 16, nsrc=1, seed=4)):
        outs = []
        for form in ("auto",) + FORMS:
            g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
            g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)
            if form != "auto":
                g.set_option(dawn.DAWN_OPT_FRONTIER,
                             dawn.DAWN_FRONTIER_QUEUE if form == "queue" else dawn.DAWN_FRONTIER_BITMAP)
            outs.append(solve(g, wl.sources[0]))
        for o in outs[1:]:
            assert all(np.array_equal(bits(a), bits(b)) for a, b in zip(outs[0], o))


@pytest.mark.parametrize("form", FORMS)
def test_signed_weights_both_forms(dawn, form):
    # int32 weights with negative entries but no negative cycle: potentials
    # reweighting keeps every cycle non-negative
    rp, cl = gg.erdos_renyi(3000, 3000 * 6, seed=11)
    base = gg.weights_u32(len(cl), 1, 40, seed=12).astype(np.int64)
    pot = gg.below(13, 0, 3000, 60).astype(np.int64)
    tails = np.repeat(np.arange(3000), np.diff(rp))
    w = (base + pot[tails] - pot[cl]).astype(np.int32)
    assert (w < 0).any()
    g = graph(dawn, (rp, cl, w), form)
    for s in (0, 17, 2999):
        exact(rp, cl, w, s, *solve(g, s))


@pytest.mark.parametrize("form", FORMS)
def test_msssp_both_forms(dawn, form):
    # launches of several instances keep the queue form whatever the option says
    wl = gg.grid_f32(90, 0.02, nsrc=40, seed=5)
    g = graph(dawn, wl, form)
    dist, par = g.msssp(wl.sources)
    dist, par = dist.cpu().numpy(), par.cpu().numpy()
    for i in (0, 13, 39):
        d_ref, p_ref, _ = oracle.sssp(wl.row_ptr, wl.col, wl.weights, int(wl.sources[i]))
        assert np.array_equal(bits(dist[i]), bits(d_ref)) and np.array_equal(par[i], p_ref), i
    # several launches of one call (batch of 7)
    g.set_option(dawn.DAWN_OPT_BATCH, 7)
    d2, p2 = g.msssp(wl.sources)
    assert np.array_equal(bits(d2.cpu().numpy()), bits(dist)) and np.array_equal(p2.cpu().numpy(), par)


@pytest.mark.parametrize("form", FORMS)
def test_roots_forest_both_forms(dawn, form):
    wb = gg.er_batch(count=12, nlo=200, nhi=20000, dlo=2, dhi=20, seed=6)
    g = graph(dawn, wb, form)
    d, p, pe = g.sssp_roots(wb.sources, parent=True, parent_edge=True)
    exact(wb.row_ptr, wb.col, wb.weights, wb.sources, d.cpu().numpy(), p.cpu().numpy(), pe.cpu().numpy())


def test_direct_unit_weights_mu_one(dawn):
    # Section 4.2: with unit weights every reached vertex enters beta once
    rp, cl = gg.grid(150, 0.0, seed=1)[:2]
    w = np.ones(len(cl), np.float32)
    g = graph(dawn, (rp, cl, w), "bitmap")
    d, p, pe = solve(g, 0)
    exact(rp, cl, w, 0, d, p, pe)
    st = g.stats()
    assert st["updates"] == int(np.isfinite(d).sum()) - 1
    # one step per BFS level (the grid's hop diameter from a corner is 298),
    # plus the step that expands the last level
    assert st["steps"] == 299


def test_direct_trace_and_counters(dawn):
    wl = gg.grid_f32(100, 0.01, nsrc=1, seed=8)
    g = graph(dawn, wl, "bitmap")
    g.set_option(dawn.DAWN_OPT_TRACE_STEPS, 4096)
    d, p, pe = solve(g, wl.sources[0])
    exact(wl.row_ptr, wl.col, wl.weights, int(wl.sources[0]), d, p, pe)
    rows = dawn.dawn_get_trace(g.handle)
    st = g.stats()
    assert len(rows) == st["steps"]
    assert sum(r[1] for r in rows) == st["frontier_sum"] and sum(r[2] for r in rows) == st["edges_scanned"]


def test_direct_negative_cycle_hits_step_cap(dawn):
    # a negative cycle reachable from the source: Algorithm 2's step bound n
    # ends the solve with DAWN_ERR_NOT_CONVERGED
    rp, cl, w = gg.csr_from_edges(6, [(0, 1), (1, 2), (2, 3), (3, 1), (3, 4), (4, 5)], [2, 1, -3, 1, 1, 1],
                                  dtype=np.int32)
    g = graph(dawn, (rp, cl, w), "bitmap")
    g.sssp(0, check=False)
    assert dawn.dawn_status(g.handle, True) == dawn.DAWN_ERR_NOT_CONVERGED


def test_direct_timeout_and_gsvm(dawn):
    wl = gg.grid_f32(64, 0.01, nsrc=1, seed=9)
    g = graph(dawn, wl, "bitmap")
    g.set_option(dawn.DAWN_OPT_WAIT_LIMIT_NS, 50_000_000)
    g.set_option(dawn.DAWN_OPT_TEST_STALL, 1)
    g.sssp(int(wl.sources[0]), check=False)
    assert dawn.dawn_status(g.handle, True) == dawn.DAWN_ERR_TIMEOUT
    g.set_option(dawn.DAWN_OPT_TEST_STALL, 0)
    g.set_option(dawn.DAWN_OPT_WAIT_LIMIT_NS, 4_000_000_000)
    exact(wl.row_ptr, wl.col, wl.weights, int(wl.sources[0]), *solve(g, wl.sources[0]))
    # Algorithm 1 keeps the queue form whatever the option says
    g.set_option(dawn.DAWN_OPT_GSVM, 1)
    exact(wl.row_ptr, wl.col, wl.weights, int(wl.sources[0]), *solve(g, wl.sources[0]))


def test_frontier_option_rejects_bad_values(dawn):
    wl = gg.grid_f32(16, 0.0, nsrc=1, seed=1)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    for v in (-1, 3):
        with pytest.raises(dawn.DawnError) as e:
            g.set_option(dawn.DAWN_OPT_FRONTIER, v)
        assert e.value.code == dawn.DAWN_ERR_INVALID


@pytest.mark.parametrize("form", FORMS)
def test_skip_remarked_same_results(dawn, form):
    # in bitmap steps a frontier vertex marked again earlier in its own step
    # is expanded in the next step only: the fixpoint (distances,
    # lowest-index parents) is the same with and without the skip; queue
    # steps never skip
    for wl in (gg.rmat_u32(14, 16, nsrc=2, seed=51), gg.grid_f32(200, 0.01, nsrc=2, seed=52)):
        g = graph(dawn, wl, form)
        for s in wl.sources:
            stats = {}
            for skip in (0, 1):
                g.set_option(dawn.DAWN_OPT_SKIP_REMARKED, skip)
                exact(wl.row_ptr, wl.col, wl.weights, int(s), *solve(g, s))
                stats[skip] = g.stats()
            assert stats[0]["edges_skipped"] == 0
            assert 0 <= stats[1]["edges_skipped"] <= stats[1]["edges_scanned"]
            if form == "queue":
                assert stats[1]["edges_skipped"] == 0
    # signed weights and Algorithm 1 (which never skips)
    rp, cl, w = gg.random_small(2000, 16000, 53, kind="u32", wlo=1, whi=30)
    g = graph(dawn, (rp, cl, w), form)
    g.set_option(dawn.DAWN_OPT_GSVM, 1)
    exact(rp, cl, w, 0, *solve(g, 0))
    assert g.stats()["edges_skipped"] == 0


def test_skip_remarked_counts_on_a_random_graph(dawn):
    # on a random graph with a wide weight range some frontier vertices are
    # lowered again before their expansion within a step: the skip finds them
    rp, cl = gg.erdos_renyi(1 << 16, 16 << 16, seed=54)
    w = gg.weights_u32(len(cl), 1, 255, seed=55)
    g = graph(dawn, (rp, cl, w), "bitmap")
    total = 0
    for s in (0, 1000, 40000):
        exact(rp, cl, w, s, *solve(g, s))
        total += g.stats()["edges_skipped"]
    assert total > 0
