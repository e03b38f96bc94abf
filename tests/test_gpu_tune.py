"""GPU tests of the launch options and the autotuner.

The 4-CTA-per-SM kernel build is separate machine code from the default
5-CTA build, so it gets its own parity cases against the oracle for every
weight type; batch sizes and grid sizes must not change any result; and the
autotuner must return a valid configuration, reject bad input, and leave
every later result bit-exact.
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dawn():
    import paper_2306_07872_gb300 as pkg
    pkg.load_library()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return pkg


def bits(a):
    a = np.asarray(a)
    return a.view(np.uint32) if a.dtype in (np.float32, np.uint32, np.int32) else a


def exact(g, rp, cl, w, s):
    d, p, pe = g.sssp(int(s), parent=True, parent_edge=True)
    d_ref, p_ref, pe_ref = oracle.sssp(rp, cl, w, int(s))
    assert np.array_equal(bits(d.cpu().numpy()), bits(d_ref))
    assert np.array_equal(p.cpu().numpy(), p_ref)
    assert np.array_equal(pe.cpu().numpy(), pe_ref)


def workloads():
    rmat = gg.rmat_u32(13, 16, nsrc=2, seed=21)
    grid = gg.grid_f32(120, 0.01, nsrc=2, seed=22)
    rp, cl, w = gg.random_small(3000, 24000, 23, kind="u32", wlo=1, whi=50)
    # potential reweighting w + pot(u) - pot(v): some edges turn negative, no cycle does
    pot = (np.arange(3000, dtype=np.int64) * 7919) % 13
    tails = np.repeat(np.arange(3000), np.diff(rp))
    signed = (w.astype(np.int64) + pot[tails] - pot[cl]).astype(np.int32)
    return [("rmat_u32", rmat.row_ptr, rmat.col, rmat.weights, rmat.sources),
            ("grid_f32", grid.row_ptr, grid.col, grid.weights, grid.sources),
            ("signed_i32", rp, cl, signed, np.array([0, 17], np.int32))]


@pytest.mark.parametrize("idx", [0, 1, 2])
@pytest.mark.parametrize("ctas", [4, 5])
def test_kernel_builds_exact(dawn, idx, ctas):
    name, rp, cl, w, srcs = workloads()[idx]
    g = dawn.Graph(rp, cl, w)
    g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)  # the persistent kernel's builds
    g.set_option(dawn.DAWN_OPT_CTAS_PER_SM, ctas)
    for blocks in (0, 1, 5, 152):
        g.set_option(dawn.DAWN_OPT_GRID_BLOCKS, blocks)
        for s in srcs:
            exact(g, rp, cl, w, s)


def test_ctas_option_validated(dawn):
    wl = gg.tiny_er()
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    for bad in (1, 3, 6, -1):
        with pytest.raises(dawn.DawnError):
            g.set_option(dawn.DAWN_OPT_CTAS_PER_SM, bad)
    with pytest.raises(dawn.DawnError):
        g.set_option(dawn.DAWN_OPT_BATCH, -2)


@pytest.mark.parametrize("batch", [0, 1, 7, 64])
def test_batch_sizes_agree(dawn, batch):
    wl = gg.rmat_u32(11, 8, nsrc=40, seed=24)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)  # batches of the persistent kernel
    g.set_option(dawn.DAWN_OPT_BATCH, batch)
    g.set_option(dawn.DAWN_OPT_CTAS_PER_SM, 4 if batch % 2 else 5)
    dist, par = g.msssp(wl.sources)
    dist, par = dist.cpu().numpy(), par.cpu().numpy()
    for i in (0, 13, 39):
        d_ref, p_ref, _ = oracle.sssp(wl.row_ptr, wl.col, wl.weights, int(wl.sources[i]))
        assert np.array_equal(dist[i], d_ref) and np.array_equal(par[i], p_ref)


def test_autotune_sssp_keeps_results_exact(dawn):
    wl = gg.rmat_u32(14, 16, nsrc=4, seed=25)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    t = g.autotune(wl.sources, mode="sssp", reps=2)
    assert t["ctas_per_sm"] in (4, 5)
    assert t["grid_blocks"] >= 0 and t["batch"] == 0
    assert t["candidates"] >= 10  # the launch shapes plus the other step form at each build
    assert 0 < t["best_ms"] <= t["default_ms"]
    assert t["frontier"] in (dawn.DAWN_FRONTIER_AUTO, dawn.DAWN_FRONTIER_QUEUE, dawn.DAWN_FRONTIER_BITMAP)
    for s in wl.sources:
        exact(g, wl.row_ptr, wl.col, wl.weights, s)


def test_autotune_frontier_form_applies(dawn):
    # whichever step form the tuner keeps is what later solves run, and it
    # gives the oracle's fixpoint; on a light graph the tuner may keep queue
    # steps only if they timed faster than the automatic bitmap steps
    wl = gg.grid_f32(300, 0.01, nsrc=4, seed=31)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)
    t = g.autotune(wl.sources, mode="sssp", reps=1)
    assert t["frontier"] in (dawn.DAWN_FRONTIER_AUTO, dawn.DAWN_FRONTIER_QUEUE)
    for s in wl.sources:
        exact(g, wl.row_ptr, wl.col, wl.weights, s)
    # the msssp mode never times a step form (batched launches use queue steps)
    t2 = g.autotune(wl.sources, mode="msssp", reps=1)
    assert t2["frontier"] == dawn.DAWN_FRONTIER_AUTO


def test_autotune_msssp_and_roots(dawn):
    wl = gg.rmat_u32(11, 16, nsrc=96, seed=26)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    t = g.autotune(wl.sources, mode="msssp", reps=1)
    assert t["ctas_per_sm"] in (4, 5) and t["batch"] >= 0 and t["candidates"] >= 2
    dist, _ = g.msssp(wl.sources, parent=False)
    dist = dist.cpu().numpy()
    for i in (0, 50, 95):
        assert np.array_equal(dist[i], oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, int(wl.sources[i])))

    ub = gg.er_batch(count=6, nlo=200, nhi=4000, dlo=4, dhi=12, seed=27)
    h = dawn.Graph(ub.row_ptr, ub.col, ub.weights)
    t = h.autotune(ub.sources, mode="roots", reps=1)
    assert t["batch"] == 0
    d, _, _ = h.sssp_roots(ub.sources)
    assert np.array_equal(d.cpu().numpy(), oracle.dijkstra(ub.row_ptr, ub.col, ub.weights, ub.sources))


def test_autotune_rejects_bad_input(dawn):
    wl = gg.rmat_u32(10, 8, nsrc=2, seed=28)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    g.set_option(dawn.DAWN_OPT_GRID_BLOCKS, 3)
    g.set_option(dawn.DAWN_OPT_CTAS_PER_SM, 4)
    for mode, src in ((0, [0, wl.n]), (0, [-1]), (7, [0]), (0, [])):
        with pytest.raises(dawn.DawnError) as e:
            dawn.dawn_autotune(g.handle, mode, np.array(src, np.int32))
        assert e.value.code == dawn.DAWN_ERR_INVALID
    exact(g, wl.row_ptr, wl.col, wl.weights, wl.sources[0])


def test_batched_counters_cover_every_launch(dawn):
    # a call split into several launches reports counters summed over all of them
    wl = gg.rmat_u32(12, 8, nsrc=40, seed=29)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    per = {}
    for batch in (0, 5):
        g.set_option(dawn.DAWN_OPT_BATCH, batch)
        g.msssp(wl.sources, parent=False)
        st = g.stats()
        assert st["instances"] == 40 and st["steps"] >= 1
        per[batch] = st
    for key in ("edges_scanned", "updates", "frontier_sum"):
        ratio = per[5][key] / per[0][key]
        assert 0.8 < ratio < 1.25, (key, per)


def test_autotune_cache_reuses_a_stored_configuration(dawn, tmp_path):
    wl = gg.rmat_u32(12, 16, nsrc=4, seed=30)
    path = str(tmp_path / "tune.json")
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    first = g.autotune(wl.sources, mode="sssp", reps=1, cache=path)
    assert first["cached"] is False
    h = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    again = h.autotune(wl.sources, mode="sssp", reps=1, cache=path)
    assert again["cached"] is True
    for f in ("ctas_per_sm", "grid_blocks", "batch", "frontier"):
        assert again[f] == first[f]
    for s in wl.sources:
        exact(h, wl.row_ptr, wl.col, wl.weights, s)
