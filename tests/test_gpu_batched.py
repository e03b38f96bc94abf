"""GPU parity of the batched forms: multi-source (per-instance frontiers in
one persistent launch, chunked for large k) and multi-root solves on a
disjoint union of uneven graphs; CUDA-graph capture of a batched solve."""
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
    return pkg


# every test runs on both kernels: the small-graph one (where the graph fits
# on-chip) and the persistent one
@pytest.fixture(params=["auto", "persistent"])
def Graph(dawn, request):
    def make(*args):
        g = dawn.Graph(*args)
        if request.param == "persistent":
            g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)
        return g
    return make


def exact_rows(wl, sources, dist, parent):
    for i, s in enumerate(sources):
        d_ref, p_ref, _ = oracle.sssp(wl.row_ptr, wl.col, wl.weights, int(s))
        assert np.array_equal(dist[i].view(np.uint32), d_ref.view(np.uint32)), i
        if parent is not None:
            assert np.array_equal(parent[i], p_ref), i


def test_msssp_matches_single_solves(dawn, Graph):
    wl = gg.rmat_u32(12, 16, nsrc=64, seed=3)
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    dist, par = g.msssp(wl.sources)
    dist, par = dist.cpu().numpy(), par.cpu().numpy()
    exact_rows(wl, wl.sources, dist, par)
    for i in (0, 17, 63):
        d1, p1, _ = g.sssp(int(wl.sources[i]))
        assert np.array_equal(d1.cpu().numpy(), dist[i]) and np.array_equal(p1.cpu().numpy(), par[i])


def test_msssp_f32_and_duplicate_sources(dawn, Graph):
    wl = gg.grid_f32(48, 0.01, nsrc=5, seed=2)
    src = np.concatenate([wl.sources, wl.sources[:2]])
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    dist, par = g.msssp(src)
    exact_rows(wl, src, dist.cpu().numpy(), par.cpu().numpy())


def test_msssp_chunks_beyond_one_launch(dawn, Graph):
    # k larger than the per-launch instance limit: several persistent launches
    wl = gg.tiny_er(n=300, avg_deg=6, seed=5)
    src = np.arange(1500, dtype=np.int32) % 300
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    dist, _ = g.msssp(src, parent=False)
    D = oracle.floyd_warshall(wl.row_ptr, wl.col, wl.weights)
    assert np.array_equal(dist.cpu().numpy(), D[src])


def test_apsp_small(dawn, Graph):
    # APSP = msssp over every vertex (Section 3.4); compare with Floyd-Warshall
    rp, cl, w = gg.random_small(200, 1600, 7, kind="dyadic", wlo=0, whi=6)
    g = Graph(rp, cl, w)
    dist, _ = g.msssp(np.arange(200, dtype=np.int32), parent=False)
    D = oracle.floyd_warshall(rp, cl, w)
    assert np.array_equal(dist.cpu().numpy().view(np.uint32), D.view(np.uint32))


def test_apsp_medium_sampled_rows(dawn, Graph):
    # all 4096 sources of an ER graph in chunked batched launches; sampled
    # rows bit-exact to Dijkstra, every sampled row certified
    wl = gg.tiny_er(n=4096, avg_deg=8, seed=11)
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    dist, par = g.msssp(np.arange(wl.n, dtype=np.int32))
    dist = dist.cpu().numpy()
    par = par.cpu().numpy()
    for s in range(0, wl.n, 257):
        d_ref = oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, s)
        assert np.array_equal(dist[s], d_ref), s
        pe = oracle.parent_edges(wl.row_ptr, wl.col, wl.weights, s, d_ref)
        assert np.array_equal(par[s], oracle.parent_vertices(wl.row_ptr, s, d_ref, pe, "u32")), s


def test_roots_on_uneven_batch(dawn, Graph):
    wl = gg.er_batch(count=12, nlo=100, nhi=20000, dlo=4, dhi=32, seed=6)
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    d, p, pe = g.sssp_roots(wl.sources, parent=True, parent_edge=True)
    d_ref = oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, wl.sources)
    pe_ref = oracle.parent_edges(wl.row_ptr, wl.col, wl.weights, wl.sources, d_ref)
    p_ref = oracle.parent_vertices(wl.row_ptr, wl.sources, d_ref, pe_ref, "u32")
    assert np.array_equal(d.cpu().numpy(), d_ref)
    assert np.array_equal(pe.cpu().numpy(), pe_ref) and np.array_equal(p.cpu().numpy(), p_ref)
    # per-graph solves give the same rows
    offs = wl.extra["offsets"]
    for i in (0, 5, 11):
        d1, _, _ = g.sssp(int(wl.sources[i]))
        sl = slice(int(offs[i]), int(offs[i + 1]))
        assert np.array_equal(d1.cpu().numpy()[sl], d_ref[sl])


def test_roots_duplicates_and_invalid(dawn, Graph):
    wl = gg.rmat_u32(10, 8, nsrc=4, seed=1)
    roots = np.array([wl.sources[0], wl.sources[1], wl.sources[0]], np.int32)
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    d, p, _ = g.sssp_roots(roots)
    d_ref = oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, roots)
    assert np.array_equal(d.cpu().numpy(), d_ref)
    with pytest.raises(dawn.DawnError):
        g.sssp_roots(np.array([0, wl.n], np.int32))


def test_msssp_captured_in_cuda_graph(dawn, Graph):
    wl = gg.rmat_u32(11, 8, nsrc=16, seed=8)
    g = Graph(wl.row_ptr, wl.col, wl.weights)
    dawn.dawn_reserve(g.handle, 16)
    src = torch.from_numpy(wl.sources).cuda()
    dist = torch.empty((16, wl.n), dtype=torch.uint32, device="cuda")
    par = torch.empty((16, wl.n), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        dawn.dawn_msssp(g.handle, src, dist, par, stream=s)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        dawn.dawn_msssp(g.handle, src, dist, par)
    dist.fill_(0)
    par.fill_(0)
    for _ in range(3):
        cg.replay()
    torch.cuda.synchronize()
    assert dawn.dawn_status(g.handle) == 0
    exact_rows(wl, wl.sources, dist.cpu().numpy(), par.cpu().numpy())


def test_msssp_automatic_batch_on_a_graph_larger_than_l2(dawn):
    # on R-MAT s20 fewer than 32 instances' packed states (8 MB each) fit L2
    # together, so the automatic batch splits 24 sources into launches of as
    # many as fit; every row must equal the single-source solve, and sampled
    # rows the oracle
    wl = gg.rmat_u32(20, 16, nsrc=24, seed=12)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)
    D, P = g.msssp(wl.sources)
    D, P = D.cpu().numpy(), P.cpu().numpy()
    assert g.stats()["instances"] == len(wl.sources)
    for i, s in enumerate(wl.sources):
        d1, p1, _ = g.sssp(int(s), parent=True)
        assert np.array_equal(D[i], d1.cpu().numpy()), i
        assert np.array_equal(P[i], p1.cpu().numpy()), i
    for i in (0, 23):
        d_ref, p_ref, _ = oracle.sssp(wl.row_ptr, wl.col, wl.weights, int(wl.sources[i]))
        assert np.array_equal(D[i], d_ref), i
        assert np.array_equal(P[i], p_ref), i
    g.close()
