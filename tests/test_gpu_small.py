"""GPU parity of the small-graph kernel (one block per instance, the solver
state and, when it fits, the CSR in shared memory) against the oracle and
against the persistent kernel on the same inputs: distances bit for bit,
parents and parent edges exactly, for every weight type and solve form."""
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


def both_paths(dawn, rp, cl, w, s, mode):
    out = []
    for path in (mode, dawn.DAWN_SMALL_NEVER):
        g = dawn.Graph(rp, cl, w)
        g.set_option(dawn.DAWN_OPT_SMALL_PATH, path)
        d, p, pe = g.sssp(int(s), parent=True, parent_edge=True)
        out.append((d.cpu().numpy(), p.cpu().numpy(), pe.cpu().numpy(), g.stats()))
    return out


def signed_graph(n, m, seed):
    rp, cl, w = gg.random_small(n, m, seed, kind="u32", wlo=1, whi=40)
    pot = (np.arange(n, dtype=np.int64) * 104729) % 17
    tails = np.repeat(np.arange(n), np.diff(rp))
    return rp, cl, (w.astype(np.int64) + pot[tails] - pot[cl]).astype(np.int32)


CASES = [
    ("tiny_u32", lambda: (lambda wl: (wl.row_ptr, wl.col, wl.weights, 0))(gg.tiny_er())),
    ("grid_f32", lambda: (lambda wl: (wl.row_ptr, wl.col, wl.weights, int(wl.sources[0])))(gg.grid_f32(60, 0.01, nsrc=1, seed=41))),
    ("multigraph_u32", lambda: gg.random_small(700, 5000, 42, kind="u32", wlo=0, whi=9, self_loops=True) + (3,)),
    ("dyadic_f32", lambda: gg.random_small(900, 6000, 43, kind="dyadic", wlo=0, whi=6) + (5,)),
    ("signed_i32", lambda: signed_graph(1200, 9000, 44) + (7,)),
    ("rmat_hubs_u32", lambda: (lambda wl: (wl.row_ptr, wl.col, wl.weights, int(wl.sources[0])))(gg.rmat_u32(10, 16, nsrc=1, seed=45))),
]


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_small_kernel_matches_oracle_and_persistent_kernel(dawn, name):
    rp, cl, w, s = dict(CASES)[name]()
    (d, p, pe, st), (d2, p2, pe2, _) = both_paths(dawn, rp, cl, w, s, dawn.DAWN_SMALL_AUTO)
    d_ref, p_ref, pe_ref = oracle.sssp(rp, cl, w, s)
    assert np.array_equal(bits(d), bits(d_ref))
    assert np.array_equal(p, p_ref) and np.array_equal(pe, pe_ref)
    assert np.array_equal(bits(d), bits(d2)) and np.array_equal(p, p2) and np.array_equal(pe, pe2)
    assert st["steps"] >= 1 and st["edges_scanned"] >= 1


def test_small_kernel_with_csr_in_global_memory(dawn):
    # the state fits on-chip, the CSR does not: edges are read from global memory
    wl = gg.rmat_u32(13, 16, nsrc=3, seed=46)
    for s in wl.sources:
        (d, p, pe, _), (d2, p2, pe2, _) = both_paths(dawn, wl.row_ptr, wl.col, wl.weights, s,
                                                    dawn.DAWN_SMALL_WHEN_STATE_FITS)
        d_ref, p_ref, pe_ref = oracle.sssp(wl.row_ptr, wl.col, wl.weights, int(s))
        assert np.array_equal(d, d_ref) and np.array_equal(p, p_ref) and np.array_equal(pe, pe_ref)
        assert np.array_equal(d, d2)


def test_small_kernel_batched_and_roots(dawn):
    wl = gg.tiny_er(n=800, avg_deg=6, seed=47)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    src = np.arange(0, 800, 3, dtype=np.int32)
    dist, par = g.msssp(src)
    D = oracle.floyd_warshall(wl.row_ptr, wl.col, wl.weights)
    assert np.array_equal(dist.cpu().numpy(), D[src])
    par = par.cpu().numpy()
    for i in (0, 100, len(src) - 1):
        _, p_ref, _ = oracle.sssp(wl.row_ptr, wl.col, wl.weights, int(src[i]))
        assert np.array_equal(par[i], p_ref)
    st = g.stats()
    assert st["instances"] == len(src)
    roots = np.array([5, 17, 5, 300], np.int32)
    d, p, pe = g.sssp_roots(roots, parent=True, parent_edge=True)
    d_ref = oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, roots)
    pe_ref = oracle.parent_edges(wl.row_ptr, wl.col, wl.weights, roots, d_ref)
    assert np.array_equal(d.cpu().numpy(), d_ref) and np.array_equal(pe.cpu().numpy(), pe_ref)


def test_small_kernel_edge_cases_and_errors(dawn):
    # n = 1, no edges
    g = dawn.Graph(np.array([0, 0], np.int32), np.zeros(0, np.int32), np.zeros(0, np.uint32))
    d, p, pe = g.sssp(0, parent=True, parent_edge=True)
    assert d.cpu().tolist() == [0] and p.cpu().tolist() == [0] and pe.cpu().tolist() == [-1]
    # unreachable part and a source without out-edges
    rp, cl, w = gg.csr_from_edges(5, [(0, 1), (1, 2), (3, 4)], [2, 3, 1], np.uint32)
    g = dawn.Graph(rp, cl, w)
    d, p, _ = g.sssp(0)
    assert d.cpu().numpy().tolist() == [0, 2, 5, 0xFFFFFFFF, 0xFFFFFFFF] and p.cpu().tolist() == [0, 0, 1, -1, -1]
    d, p, _ = g.sssp(2)
    assert d.cpu().numpy().tolist() == [0xFFFFFFFF, 0xFFFFFFFF, 0, 0xFFFFFFFF, 0xFFFFFFFF]
    # step cap on a path: NOT_CONVERGED
    n = 64
    rp, cl, w = gg.csr_from_edges(n, [(i, i + 1) for i in range(n - 1)], [1] * (n - 1), np.uint32)
    g = dawn.Graph(rp, cl, w)
    g.set_option(dawn.DAWN_OPT_MAX_STEPS, 10)
    with pytest.raises(dawn.DawnError) as e:
        g.sssp(0)
    assert e.value.code == dawn.DAWN_ERR_NOT_CONVERGED
    # a reachable negative cycle hits the step cap too
    rp, cl, w = gg.csr_from_edges(4, [(0, 1), (1, 2), (2, 1), (2, 3)], [1, -2, 1, 5], np.int32)
    g = dawn.Graph(rp, cl, w)
    with pytest.raises(dawn.DawnError) as e:
        g.sssp(0)
    assert e.value.code == dawn.DAWN_ERR_NOT_CONVERGED
    # invalid weights set without a synchronous check are refused by the solve
    wl = gg.grid_f32(20, 0.0, nsrc=1, seed=48)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    bad = torch.from_numpy(wl.weights).cuda().clone()
    bad[3] = -1.0
    dawn.dawn_set_weights(g.handle, bad, defer_check=True)
    dist = torch.full((g.n,), 9, dtype=torch.float32, device="cuda")
    dawn.dawn_sssp(g.handle, 0, dist)
    assert dawn.dawn_status(g.handle) == dawn.DAWN_ERR_INVALID and bool((dist == 9).all())


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("mode", ["auto", "state"])
def test_small_kernel_compact_form_without_parents(dawn, name, mode):
    # solves that want no parents on graphs of non-negative weights run the
    # compact form (32-bit keys, 16-bit frontier ids, two blocks per SM):
    # the same distances as the oracle; signed weights keep the packed form
    rp, cl, w, s = dict(CASES)[name]()
    g = dawn.Graph(rp, cl, w)
    g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_AUTO if mode == "auto" else dawn.DAWN_SMALL_WHEN_STATE_FITS)
    d_ref = oracle.sssp(rp, cl, w, s)[0]
    d, _, _ = g.sssp(int(s), parent=False)
    assert np.array_equal(bits(d.cpu().numpy()), bits(d_ref))
    srcs = np.array([s, 0, len(rp) - 2, s], np.int32)
    D, _ = g.msssp(srcs, parent=False)
    D = D.cpu().numpy()
    for i, r in enumerate(srcs):
        assert np.array_equal(bits(D[i]), bits(oracle.sssp(rp, cl, w, int(r))[0])), i
    dr, _, _ = g.sssp_roots(srcs[:3], parent=False)
    assert np.array_equal(bits(dr.cpu().numpy()), bits(oracle.sssp(rp, cl, w, srcs[:3])[0]))


def test_small_kernel_compact_apsp_against_floyd_warshall(dawn):
    # every vertex a source, no parents: the compact form, checked against
    # all-pairs Floyd-Warshall (exact for integer weights)
    wl = gg.tiny_er(n=512, avg_deg=6, seed=46)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    D, _ = g.msssp(np.arange(wl.n, dtype=np.int32), parent=False)
    assert np.array_equal(D.cpu().numpy(), oracle.floyd_warshall(wl.row_ptr, wl.col, wl.weights))


def hub_graph(seed, hubs=300, hub_deg=300, n=8192):
    """A source with an edge to each of `hubs` hubs, each hub with `hub_deg`
    out-edges to random vertices, and a sparse random background: hundreds of
    vertices in one frontier with far more out-edges than a thread group
    takes."""
    rng = np.random.default_rng(seed)
    hub_ids = rng.choice(np.arange(1, n), size=hubs, replace=False)
    src, dst = [np.zeros(hubs, np.int64)], [hub_ids.astype(np.int64)]
    for h in hub_ids:
        src.append(np.full(hub_deg, h, np.int64))
        dst.append(rng.integers(0, n, hub_deg))
    bg = 2 * n
    src.append(rng.integers(0, n, bg))
    dst.append(rng.integers(0, n, bg))
    src, dst = np.concatenate(src), np.concatenate(dst)
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    rp = np.zeros(n + 1, np.int32)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    w = rng.integers(1, 50, len(dst)).astype(np.uint32)
    return rp, dst.astype(np.int32), w


@pytest.mark.parametrize("parents", [True, False])
def test_small_kernel_many_hubs_in_one_frontier(dawn, parents):
    # 300 hubs enter the frontier together, each with about 19 times the
    # average out-degree; distances (compact form without parents, packed
    # form with them) and parents must equal the oracle's
    rp, cl, w = hub_graph(46)
    n = len(rp) - 1
    g = dawn.Graph(rp, cl, w)
    g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_WHEN_STATE_FITS)
    src = torch.tensor([0, 7, 1234], dtype=torch.int32, device="cuda")
    D = torch.empty((3, n), dtype=torch.uint32, device="cuda")
    P = torch.empty((3, n), dtype=torch.int32, device="cuda") if parents else None
    dawn.dawn_msssp(g.handle, src, D, P)
    g.check()
    for i, s in enumerate((0, 7, 1234)):
        d_ref, p_ref, _ = oracle.sssp(rp, cl, w, s)
        assert np.array_equal(D[i].cpu().numpy(), d_ref), i
        if parents:
            assert np.array_equal(P[i].cpu().numpy(), p_ref), i
    g.close()
