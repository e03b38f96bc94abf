"""GPU tests of dawn_sssp_noalloc, the allocation-free solve.

Some callers cannot allocate device memory while they run: code inside a
memory budget fixed up front, hosts that forbid allocator calls once they are
running, and code that must not pay the implicit synchronisation of
cudaMalloc / cudaFree.  dawn_sssp_noalloc serves them by taking its workspace
from a fixed 32 MiB device array inside the library.

These tests call it through the C ABI twice in a row per source and check
each result against the CPU oracle (distances bit for bit, parents and parent
edges exactly: the same bar as every other parity test here) and against
dawn_sssp on the same handle.  They also check the status path (weights whose
deferred validation fails are refused through status_out and through
dawn_status) and that a graph too large for the fixed array is refused before
anything runs.  The file name makes pytest collect it last.
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
    assert torch.cuda.is_available()
    return pkg


def noalloc(dawn, g, source, status=True):
    n = g.n
    dist = torch.empty(n, dtype=g.dist_dtype, device="cuda")
    par = torch.empty(n, dtype=torch.int32, device="cuda")
    pe = torch.empty(n, dtype=torch.int32, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda") if status else None
    dawn.dawn_sssp_noalloc(g.handle, source, dist, par, pe, st)
    return dist, par, pe, st


def check_source(dawn, g, wl, source):
    d_ref, p_ref, pe_ref = oracle.sssp(wl.row_ptr, wl.col, wl.weights, source)
    mine = g.sssp(source, parent=True, parent_edge=True)
    for _ in range(2):  # two calls in a row share (and reuse) the fixed array
        dist, par, pe, st = noalloc(dawn, g, source)
        torch.cuda.synchronize()
        assert int(st.item()) == dawn.DAWN_OK
        assert dawn.dawn_status(g.handle, True) == dawn.DAWN_OK
        d = dist.cpu().numpy()
        assert np.array_equal(d.view(np.uint32), np.asarray(d_ref).view(np.uint32))
        assert np.array_equal(par.cpu().numpy(), p_ref)
        assert np.array_equal(pe.cpu().numpy(), pe_ref)
        assert np.array_equal(d.view(np.uint32), mine[0].cpu().numpy().view(np.uint32))
        assert torch.equal(par, mine[1]) and torch.equal(pe, mine[2])
        # the handle reports this solve's counters
        assert g.stats()["steps"] >= 1 and g.stats()["instances"] == 1


def test_noalloc_matches_oracle_uint32(dawn):
    wl = gg.tiny_er()
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    check_source(dawn, g, wl, 0)
    check_source(dawn, g, wl, 17)


def test_noalloc_matches_oracle_float32_after_a_larger_graph(dawn):
    big = gg.rmat_u32(15, 16, nsrc=1, seed=2)  # leaves a larger workspace behind in the array
    gb = dawn.Graph(big.row_ptr, big.col, big.weights)
    check_source(dawn, gb, big, int(big.sources[0]))
    wl = gg.grid_f32(96, 0.01, nsrc=2, seed=3)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    check_source(dawn, g, wl, int(wl.sources[0]))
    check_source(dawn, g, wl, int(wl.sources[1]))


def test_noalloc_reports_deferred_invalid_weights(dawn):
    wl = gg.grid_f32(32, 0.0, nsrc=1, seed=4)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    bad = torch.from_numpy(wl.weights.copy())
    bad[5] = -1.0
    dawn.dawn_set_weights(g.handle, bad.cuda(), defer_check=True)
    dist, _, _, st = noalloc(dawn, g, 0)
    torch.cuda.synchronize()
    assert int(st.item()) == dawn.DAWN_ERR_INVALID
    assert dawn.dawn_status(g.handle, True) == dawn.DAWN_ERR_INVALID
    # without status_out the handle's status is the only report
    dist, _, _, _ = noalloc(dawn, g, 0, status=False)
    assert dawn.dawn_status(g.handle, True) == dawn.DAWN_ERR_INVALID
    # valid weights again: the next call succeeds and matches the oracle
    dawn.dawn_set_weights(g.handle, torch.from_numpy(wl.weights).cuda())
    dist, par, pe, st = noalloc(dawn, g, 0)
    torch.cuda.synchronize()
    assert int(st.item()) == dawn.DAWN_OK and dawn.dawn_status(g.handle, True) == dawn.DAWN_OK
    d_ref, p_ref, _ = oracle.sssp(wl.row_ptr, wl.col, wl.weights, 0)
    assert np.array_equal(dist.cpu().numpy().view(np.uint32), d_ref.view(np.uint32))
    assert np.array_equal(par.cpu().numpy(), p_ref)


def test_noalloc_refuses_graphs_beyond_the_fixed_array(dawn):
    n = 2_000_000  # about 24 bytes per vertex: needs more than 32 MiB
    rp = np.zeros(n + 1, dtype=np.int32)
    rp[1:] = 1
    g = dawn.Graph(rp, np.array([1], np.int32), np.array([3], np.uint32))
    dist = torch.empty(n, dtype=torch.uint32, device="cuda")
    with pytest.raises(dawn.DawnError) as e:
        dawn.dawn_sssp_noalloc(g.handle, 0, dist)
    assert e.value.code == dawn.DAWN_ERR_INVALID
