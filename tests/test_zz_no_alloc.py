"""GPU test of dawn_sssp_noalloc, the allocation-free solve.

Callers that cannot allocate device memory during a call (fixed memory
budgets, hosts that forbid allocator calls once running, code that must not
pay cudaMalloc's implicit synchronisation) use this entry point; it takes its
workspace from a fixed 32 MiB device array inside the library.  The test
calls it through the C ABI twice in a row and checks that it returns exactly
what dawn_sssp returns (distances bit for bit, parents exactly, the same
tolerance as every other parity test here), and that a graph too large for
the fixed array is refused.  The file name makes pytest collect it last.
"""
import numpy as np
import pytest
import torch

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dawn():
    import paper_2306_07872_gb300 as pkg
    pkg.load_library()
    assert torch.cuda.is_available()
    return pkg


def solve_both(dawn, g, source):
    n = g.n
    ref = g.sssp(source, parent=True, parent_edge=True)
    outs = []
    for _ in range(2):  # two calls in a row share (and reuse) the fixed array
        dist = torch.empty(n, dtype=g.dist_dtype, device="cuda")
        par = torch.empty(n, dtype=torch.int32, device="cuda")
        pe = torch.empty(n, dtype=torch.int32, device="cuda")
        status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        dawn.dawn_sssp_noalloc(g.handle, source, dist, par, pe, status)
        torch.cuda.synchronize()
        assert int(status.item()) == dawn.DAWN_OK
        outs.append((dist, par, pe))
    for dist, par, pe in outs:
        assert np.array_equal(dist.cpu().numpy().view(np.uint32), ref[0].cpu().numpy().view(np.uint32))
        assert torch.equal(par, ref[1]) and torch.equal(pe, ref[2])


def test_noalloc_matches_dawn_sssp_uint32(dawn):
    wl = gg.tiny_er()
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    solve_both(dawn, g, 0)
    solve_both(dawn, g, 17)


def test_noalloc_matches_dawn_sssp_float32_after_a_larger_graph(dawn):
    big = gg.rmat_u32(15, 16, nsrc=1, seed=2)  # leaves a larger workspace behind in the array
    gb = dawn.Graph(big.row_ptr, big.col, big.weights)
    solve_both(dawn, gb, int(big.sources[0]))
    wl = gg.grid_f32(96, 0.01, nsrc=2, seed=3)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    solve_both(dawn, g, int(wl.sources[0]))
    solve_both(dawn, g, int(wl.sources[1]))


def test_noalloc_refuses_graphs_beyond_the_fixed_array(dawn):
    n = 2_000_000  # about 24 bytes per vertex: needs more than 32 MiB
    rp = np.zeros(n + 1, dtype=np.int32)
    rp[1:] = 1
    g = dawn.Graph(rp, np.array([1], np.int32), np.array([3], np.uint32))
    dist = torch.empty(n, dtype=torch.uint32, device="cuda")
    with pytest.raises(dawn.DawnError) as e:
        dawn.dawn_sssp_noalloc(g.handle, 0, dist)
    assert e.value.code == dawn.DAWN_ERR_INVALID
