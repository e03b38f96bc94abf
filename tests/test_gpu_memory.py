"""GPU tests of the library's device memory: every handle allocates from a
stream-ordered pool per device.  A graph created on its own stream while
another handle's solves run, then the old handle destroyed (a serving loop),
gives the oracle's results; a destroyed handle's memory serves the next
handle, stays in the pool and goes back to the device on dawn_trim_memory;
allocation is
refused while the stream is being captured; host threads that create, solve
and destroy their own graphs at the same time share the pool safely."""
import gc

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

MB = 1 << 20


@pytest.fixture(scope="module")
def dawn():
    import paper_2306_07872_gb300 as pkg
    pkg.load_library()
    return pkg


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def host_create(dawn, wl, stream=None):
    return dawn.dawn_create_graph(torch.from_numpy(wl.row_ptr), torch.from_numpy(wl.col),
                                  torch.from_numpy(wl.weights), stream)


def test_pipelined_create_solve_destroy_matches_oracle(dawn):
    # each step: the step's solves run on one stream while the next graph is
    # created on another; the old handle is destroyed once its results are in
    wls = [gg.rmat_u32(13, 8, nsrc=3, seed=40 + i) for i in range(4)]
    solve_s, ingest_s = torch.cuda.Stream(), torch.cuda.Stream()
    dist = [torch.empty((3, wl.n), dtype=torch.uint32, device="cuda") for wl in wls]
    par = [torch.empty((3, wl.n), dtype=torch.int32, device="cuda") for wl in wls]
    torch.cuda.synchronize()
    h = host_create(dawn, wls[0], ingest_s)
    for i, wl in enumerate(wls):
        dawn.dawn_set_option(h, dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)  # needs a workspace
        solve_s.wait_stream(ingest_s)
        for j, s in enumerate(wl.sources):
            dawn.dawn_sssp(h, int(s), dist[i][j], par[i][j], None, solve_s)
        h_next = host_create(dawn, wls[i + 1], ingest_s) if i + 1 < len(wls) else None
        assert dawn.dawn_status(h, True) == 0
        dawn.dawn_destroy(h)
        h = h_next
    torch.cuda.synchronize()
    for i, wl in enumerate(wls):
        d, p = dist[i].cpu().numpy(), par[i].cpu().numpy()
        for j, s in enumerate(wl.sources):
            d_ref, p_ref, _ = oracle.sssp(wl.row_ptr, wl.col, wl.weights, int(s))
            assert np.array_equal(d[j].view(np.uint32), d_ref.view(np.uint32)), (i, j)
            assert np.array_equal(p[j], p_ref), (i, j)


def test_destroyed_handle_memory_is_reused_then_returned(dawn):
    wl = gg.rmat_u32(19, 16, nsrc=1, seed=3)  # about 100 MB of graph and workspace per handle
    src = int(wl.sources[0])
    d_ref, _, _ = oracle.sssp(wl.row_ptr, wl.col, wl.weights, src)
    dist = torch.empty(wl.n, dtype=torch.uint32, device="cuda")

    def make():
        h = host_create(dawn, wl)
        dawn.dawn_set_option(h, dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)
        dawn.dawn_sssp(h, src, dist)
        assert dawn.dawn_status(h, True) == 0
        assert np.array_equal(dist.cpu().numpy(), d_ref)
        return h

    gc.collect()  # handles of earlier tests are gone
    dawn.dawn_trim_memory()  # and the pool holds nothing
    free0 = free_bytes()
    a = make()
    b = make()
    free_ab = free_bytes()
    per_handle = (free0 - free_ab) / 2
    assert per_handle > 60 * MB
    dawn.dawn_destroy(a)
    assert abs(free_bytes() - free_ab) <= 4 * MB  # kept in the pool while b lives
    c = make()  # served mostly from a's freed blocks
    assert free_ab - free_bytes() < per_handle / 2
    dawn.dawn_destroy(b)
    dawn.dawn_destroy(c)
    free_kept = free_bytes()
    assert free_kept < free0 - per_handle  # with no handle left the pool still holds the memory
    dawn.dawn_trim_memory()
    assert free_bytes() >= free0 - 8 * MB  # and gives it back when trimmed
    h = make()  # a trimmed pool serves new handles as before
    dawn.dawn_destroy(h)
    dawn.dawn_trim_memory()


def test_allocation_refused_during_capture_then_reserve(dawn):
    wl = gg.rmat_u32(11, 8, nsrc=1, seed=5)
    src = int(wl.sources[0])
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    g.set_option(dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)
    dist = torch.empty(wl.n, dtype=torch.uint32, device="cuda")
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(cg):
        try:
            dawn.dawn_sssp(g.handle, src, dist)  # no workspace yet: it would allocate
        except dawn.DawnError as e:
            refused = e
    assert refused is not None and refused.code == dawn.DAWN_ERR_CUDA
    dawn.dawn_reserve(g.handle, 1)
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        dawn.dawn_sssp(g.handle, src, dist)
    dist.fill_(0)
    cg.replay()
    torch.cuda.synchronize()
    assert dawn.dawn_status(g.handle) == 0
    d_ref, _, _ = oracle.sssp(wl.row_ptr, wl.col, wl.weights, src)
    assert np.array_equal(dist.cpu().numpy(), d_ref)
    g.close()


def test_handles_created_and_destroyed_on_several_threads(dawn):
    # host threads share the library's pool: each creates, solves and
    # destroys its own graphs on its own stream while the others do the same
    import threading
    wls = [[gg.rmat_u32(12, 8, nsrc=2, seed=60 + 10 * t + i) for i in range(3)] for t in range(4)]
    results, errors = {}, []

    def work(t):
        try:
            s = torch.cuda.Stream()
            for i, wl in enumerate(wls[t]):
                h = host_create(dawn, wl, s)
                dawn.dawn_set_option(h, dawn.DAWN_OPT_SMALL_PATH, dawn.DAWN_SMALL_NEVER)
                dist = torch.empty((2, wl.n), dtype=torch.uint32, device="cuda")
                par = torch.empty((2, wl.n), dtype=torch.int32, device="cuda")
                s.wait_stream(torch.cuda.current_stream())  # the outputs' allocation is ordered before the solves
                for j, src in enumerate(wl.sources):
                    dawn.dawn_sssp(h, int(src), dist[j], par[j], None, s)
                assert dawn.dawn_status(h, True) == 0
                dawn.dawn_destroy(h)
                results[(t, i)] = (dist.cpu().numpy(), par.cpu().numpy())
        except Exception as e:  # reported by the main thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    for t in range(4):
        for i, wl in enumerate(wls[t]):
            d, p = results[(t, i)]
            for j, src in enumerate(wl.sources):
                d_ref, p_ref, _ = oracle.sssp(wl.row_ptr, wl.col, wl.weights, int(src))
                assert np.array_equal(d[j], d_ref), (t, i, j)
                assert np.array_equal(p[j], p_ref), (t, i, j)
