"""GPU tests of weight replacement (dawn_set_weights): synchronous and
deferred validation, and the solve-side refusal of weights that failed it.

Every solve checks the validation verdict of the weights in force, so a
deferred check (no host synchronisation) still stops a solve on invalid
weights: it writes no output and reports DAWN_ERR_INVALID.
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


def solve_raw(dawn, g, s):
    dist = torch.full((g.n,), 7, dtype=g.dist_dtype, device="cuda")
    dawn.dawn_sssp(g.handle, s, dist)
    return dist, dawn.dawn_status(g.handle, True)


def test_deferred_check_refuses_negative_float_weight(dawn):
    wl = gg.grid_f32(40, 0.01, nsrc=1, seed=31)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    s = int(wl.sources[0])
    bad = torch.from_numpy(wl.weights).cuda().clone()
    bad[123] = -0.5
    dawn.dawn_set_weights(g.handle, bad, defer_check=True)  # returns at once
    dist, code = solve_raw(dawn, g, s)
    assert code == dawn.DAWN_ERR_INVALID
    assert bool((dist == 7).all())  # nothing written
    for v in (float("nan"), float("inf")):
        bad[123] = v
        dawn.dawn_set_weights(g.handle, bad, defer_check=True)
        assert solve_raw(dawn, g, s)[1] == dawn.DAWN_ERR_INVALID
    good = torch.from_numpy(wl.weights).cuda()
    dawn.dawn_set_weights(g.handle, good, defer_check=True)
    dist, code = solve_raw(dawn, g, s)
    assert code == dawn.DAWN_OK
    d_ref = oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, s)
    assert np.array_equal(dist.cpu().numpy().view(np.uint32), d_ref.view(np.uint32))


def test_synchronous_rejection_also_blocks_later_solves(dawn):
    wl = gg.rmat_u32(10, 8, nsrc=1, seed=32)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    s = int(wl.sources[0])
    huge = np.full_like(wl.weights, 0xFFFFFF00)  # n * max(w) overflows the uint32 distance range
    with pytest.raises(dawn.DawnError) as e:
        dawn.dawn_set_weights(g.handle, torch.from_numpy(huge))
    assert e.value.code == dawn.DAWN_ERR_INVALID
    assert solve_raw(dawn, g, s)[1] == dawn.DAWN_ERR_INVALID
    dawn.dawn_set_weights(g.handle, torch.from_numpy(wl.weights))  # host input, checked synchronously
    dist, code = solve_raw(dawn, g, s)
    assert code == dawn.DAWN_OK
    assert np.array_equal(dist.cpu().numpy(), oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, s))


def test_deferred_overflow_check_signed(dawn):
    rp, cl, w = gg.random_small(500, 3000, 33, kind="u32", wlo=1, whi=9)
    wi = w.astype(np.int32)
    g = dawn.Graph(rp, cl, wi)
    big = wi.copy()
    big[0] = -(2**30)  # n * max|w| leaves the int32 range
    dawn.dawn_set_weights(g.handle, torch.from_numpy(big).cuda(), defer_check=True)
    assert solve_raw(dawn, g, 0)[1] == dawn.DAWN_ERR_INVALID
    dawn.dawn_set_weights(g.handle, torch.from_numpy(wi).cuda(), defer_check=True)
    dist, code = solve_raw(dawn, g, 0)
    assert code == dawn.DAWN_OK
    d_ref, _, _ = oracle.sssp(rp, cl, wi, 0)
    assert np.array_equal(dist.cpu().numpy(), d_ref)


def test_bad_flags_rejected(dawn):
    wl = gg.tiny_er()
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    lib = dawn.load_library()
    import ctypes
    w = torch.from_numpy(wl.weights).cuda()
    rc = lib.dawn_set_weights(ctypes.c_void_p(g.handle), ctypes.c_void_p(w.data_ptr()), 4, None)
    assert rc == dawn.DAWN_ERR_INVALID


def test_autograd_without_sync_matches(dawn):
    wl = gg.rmat_f32_diff(scale=11, edge_factor=8, ntargets=32, seed=34)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    w = torch.from_numpy(wl.weights).cuda()
    tg = torch.from_numpy(wl.extra["targets"]).long().cuda()
    cf = torch.from_numpy(wl.extra["coef"]).float().cuda()
    grads = []
    for check in (True, False):
        ww = w.clone().requires_grad_(True)
        d = dawn.DawnSSSP.apply(ww, g, 0, check)
        (d[tg] * cf).sum().backward()
        g.check()
        grads.append((d.detach().cpu().numpy(), ww.grad.cpu().numpy()))
    assert np.array_equal(grads[0][0].view(np.uint32), grads[1][0].view(np.uint32))
    # the backward sums with float32 atomics, whose order varies between runs
    np.testing.assert_allclose(grads[0][1], grads[1][1], rtol=1e-5, atol=1e-6)


def test_host_weights_staging_allocation_failure(dawn):
    # host weights go through a device staging copy, allocated on the first
    # such call; a failed allocation leaves the weights in force untouched
    wl = gg.grid_f32(30, 0.01, nsrc=1, seed=35)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    s = int(wl.sources[0])
    w2 = (wl.weights * np.float32(2.0)).astype(np.float32)
    g.set_option(dawn.DAWN_OPT_TEST_FAIL_ALLOC, 1)
    with pytest.raises(dawn.DawnError) as e:
        dawn.dawn_set_weights(g.handle, torch.from_numpy(w2))
    assert e.value.code == dawn.DAWN_ERR_OOM
    dist, code = solve_raw(dawn, g, s)
    assert code == dawn.DAWN_OK
    assert np.array_equal(dist.cpu().numpy().view(np.uint32),
                          oracle.dijkstra(wl.row_ptr, wl.col, wl.weights, s).view(np.uint32))
    dawn.dawn_set_weights(g.handle, torch.from_numpy(w2))  # allocates and copies now
    dawn.dawn_set_weights(g.handle, torch.from_numpy(w2))  # reuses the staging copy
    dist, code = solve_raw(dawn, g, s)
    assert code == dawn.DAWN_OK
    assert np.array_equal(dist.cpu().numpy().view(np.uint32), oracle.dijkstra(wl.row_ptr, wl.col, w2, s).view(np.uint32))
