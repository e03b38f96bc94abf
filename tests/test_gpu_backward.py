"""GPU parity of the differentiable solver: the backward kernel's dL/dw
against the oracle's float64 subtree-sum gradient and float64 central finite
differences, with the parent tree as the only saved state.

Tolerance: |g - g_ref| <= 1e-4 * max(|g_ref|, sum over the edge's subtree of
|c_t|); the scale term covers fp32 atomic accumulation of many terms.
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
    return pkg


def run_diff(dawn, wl):
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    w = torch.from_numpy(wl.weights).cuda().requires_grad_(True)
    dist = dawn.DawnSSSP.apply(w, g, 0)
    tg = torch.from_numpy(wl.extra["targets"]).long().cuda()
    cf = torch.from_numpy(wl.extra["coef"]).float().cuda()
    loss = (dist[tg] * cf).sum()
    loss.backward()
    c = np.zeros(wl.n)
    c[wl.extra["targets"]] = wl.extra["coef"].astype(np.float32).astype(np.float64)
    return g, dist.detach().cpu().numpy(), w.grad.cpu().numpy(), c


def subtree_abs(wl, pe, c):
    return oracle.subtree_grad(wl.row_ptr, wl.col, wl.weights, 0, np.abs(c), parent_edge=pe)


def test_backward_matches_reference_gradient(dawn):
    wl = gg.rmat_f32_diff(scale=12, edge_factor=16, ntargets=128, seed=2)
    g, dist, grad, c = run_diff(dawn, wl)
    d_ref, _, pe_ref = oracle.sssp(wl.row_ptr, wl.col, wl.weights, 0)
    assert np.array_equal(dist.view(np.uint32), d_ref.view(np.uint32))
    g_ref = oracle.subtree_grad(wl.row_ptr, wl.col, wl.weights, 0, c, parent_edge=pe_ref)
    scale = np.maximum(np.abs(g_ref), subtree_abs(wl, pe_ref, c))
    assert np.all(np.abs(grad - g_ref) <= 1e-4 * scale + 1e-30)
    assert np.all(grad[g_ref == 0] == 0)  # off-tree edges are exactly zero


def test_backward_against_finite_differences(dawn):
    wl = gg.rmat_f32_diff(scale=11, edge_factor=16, ntargets=64, seed=4)
    g, dist, grad, c = run_diff(dawn, wl)
    nz = np.nonzero(grad)[0]
    pick = nz[gg.below(5, 0, 60, len(nz))]
    fd, stable = oracle.fd_grad(wl.row_ptr, wl.col, wl.weights, 0, c, pick, h=1e-3)
    assert stable.sum() >= 40
    _, _, pe_ref = oracle.sssp(wl.row_ptr, wl.col, wl.weights, 0)
    scale = np.maximum(np.abs(fd), subtree_abs(wl, pe_ref, c)[pick])
    assert np.all(np.abs(grad[pick] - fd)[stable] <= 1e-4 * scale[stable])


def test_backward_dense_grad_and_unreachable(dawn):
    # dense dL/ddist including unreachable vertices (ignored) and the root
    wl = gg.rmat_f32_diff(scale=10, edge_factor=4, ntargets=4, seed=3)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    dist, _, pe = g.sssp(0, parent=False, parent_edge=True)
    cvec = torch.from_numpy(gg.uniform01(9, 0, wl.n).astype(np.float32) - 0.5).cuda()
    grad_w = torch.empty(wl.m, dtype=torch.float32, device="cuda")
    dawn.dawn_sssp_backward(g.handle, pe, cvec, grad_w)
    g.check()
    c = cvec.cpu().numpy().astype(np.float64)
    fin = np.isfinite(dist.cpu().numpy())
    c_eff = np.where(fin, c, 0.0)
    pe_np = pe.cpu().numpy()
    g_ref = oracle.subtree_grad(wl.row_ptr, wl.col, wl.weights, 0, c_eff, parent_edge=pe_np)
    scale = np.maximum(np.abs(g_ref), subtree_abs(wl, pe_np, c_eff))
    assert np.all(np.abs(grad_w.cpu().numpy() - g_ref) <= 1e-4 * scale + 1e-30)


def test_backward_rejects_cyclic_parent_array(dawn):
    rp, cl, w = gg.csr_from_edges(3, [(0, 1), (1, 2), (2, 1)], [1.0, 1.0, 1.0], np.float32)
    g = dawn.Graph(rp, cl, w)
    pe = torch.tensor([-1, 2, 1], dtype=torch.int32, device="cuda")  # 1 <- 2 <- 1
    gd = torch.ones(3, dtype=torch.float32, device="cuda")
    gw = torch.empty(3, dtype=torch.float32, device="cuda")
    dawn.dawn_sssp_backward(g.handle, pe, gd, gw)
    assert dawn.dawn_status(g.handle) == dawn.DAWN_ERR_INVALID


def test_backward_dense_grad_on_deep_tree(dawn):
    # every vertex of a grid (tree depth in the hundreds) carries a gradient:
    # each tree edge is handled once, children before parents
    wl = gg.grid_f32(160, 0.0, nsrc=1, seed=5)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    s = int(wl.sources[0])
    dist, _, pe = g.sssp(s, parent=False, parent_edge=True)
    cvec = torch.from_numpy(gg.uniform01(11, 0, wl.n).astype(np.float32) + 0.5).cuda()
    grad_w = torch.empty(wl.m, dtype=torch.float32, device="cuda")
    for _ in range(2):  # the scratch of the first call is reused by the second
        dawn.dawn_sssp_backward(g.handle, pe, cvec, grad_w)
        g.check()
        pe_np = pe.cpu().numpy()
        c = cvec.cpu().numpy().astype(np.float64)
        g_ref = oracle.subtree_grad(wl.row_ptr, wl.col, wl.weights, s, c, parent_edge=pe_np)
        got = grad_w.cpu().numpy()
        assert np.all(np.abs(got - g_ref) <= 1e-4 * np.abs(g_ref) + 1e-30)
        on_tree = np.zeros(wl.m, bool)
        on_tree[pe_np[pe_np >= 0]] = True
        assert np.all(got[~on_tree] == 0) and np.all(got[on_tree] > 0)


def test_backward_scratch_allocation_failure(dawn):
    wl = gg.rmat_f32_diff(scale=10, edge_factor=4, ntargets=4, seed=6)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    dist, _, pe = g.sssp(0, parent=False, parent_edge=True)
    gd = torch.ones(wl.n, dtype=torch.float32, device="cuda")
    gw = torch.empty(wl.m, dtype=torch.float32, device="cuda")
    g.set_option(dawn.DAWN_OPT_TEST_FAIL_ALLOC, 1)  # the scratch allocation
    with pytest.raises(dawn.DawnError) as e:
        dawn.dawn_sssp_backward(g.handle, pe, gd, gw)
    assert e.value.code == dawn.DAWN_ERR_OOM
    dawn.dawn_sssp_backward(g.handle, pe, gd, gw)  # allocates again and runs
    g.check()
    pe_np = pe.cpu().numpy()
    c = np.where(np.isfinite(dist.cpu().numpy()), 1.0, 0.0)
    g_ref = oracle.subtree_grad(wl.row_ptr, wl.col, wl.weights, 0, c, parent_edge=pe_np)
    assert np.all(np.abs(gw.cpu().numpy() - g_ref) <= 1e-4 * np.abs(g_ref) + 1e-30)


def test_autograd_step_captured_in_cuda_graph(dawn):
    # forward (weights loaded + solve), loss and backward captured once and
    # replayed with new weights written into the same tensor: every replay
    # gives the oracle's distances and gradient for those weights
    wl = gg.rmat_f32_diff(scale=12, edge_factor=8, ntargets=32, seed=36)
    g = dawn.Graph(wl.row_ptr, wl.col, wl.weights)
    ww = torch.from_numpy(wl.weights).cuda().requires_grad_(True)
    tg = torch.from_numpy(wl.extra["targets"]).long().cuda()
    cf = torch.from_numpy(wl.extra["coef"]).float().cuda()

    def step():
        d = dawn.DawnSSSP.apply(ww, g, 0, False)
        (d[tg] * cf).sum().backward()
        return d
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside capture (the first backward allocates its scratch)
        for _ in range(2):
            ww.grad = None
            step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    ww.grad = None
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        d_static = step()
    c = np.zeros(wl.n)
    c[wl.extra["targets"]] = wl.extra["coef"].astype(np.float32).astype(np.float64)
    for scale in (1.0, 0.75, 1.25):
        w_np = (wl.weights * np.float32(scale)).astype(np.float32)
        with torch.no_grad():
            ww.copy_(torch.from_numpy(w_np).cuda())
        cg.replay()
        torch.cuda.synchronize()
        g.check()
        d_ref, _, pe_ref = oracle.sssp(wl.row_ptr, wl.col, w_np, 0)
        assert np.array_equal(d_static.detach().cpu().numpy().view(np.uint32), d_ref.view(np.uint32))
        g_ref = oracle.subtree_grad(wl.row_ptr, wl.col, w_np, 0, c, parent_edge=pe_ref)
        sabs = oracle.subtree_grad(wl.row_ptr, wl.col, w_np, 0, np.abs(c), parent_edge=pe_ref)
        got = ww.grad.cpu().numpy()
        assert np.all(np.abs(got - g_ref) <= 1e-4 * np.maximum(np.abs(g_ref), sabs) + 1e-30), scale
