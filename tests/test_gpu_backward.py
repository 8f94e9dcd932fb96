"""The hand-written backward kernels against the oracle's analytic Jacobian
and FP64 finite differences (4-point offset regression workload)."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2402_18008_gb300 import _lib
from paper_2402_18008_gb300.autograd import ACAFunction, ACARectFunction
from tests.gpu_util import cuda

pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-3   # max |g_gpu - g_ref| / max |g_ref| per set


def _rel(g, ref):
    return (np.abs(g - ref).max(axis=0) / np.abs(ref).max(axis=0)).max()


def test_general_backward_matches_analytic_jacobian():
    n = 4096
    ms = workloads.minimal_sets(n, seed=0)
    rng = np.random.default_rng(1)
    G = rng.standard_normal((9, n)).astype(np.float32)
    gt = torch.empty((8, n), device="cuda")
    _lib.aca_backward(cuda(ms.pts), cuda(G), gt)
    torch.cuda.synchronize()
    J = oracle.aca_jacobian(ms.pts)
    ref = np.einsum("nik,in->kn", J, G.astype(np.float64))
    r = _rel(gt.cpu().numpy(), ref)
    print(f"aca_backward rel err {r:.3e}")
    assert r < GRAD_TOL


@pytest.mark.parametrize("n,ld", [(1, 1), (5, 8), (7, 7), (1023, 1024), ((1 << 18) + 3, (1 << 18) + 4)])
def test_backward_ragged(n, ld):
    ms = workloads.minimal_sets(n, seed=2)
    pts = torch.zeros((16, ld), device="cuda")
    pts[:, :n] = cuda(ms.pts)
    G = torch.zeros((9, ld), device="cuda")
    G[:, :n] = torch.randn((9, n), generator=torch.Generator().manual_seed(3)).cuda()
    gt = torch.full((8, ld), 7.0, device="cuda")
    _lib.aca_backward(pts, G, gt, n=n)
    torch.cuda.synchronize()
    ref = np.einsum("nik,in->kn", oracle.aca_jacobian(ms.pts), G[:, :n].cpu().numpy().astype(np.float64))
    assert _rel(gt[:, :n].cpu().numpy(), ref) < GRAD_TOL
    if ld > n:
        assert torch.all(gt[:, n:] == 7.0)


@pytest.mark.parametrize("B", [65536, (1 << 18) + 1])
def test_rect_backward_matches_analytic_jacobian(B):
    rb = workloads.rect_batch(B, seed=0)
    rng = np.random.default_rng(4)
    G = rng.standard_normal((9, B)).astype(np.float32)
    gt = torch.empty((8, B), device="cuda")
    _lib.aca_rect_backward(cuda(rb.tgt), rb.rect, cuda(G), gt)
    torch.cuda.synchronize()
    J = oracle.aca_rect_jacobian(rb.tgt, rb.rect)
    ref = np.einsum("nik,in->kn", J, G.astype(np.float64))
    r = _rel(gt.cpu().numpy(), ref)
    print(f"rect backward rel err {r:.3e}")
    assert r < GRAD_TOL


def _grid_loss_fp64(H_rows, Hgt_rows, grid):
    X = np.stack([grid[:, 0], grid[:, 1], np.ones(len(grid))])
    L = 0.0
    for h, hg in zip(H_rows, Hgt_rows):
        a = h.reshape(3, 3) @ X
        b = hg.reshape(3, 3) @ X
        L += np.sum((a[:2] / a[2] - b[:2] / b[2]) ** 2)
    return L


def test_autograd_offset_regression_loss_vs_fp64_finite_differences():
    B = 65536
    rb = workloads.rect_batch(B, seed=0)
    x0, y0, w, r = rb.rect
    grid = workloads.grid_points(x0, y0, w, w / r, 8)
    tgt = cuda(rb.tgt).requires_grad_(True)
    H = ACARectFunction.apply(tgt, rb.rect)
    with torch.no_grad():
        Hgt = torch.empty((9, B), device="cuda")
        _lib.aca_rect_solve(cuda(rb.tgt_gt), rb.rect, Hgt)
    g = torch.tensor(grid.T, dtype=torch.float32, device="cuda")
    Hm = H.t().reshape(B, 3, 3)
    Hg = Hgt.t().reshape(B, 3, 3)
    Xh = torch.cat([g, torch.ones((1, 64), device="cuda")], 0)
    a = Hm @ Xh
    b = Hg @ Xh
    loss = ((a[:, :2] / a[:, 2:] - b[:, :2] / b[:, 2:]) ** 2).sum()
    loss.backward()
    grad = tgt.grad[:, :64].cpu().numpy().astype(np.float64)
    # FP64 central differences of the same loss through the oracle, 64 sets
    t64 = rb.tgt[:, :64].astype(np.float64)
    Hgt64 = oracle.aca_rect(rb.tgt_gt[:, :64], rb.rect)
    fd = np.zeros((8, 64))
    step = 1e-6
    for k in range(8):
        tp, tm = t64.copy(), t64.copy()
        tp[k] += step
        tm[k] -= step
        for i in range(64):
            Lp = _grid_loss_fp64(oracle.aca_rect(tp[:, i:i + 1], rb.rect), Hgt64[i:i + 1], grid)
            Lm = _grid_loss_fp64(oracle.aca_rect(tm[:, i:i + 1], rb.rect), Hgt64[i:i + 1], grid)
            fd[k, i] = (Lp - Lm) / (2 * step)
    rel = np.abs(grad - fd).max(axis=0) / np.maximum(np.abs(fd).max(axis=0), 1e-12)
    print(f"offset regression grad vs FP64 FD: max rel {rel.max():.3e}")
    assert rel.max() < 1e-2


def test_general_autograd_function_gradient():
    n = 256
    ms = workloads.minimal_sets(n, seed=11)
    src = cuda(ms.pts[:8])
    tgt = cuda(ms.pts[8:]).requires_grad_(True)
    H = ACAFunction.apply(src, tgt)
    G = torch.randn((9, n), generator=torch.Generator().manual_seed(5)).cuda()
    (H * G).sum().backward()
    ref = np.einsum("nik,in->kn", oracle.aca_jacobian(ms.pts), G.cpu().numpy().astype(np.float64))
    assert _rel(tgt.grad.cpu().numpy(), ref) < GRAD_TOL
