"""Stream order of the library's kernels.

The solve, affine, rectangle and backward kernels are launched as
programmatic dependents of the kernel before them in the stream: one may be
scheduled while its predecessor's last blocks still run, and it waits for
the predecessor at entry before it reads or writes anything.  These tests
run chains in which each call reads what the call before it wrote
(read-after-write), or writes what the call before it read
(write-after-read), mixed with torch kernels, with no synchronisation inside
the chain, and require the results of the same calls made one at a time
with a device synchronisation after each: bit for bit.
"""
import pytest
import torch

from paper_2402_18008_gb300 import _lib

pytestmark = pytest.mark.gpu

RECT = (40.0, 30.0, 256.0, 0.75)


def _same(x, y):
    """Bitwise equality (NaN and inf included)."""
    return torch.equal(x.view(torch.int32), y.view(torch.int32))


def _sets(n, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    return torch.rand((16, n), device="cuda", generator=g) * 512.0


def _rect_chain(tgt0, steps, sync):
    n = tgt0.shape[1]
    tgt = torch.empty_like(tgt0)
    H = torch.empty((9, n), device="cuda")
    G = torch.empty((8, n), device="cuda")
    out = []
    for i in range(steps):
        torch.add(tgt0, 0.25 * i, out=tgt)            # torch kernel writes the input
        if sync:
            torch.cuda.synchronize()
        _lib.aca_rect_solve(tgt, RECT, H)             # reads it, writes H
        if sync:
            torch.cuda.synchronize()
        _lib.aca_rect_backward(tgt, RECT, H, G)       # reads H (read-after-write on the forward)
        if sync:
            torch.cuda.synchronize()
        _lib.aca_rect_solve(tgt, RECT, H)             # rewrites H (write-after-read on the backward)
        if sync:
            torch.cuda.synchronize()
        out.append(torch.cat([H, G]))                 # torch kernel reads both
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("n", [1, 1000, 65536 + 37, (1 << 18) + 8])
def test_rect_forward_backward_chain_matches_synchronised_calls(n):
    # below 2^18 sets the scalar kernels run, from 2^18 the vectorised ones
    g = torch.Generator(device="cuda").manual_seed(n)
    tgt0 = (torch.rand((8, n), device="cuda", generator=g) - 0.5) * 40.0
    a = _rect_chain(tgt0, 6, sync=False)
    b = _rect_chain(tgt0, 6, sync=True)
    for x, y in zip(a, b):
        assert _same(x, y)


def _aca_chain(pts0, steps, sync, stream):
    n = pts0.shape[1]
    with torch.cuda.stream(stream):
        pts = torch.empty_like(pts0)
        H = torch.empty((9, n), device="cuda")
        G = torch.empty((8, n), device="cuda")
        out = []
        for i in range(steps):
            torch.mul(pts0, 1.0 + 0.01 * i, out=pts)
            if sync:
                torch.cuda.synchronize()
            _lib.aca_solve(pts, H)                    # writes H
            if sync:
                torch.cuda.synchronize()
            _lib.aca_backward(pts, H, G)              # reads H as the upstream gradient
            if sync:
                torch.cuda.synchronize()
            _lib.sks_solve(pts, H)                    # rewrites H after the backward read it
            if sync:
                torch.cuda.synchronize()
            out.append(torch.cat([H, G]))
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("n", [3, 4096, (1 << 18) + 4])
def test_solve_backward_chain_on_a_side_stream_matches_synchronised_calls(n):
    pts0 = _sets(n, 7 + n)
    s = torch.cuda.Stream()
    a = _aca_chain(pts0, 5, False, s)
    b = _aca_chain(pts0, 5, True, s)
    for x, y in zip(a, b):
        assert _same(x, y)


def test_chain_captured_in_a_cuda_graph_matches_eager_calls():
    # the same chain captured once and replayed: programmatic edges inside
    # the graph keep the order
    n = 50000
    pts0 = _sets(n, 11)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pts = torch.empty_like(pts0)
        H = torch.empty((9, n), device="cuda")
        G = torch.empty((8, n), device="cuda")
        res = torch.empty((17, n), device="cuda")

        def step():
            torch.mul(pts0, 1.5, out=pts)
            _lib.aca_solve(pts, H, stream=s)
            _lib.aca_backward(pts, H, G, stream=s)
            _lib.aca_solve(pts, H, norm=_lib.ACA_NORM_FROB, stream=s)
            res[:9].copy_(H)
            res[9:].copy_(G)

        step()
    torch.cuda.synchronize()
    ref = res.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            step()
    for _ in range(3):
        res.zero_()
        H.zero_()
        G.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert _same(res, ref)
