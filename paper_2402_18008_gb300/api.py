"""Convenience layer over the C ABI: allocates outputs and workspaces with
torch, keeps RANSAC launch plans and CUDA graphs.  No arithmetic of the
method runs here; every step is a kernel of the CUDA library.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import _lib
from ._lib import ACA_NORM_NONE, RansacParams

_SOLVERS = {"aca": _lib.aca_solve, "sks": _lib.sks_solve}


def _require_cuda(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must live on a CUDA device (the library has no CPU path)")


def solve(pts: torch.Tensor, norm: int = ACA_NORM_NONE, solver: str = "aca", with_flags: bool = False,
          n: int | None = None, out: torch.Tensor | None = None, flags_out: torch.Tensor | None = None):
    """Batched minimal solve.  pts: (16, ld) float32 CUDA planes.  Returns H
    (9, ld) and, if requested, per-set flags (ld,) uint8."""
    _require_cuda(pts, "pts")
    ld = pts.stride(0)
    H = out if out is not None else torch.empty((9, ld), dtype=torch.float32, device=pts.device)
    fl = None
    if with_flags:
        fl = flags_out if flags_out is not None else torch.empty(ld, dtype=torch.uint8, device=pts.device)
    _SOLVERS[solver](pts, H, fl, n=pts.shape[1] if n is None else n, norm=norm)
    return (H, fl) if with_flags else H


class PinnedSolver:
    """ACA on page-locked host planes through device staging buffers: the
    sets are copied to the device chunk by chunk (one cudaMemcpyAsync per
    plane segment), solved there, and the homographies copied back, with
    `streams` chunks in flight on streams of their own so that the two copy
    directions and the solves overlap.  The alternative to calling
    aca_solve on the host buffers directly (zero-copy: the kernel itself
    reads and writes over the host link).  Staging buffers are allocated
    once, here: streams x 25 planes x chunk floats."""

    def __init__(self, device, chunk: int = 1 << 22, streams: int = 3):
        self.chunk = int(chunk)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(streams)]
        self.pts = [torch.empty((16, self.chunk), dtype=torch.float32, device=device) for _ in range(streams)]
        self.H = [torch.empty((9, self.chunk), dtype=torch.float32, device=device) for _ in range(streams)]

    def __call__(self, pts_h: torch.Tensor, H_h: torch.Tensor, n: int | None = None):
        if not (pts_h.is_pinned() and H_h.is_pinned()):
            raise ValueError("pts_h and H_h must be page-locked host tensors")
        n = pts_h.shape[1] if n is None else int(n)
        cur = torch.cuda.current_stream()
        for s in self.streams:
            s.wait_stream(cur)
        for j, a in enumerate(range(0, n, self.chunk)):
            c = min(self.chunk, n - a)
            k = j % len(self.streams)
            s, dp, dh = self.streams[k], self.pts[k], self.H[k]
            with torch.cuda.stream(s):
                for r in range(16):
                    dp[r, :c].copy_(pts_h[r, a:a + c], non_blocking=True)
                _lib.aca_solve(dp, dh, None, n=c, stream=s)
                for r in range(9):
                    H_h[r, a:a + c].copy_(dh[r, :c], non_blocking=True)
        for s in self.streams:
            cur.wait_stream(s)


def shard_ranges(costs, world: int):
    """Split problems 0..P-1 over `world` ranks as contiguous ranges of about
    equal total cost (e.g. hypotheses x points per RANSAC problem): rank r
    takes [start_r, start_{r+1}), start_r the first problem whose cost prefix
    reaches r / world of the total.  Contiguous ranges keep the sampling
    streams: a rank runs its range with problem_base = start_r and gets the
    same results as one run over all problems.  Host logic only."""
    import numpy as np
    c = np.asarray(costs, dtype=np.float64)
    P = c.size
    if world < 1:
        raise ValueError("world must be >= 1")
    pre = np.concatenate([[0.0], np.cumsum(c)])
    tot = pre[-1]
    starts = [0] + [int(np.searchsorted(pre[1:], tot * r / world, side="left")) + 1 if tot > 0 else (P * r) // world
                    for r in range(1, world)] + [P]
    for r in range(1, world + 1):                      # non-decreasing, within [0, P]
        starts[r] = min(P, max(starts[r], starts[r - 1]))
    return [(starts[r], starts[r + 1]) for r in range(world)]


def rect_solve(tgt: torch.Tensor, rect, out: torch.Tensor | None = None):
    """Rectangle-source ACA (Eq. 42).  tgt: (8, ld) float32; rect = (x0, y0, w, r)."""
    _require_cuda(tgt, "tgt")
    H = out if out is not None else torch.empty((9, tgt.stride(0)), dtype=torch.float32, device=tgt.device)
    _lib.aca_rect_solve(tgt, rect, H)
    return H


def affine_solve(pts: torch.Tensor, norm: int = ACA_NORM_NONE, n: int | None = None,
                 out: torch.Tensor | None = None):
    """3-point affine maps (Eq. 38).  pts: (12, ld) float32 planes M1 N1 P1 M2
    N2 P2 (x, y each).  Returns H (9, ld)."""
    _require_cuda(pts, "pts")
    H = out if out is not None else torch.empty((9, pts.stride(0)), dtype=torch.float32, device=pts.device)
    _lib.aca_affine_solve(pts, H, n=pts.shape[1] if n is None else n, norm=norm)
    return H


def to_planes(src: torch.Tensor, tgt: torch.Tensor, ld: int | None = None) -> torch.Tensor:
    """(B, 4, 2) source and target corners (M, N, P, Q order) -> (16, ld) planes."""
    B = src.shape[0]
    ld = B if ld is None else ld
    pts = torch.zeros((16, ld), dtype=torch.float32, device=src.device)
    pts[:8, :B] = src.reshape(B, 8).t()
    pts[8:, :B] = tgt.reshape(B, 8).t()
    return pts


def planes_to_mats(H: torch.Tensor, n: int) -> torch.Tensor:
    """(9, ld) planes -> (n, 3, 3)."""
    return H[:, :n].t().reshape(n, 3, 3)


@dataclass
class RansacResult:
    best_H: torch.Tensor      # (P, 9) float32, unit Frobenius, sign fixed
    best_count: torch.Tensor  # (P,) int32
    best_hyp: torch.Tensor    # (P,) int32
    hyp_counts: torch.Tensor | None
    inlier_mask: torch.Tensor | None
    n_evaluated: torch.Tensor | None = None  # (P,) hypotheses before the online stop (adaptive plans)
    refit_H: torch.Tensor | None = None     # (P, 9) after the refit on all inliers
    refit_rms: torch.Tensor | None = None   # (P,) RMS reprojection error (px) of refit_H


class RansacPlan:
    """Buffers and launch parameters for repeated ransac_aca calls on one
    batch layout (P problems, total_hyps hypotheses, total points).

    With ``confidence`` set, ``n_hyp`` is the cap per problem and the loop
    stops online (ransac_aca_adaptive): hypothesis h is evaluated only while
    h < K(best count so far) at that confidence.

    ``run()`` enqueues one full RANSAC (prep, scoring, argmax) on the current
    stream, followed, when ``refit_iters`` is not None, by the refit of each
    best H on all of its inliers (aca_refit with that many LM steps);
    ``capture()`` records it into a CUDA graph and ``replay()`` launches that
    graph.
    """

    def __init__(self, corr: torch.Tensor, offsets: torch.Tensor, n_hyp: torch.Tensor, threshold_px: float,
                 seed: int, total_hyps: int, problem_base: int = 0, block_warps: int = 0,
                 hyps_per_thread: int = 0, tile_points: int = 0, grid_blocks: int = 0,
                 want_counts: bool = False, want_mask: bool = False, refit_iters: int | None = None,
                 confidence: float | None = None):
        _require_cuda(corr, "corr")
        want_mask = want_mask or refit_iters is not None
        self.confidence = confidence
        self.total_hyps = int(total_hyps)
        dev = corr.device
        self.corr, self.offsets, self.n_hyp = corr, offsets, n_hyp
        self.P = n_hyp.numel()
        self.params = RansacParams(threshold_px=float(threshold_px), problem_base=int(problem_base),
                                   seed=int(seed), block_warps=int(block_warps),
                                   hyps_per_thread=int(hyps_per_thread), grid_blocks=int(grid_blocks),
                                   tile_points=int(tile_points))
        ws = (_lib.ransac_aca_adaptive_workspace_size(self.P, int(total_hyps)) if confidence is not None
              else _lib.ransac_aca_workspace_size(self.P, int(total_hyps)))
        # zeroed: the one-launch path of small batches needs its done counter
        # at zero before the first call (every call leaves it zero)
        self.workspace = torch.zeros(max(ws, 256), dtype=torch.uint8, device=dev)
        self.best_H = torch.empty((self.P, 9), dtype=torch.float32, device=dev)
        self.best_count = torch.empty(self.P, dtype=torch.int32, device=dev)
        self.best_hyp = torch.empty(self.P, dtype=torch.int32, device=dev)
        self.hyp_counts = torch.empty(max(int(total_hyps), 1), dtype=torch.int32, device=dev) if want_counts else None
        self.inlier_mask = torch.empty(max(corr.shape[0], 1), dtype=torch.uint8, device=dev) if want_mask else None
        self.n_evaluated = torch.empty(self.P, dtype=torch.int32, device=dev) if confidence is not None else None
        self.refit_iters = refit_iters
        self.refit_H = torch.empty((self.P, 9), dtype=torch.float32, device=dev) if refit_iters is not None else None
        self.refit_rms = torch.empty(self.P, dtype=torch.float32, device=dev) if refit_iters is not None else None
        self.graph = None

    def run(self) -> RansacResult:
        if self.confidence is not None:
            _lib.ransac_aca_adaptive(self.corr, self.offsets, self.n_hyp, self.total_hyps, self.params,
                                     self.confidence, self.best_H, self.best_count, self.best_hyp, self.workspace,
                                     n_evaluated=self.n_evaluated, hyp_counts=self.hyp_counts,
                                     inlier_mask=self.inlier_mask)
        else:
            _lib.ransac_aca(self.corr, self.offsets, self.n_hyp, self.params, self.best_H, self.best_count,
                            self.best_hyp, self.workspace, hyp_counts=self.hyp_counts, inlier_mask=self.inlier_mask)
        if self.refit_iters is not None:
            _lib.aca_refit(self.corr, self.offsets, self.refit_H, mask=self.inlier_mask, lm_iters=self.refit_iters,
                           rms=self.refit_rms)
        return self.result()

    def capture(self, warmup: int = 1) -> "RansacPlan":
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.run()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return self

    def replay(self) -> RansacResult:
        self.graph.replay()
        return self.result()

    def result(self) -> RansacResult:
        return RansacResult(self.best_H, self.best_count, self.best_hyp, self.hyp_counts, self.inlier_mask,
                            self.n_evaluated, self.refit_H, self.refit_rms)


def ransac(corr: torch.Tensor, offsets: torch.Tensor, n_hyp: torch.Tensor, threshold_px: float, seed: int,
           total_hyps: int | None = None, want_counts: bool = False, want_mask: bool = False,
           refit_iters: int | None = None, confidence: float | None = None, **tuning) -> RansacResult:
    """One-shot RANSAC over CSR problems (see include/aca.h, ransac_aca; with
    `confidence`, ransac_aca_adaptive and n_hyp as the caps), optionally
    followed by the refit on all inliers (refit_iters LM steps)."""
    if total_hyps is None:
        total_hyps = int(n_hyp.sum().item())
    plan = RansacPlan(corr, offsets, n_hyp, threshold_px, seed, total_hyps, want_counts=want_counts,
                      want_mask=want_mask, refit_iters=refit_iters, confidence=confidence, **tuning)
    return plan.run()


def refit(corr: torch.Tensor, offsets: torch.Tensor, mask: torch.Tensor | None = None, lm_iters: int = 10):
    """Homography per problem from all masked points: normalised DLT, then
    lm_iters Levenberg-Marquardt steps (include/aca.h, aca_refit).  Returns
    (H (P, 9), n_used (P,), rms (P,))."""
    _require_cuda(corr, "corr")
    P = offsets.numel() - 1
    H = torch.empty((P, 9), dtype=torch.float32, device=corr.device)
    n_used = torch.empty(P, dtype=torch.int32, device=corr.device)
    rms = torch.empty(P, dtype=torch.float32, device=corr.device)
    _lib.aca_refit(corr, offsets, H, mask=mask, lm_iters=lm_iters, n_used=n_used, rms=rms)
    return H, n_used, rms
