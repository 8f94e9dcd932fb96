"""Shared helpers of the GPU parity tests (comparison metrics only)."""
import numpy as np
import torch

# FP32 gate on the homography, relative to |H|_F with both sides scaled to
# unit Frobenius norm and the GPU sign aligned to the oracle's: the stated
# tolerance 1e-4, widened on a set only where the oracle's first-order bound
# beta on the rounding error of the library's FP32 evaluation order
# (oracle/fp32_bounds.c: every rounding event of that order, each bounded by
# a published rule) exceeds it.  beta is derived from the arithmetic, not
# calibrated; beta^2 allows for the neglected second-order terms.
H_TOL = 1e-4


def bound_gate(err, beta, label=""):
    """Assert err <= max(H_TOL, beta + beta^2) per set; returns a summary."""
    err = np.asarray(err, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    bound = np.maximum(H_TOL, beta + beta * beta)
    within = beta <= H_TOL
    summary = dict(n=int(err.size), bound_below_tol=int(within.sum()),
                   max_err_bound_below_tol=float(err[within].max()) if within.any() else 0.0,
                   max_err_all=float(err.max()), n_above_1e4=int((err > H_TOL).sum()),
                   max_err_over_beta=float(np.max(err / np.maximum(beta, 1e-300))),
                   worst_ratio=float(np.max(err / bound)))
    print(label, summary)
    assert np.all(err <= bound), summary
    return summary


def unit_aligned_err(H_gpu_rows, H_ref_rows):
    """Max |H_gpu/|H_gpu| * s - H_ref/|H_ref||, per row; s = sign of their inner product."""
    a = np.asarray(H_gpu_rows, dtype=np.float64).reshape(-1, 9)
    b = np.asarray(H_ref_rows, dtype=np.float64).reshape(-1, 9)
    a = a / np.linalg.norm(a, axis=1, keepdims=True)
    b = b / np.linalg.norm(b, axis=1, keepdims=True)
    a = a * np.sign(np.sum(a * b, axis=1, keepdims=True))
    return np.abs(a - b).max(axis=1)


def planes_to_rows(H_planes, n):
    return H_planes[:, :n].detach().cpu().numpy().T.astype(np.float64)


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()
