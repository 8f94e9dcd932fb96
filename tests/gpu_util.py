"""Shared helpers of the GPU parity tests (comparison metrics only)."""
import numpy as np
import torch

# FP32 gate on the homography, relative to |H|_F with both sides scaled to
# unit Frobenius norm and the GPU sign aligned to the oracle's.
H_TOL = 1e-4
# A set is well-conditioned for FP32 when perturbing its 16 input coordinates
# by one FP32 rounding (relative 2^-24) moves the unit-Frobenius H by at most
# H_TOL / KAPPA_C to first order (kappa * u <= 6.25e-6, kappa from the
# oracle).  Well-conditioned sets must meet H_TOL; every other unflagged set
# must meet max(H_TOL, KAPPA_C * kappa * u), a backward-stability bound: the
# FP32 result is as close as FP32 rounding of the inputs alone permits.
KAPPA_C = 16.0
U32 = 2.0 ** -24


def kappa_gate(err, kappa, label=""):
    """Assert the FP32 gate above; returns a summary dict."""
    import oracle  # noqa: F401
    ku = np.asarray(kappa) * U32
    well = KAPPA_C * ku <= H_TOL
    bound = np.maximum(H_TOL, KAPPA_C * ku)
    summary = dict(n=int(err.size), well_conditioned=int(well.sum()),
                   max_err_well=float(err[well].max()) if well.any() else 0.0,
                   max_err_all=float(err.max()), n_above_1e4=int((err > H_TOL).sum()),
                   worst_ratio=float(np.max(err / bound)))
    print(label, summary)
    assert summary["max_err_well"] <= H_TOL, summary
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
