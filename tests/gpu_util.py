"""Shared helpers of the GPU parity tests (comparison metrics only)."""
import numpy as np
import torch

# FP32 gate on the homography, relative to |H|_F with both sides scaled to
# unit Frobenius norm and the GPU sign aligned to the oracle's.
H_TOL = 1e-4


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
