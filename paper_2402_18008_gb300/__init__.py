"""GB300-native batched minimal homography solvers (ACA / SKS of arXiv
2402.18008), fused RANSAC scoring and the ACA backward pass.

The compute path is the CUDA library in ``csrc/`` (sm_103a), reached through
the C ABI declared in ``include/aca.h``; ``_lib`` is its ctypes binding with
the same function names, ``api`` allocates buffers and captures CUDA graphs,
``autograd`` wraps the forward/backward kernels for torch.autograd.
Importing this package loads nothing; the first call loads (and if needed
builds) the shared library and fails loudly without a CUDA device.
"""
from ._lib import (ACA_FLAG_NON_FINITE, ACA_FLAG_OTHER_TRIPLE, ACA_FLAG_SRC_ANCHORS, ACA_FLAG_TGT_ANCHORS,
                   ACA_NORM_FROB, ACA_NORM_H33, ACA_NORM_NONE, AcaError, RansacParams, aca_affine_solve, aca_backward,
                   aca_rect_backward, aca_rect_solve, aca_sample_indices, aca_solve, ransac_aca,
                   ransac_aca_workspace_size, sks_solve)

__all__ = ["aca_solve", "sks_solve", "aca_rect_solve", "aca_affine_solve", "aca_backward", "aca_rect_backward", "ransac_aca",
           "ransac_aca_workspace_size", "aca_sample_indices", "RansacParams", "AcaError", "ACA_NORM_NONE", "ACA_NORM_H33",
           "ACA_NORM_FROB", "ACA_FLAG_SRC_ANCHORS", "ACA_FLAG_TGT_ANCHORS", "ACA_FLAG_OTHER_TRIPLE",
           "ACA_FLAG_NON_FINITE"]
