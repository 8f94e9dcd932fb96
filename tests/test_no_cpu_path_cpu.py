"""There is no CPU fallback: every entry of the binding and of the Python API
refuses CPU tensors with an error before anything runs (a page-locked host
tensor is the one exception, for aca_solve, whose kernel then reads it over
the host link)."""
import pytest
import torch

from paper_2402_18008_gb300 import _lib, api


def _cases():
    x16, H = torch.zeros(16, 8), torch.zeros(9, 8)
    corr, off = torch.zeros(8, 4), torch.tensor([0, 8], dtype=torch.int64)
    k = torch.tensor([4], dtype=torch.int32)
    return [
        ("_lib.aca_solve", lambda: _lib.aca_solve(x16, H)),
        ("_lib.sks_solve", lambda: _lib.sks_solve(x16, H)),
        ("_lib.aca_affine_solve", lambda: _lib.aca_affine_solve(torch.zeros(12, 8), H)),
        ("_lib.aca_refit", lambda: _lib.aca_refit(corr, off, torch.zeros(1, 9))),
        ("api.solve", lambda: api.solve(x16)),
        ("api.affine_solve", lambda: api.affine_solve(torch.zeros(12, 8))),
        ("api.ransac", lambda: api.ransac(corr, off, k, 3.0, 0, total_hyps=4)),
        ("api.refit", lambda: api.refit(corr, off, None, 10)),
    ]


@pytest.mark.parametrize("name,call", _cases(), ids=[c[0] for c in _cases()])
def test_cpu_tensors_are_refused(name, call):
    _lib.load()
    with pytest.raises(ValueError, match="CUDA"):
        call()
