"""ransac_aca_noalloc: the RANSAC entry point for callers that may not
allocate device memory (a framework plugin whose host owns all device memory,
a loop in which an allocation is not allowed, a fixed memory budget).  It
must give exactly what ransac_aca gives with a caller workspace, on
consecutive calls that reuse the library's built-in scratch.

The file name sorts after every other test file, so that a run stopping at
its first failure (pytest -x) has run all the other tests before this
optional entry point is exercised; it passes alone in a fresh process and
after the other tests."""
import numpy as np
import pytest
import torch

import workloads
from paper_2402_18008_gb300 import _lib, api

pytestmark = pytest.mark.gpu


def _inputs(seed, P, n_max, cap):
    rb = workloads.ransac_batch(P=P, seed=seed, n_max=n_max, cap=cap)
    dev = torch.device("cuda")
    return (torch.from_numpy(rb.corr).to(dev), torch.from_numpy(rb.offsets).to(dev),
            torch.from_numpy(rb.n_hyp).to(dev), int(rb.n_hyp.sum()), rb.corr.shape[0])


def _with_workspace(corr, off, k, tot, seed):
    plan = api.RansacPlan(corr, off, k, 3.0, seed, tot, want_counts=True, want_mask=True)
    r = plan.run()
    torch.cuda.synchronize()
    return {n: getattr(r, n).cpu().numpy() for n in ("best_H", "best_count", "best_hyp", "hyp_counts",
                                                       "inlier_mask")}


def _no_alloc(corr, off, k, tot, seed, total_points):
    P = k.numel()
    dev = corr.device
    out = dict(best_H=torch.full((P, 9), -7.0, device=dev),
               best_count=torch.full((P,), -7, dtype=torch.int32, device=dev),
               best_hyp=torch.full((P,), -7, dtype=torch.int32, device=dev),
               hyp_counts=torch.full((tot,), -7, dtype=torch.int32, device=dev),
               inlier_mask=torch.full((total_points,), 7, dtype=torch.uint8, device=dev))
    params = _lib.RansacParams(threshold_px=3.0, seed=seed)
    _lib.ransac_aca_noalloc(corr, off, k, tot, params, out["best_H"], out["best_count"], out["best_hyp"],
                            hyp_counts=out["hyp_counts"], inlier_mask=out["inlier_mask"])
    torch.cuda.synchronize()
    return {n: v.cpu().numpy() for n, v in out.items()}


def test_no_alloc_entry_point_matches_workspace_entry_point_on_two_consecutive_calls():
    # two different batches in a row: the second call finds the first call's
    # leftovers in the shared scratch and must not be affected by them
    # (the third call has at most 8 problems: the one-launch path, whose done
    # counter must survive the larger calls that shared the scratch before it)
    for seed, P, n_max, cap in ((31, 40, 3000, 2048), (32, 24, 6000, 4096), (37, 4, 3000, 2048)):
        corr, off, k, tot, npts = _inputs(seed, P, n_max, cap)
        ref = _with_workspace(corr, off, k, tot, seed)
        got = _no_alloc(corr, off, k, tot, seed, npts)
        for name in ref:
            assert np.array_equal(got[name], ref[name]), (seed, name)
        assert np.all(got["best_hyp"] >= 0)


def test_no_alloc_small_batch_clears_its_counts_in_the_set_up_kernel():
    # at most 65536 hypotheses: the counts are cleared by the set-up kernel
    # itself rather than by a separate launch; run it after a larger call so
    # that the shared scratch holds non-zero leftovers
    for seed, P, n_max, cap in ((34, 30, 4000, 4096), (35, 12, 1500, 256)):
        corr, off, k, tot, npts = _inputs(seed, P, n_max, cap)
        ref = _with_workspace(corr, off, k, tot, seed)
        got = _no_alloc(corr, off, k, tot, seed, npts)
        for name in ref:
            assert np.array_equal(got[name], ref[name]), (seed, name)
    assert tot <= 65536


def test_no_alloc_total_hyps_below_the_sum_of_n_hyp_is_caught_on_the_device():
    # total_hyps understating sum(n_hyp): nothing is scored, every best_hyp
    # is -2, and nothing is written past the caller's hyp_counts
    corr, off, k, tot, npts = _inputs(36, 10, 800, 300)
    short = tot - 100
    P = k.numel()
    dev = corr.device
    counts = torch.full((short + 64,), -7, dtype=torch.int32, device=dev)    # 64 canaries after the buffer
    best_hyp = torch.full((P,), -7, dtype=torch.int32, device=dev)
    best_count = torch.full((P,), -7, dtype=torch.int32, device=dev)
    params = _lib.RansacParams(threshold_px=3.0, seed=36)
    _lib.ransac_aca_noalloc(corr, off, k, short, params, torch.zeros((P, 9), device=dev), best_count, best_hyp,
                            hyp_counts=counts[:short])
    torch.cuda.synchronize()
    assert np.all(best_hyp.cpu().numpy() == -2)
    assert np.all(best_count.cpu().numpy() == 0)
    assert np.all(counts[short:].cpu().numpy() == -7)


def test_no_alloc_rejects_requests_beyond_the_built_in_scratch():
    corr, off, k, tot, _ = _inputs(33, 8, 500, 64)
    P = k.numel()
    dev = corr.device
    too_many = _lib.ACA_NOALLOC_SCRATCH_BYTES // 4       # counts alone would fill the scratch
    params = _lib.RansacParams(threshold_px=3.0, seed=1)
    with pytest.raises(_lib.AcaError) as exc:
        _lib.ransac_aca_noalloc(corr, off, k, too_many, params, torch.empty((P, 9), device=dev),
                                torch.empty(P, dtype=torch.int32, device=dev),
                                torch.empty(P, dtype=torch.int32, device=dev))
    assert exc.value.status == -3 and "scratch" in str(exc.value)
