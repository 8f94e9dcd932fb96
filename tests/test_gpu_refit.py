"""aca_refit (refit on all inliers: normalised DLT, then Levenberg-Marquardt;
the global optimisation of Sec. 6.2, stage 5) against the float64 oracle.

Gate (entry-wise, unit Frobenius, sign aligned): |H_gpu - H_ref| <=
max(REFIT_FLOOR, REFIT_C * movement), where movement is how far the oracle's
own H moves when every input coordinate is moved by 16 units of 2^-24
(oracle.refit_tolerance).  The FP32 pass is backward stable with errors of a
few units of 2^-24 in the normalised coordinates, so it must land within a
small multiple of that movement.  Problems whose movement is at most
H_TOL / REFIT_C must also meet H_TOL.  LM results must also be optimal: the
float64 reprojection cost at H_gpu may exceed the oracle's optimum by a
relative 1e-6 at most.  n_used is exact."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from paper_2402_18008_gb300 import _lib, api
from paper_2402_18008_gb300._lib import AcaError
from tests.gpu_util import H_TOL, cuda, unit_aligned_err

pytestmark = pytest.mark.gpu
REFIT_C = 4.0
REFIT_FLOOR = 1e-6
COST_REL = 1e-6


def _gpu_refit(corr, offsets, mask, lm_iters):
    c, o = cuda(corr), cuda(offsets)
    m = None if mask is None else cuda(mask.astype(np.uint8))
    H, n_used, rms = api.refit(c, o, m, lm_iters)
    torch.cuda.synchronize()
    return H.cpu().numpy().astype(np.float64), n_used.cpu().numpy(), rms.cpu().numpy()


def _gate(H, corr, offsets, mask, oracle_iters, label):
    ref, used = oracle.refit(corr, offsets, mask, oracle_iters)
    mv = oracle.refit_tolerance(corr, offsets, mask, oracle_iters)
    ok = used >= 4
    err = unit_aligned_err(H[ok], ref[ok])
    bound = np.maximum(REFIT_FLOOR, REFIT_C * mv[ok])
    well = REFIT_C * mv[ok] <= H_TOL
    summary = dict(problems=int(ok.sum()), max_err=float(err.max()), median_err=float(np.median(err)),
                   well=int(well.sum()), max_err_well=float(err[well].max()) if well.any() else 0.0,
                   worst_ratio=float(np.max(err / bound)), max_movement=float(mv[ok].max()))
    print(label, summary)
    assert np.all(err <= bound), summary
    assert summary["max_err_well"] <= H_TOL, summary
    return ref, used


def _cost_gate(H, ref, corr, offsets, mask, label):
    cg = oracle.reprojection_cost(H, corr, offsets, mask)
    cr = oracle.reprojection_cost(ref, corr, offsets, mask)
    ok = cr > 0
    excess = (cg[ok] - cr[ok]) / cr[ok]
    print(label, "max relative cost excess", float(excess.max()))
    assert np.all(excess <= COST_REL)
    return cg


@pytest.fixture(scope="module")
def batch48():
    rb = workloads.ransac_batch(P=48, seed=3, n_max=3000)
    return rb


def test_refit_dlt_matches_oracle(batch48):
    rb = batch48
    H, n_used, rms = _gpu_refit(rb.corr, rb.offsets, rb.is_inlier, 0)
    ref, used = _gate(H, rb.corr, rb.offsets, rb.is_inlier, 0, "refit DLT (48 problems)")
    assert np.array_equal(n_used, used)
    # rms: the RMS reprojection error of the returned H (oracle cost at H_gpu)
    cg = oracle.reprojection_cost(H, rb.corr, rb.offsets, rb.is_inlier)
    assert np.allclose(rms, np.sqrt(cg / used), rtol=1e-4)


@pytest.mark.parametrize("iters", [10, 50])
def test_refit_lm_matches_converged_oracle(batch48, iters):
    rb = batch48
    H, n_used, rms = _gpu_refit(rb.corr, rb.offsets, rb.is_inlier, iters)
    ref, used = _gate(H, rb.corr, rb.offsets, rb.is_inlier, 200, f"refit LM {iters} steps (48 problems)")
    assert np.array_equal(n_used, used)
    cg = _cost_gate(H, ref, rb.corr, rb.offsets, rb.is_inlier, f"LM {iters}")
    assert np.allclose(rms, np.sqrt(cg / used), rtol=1e-4)
    # LM never ends above its DLT start
    Hd, _, _ = _gpu_refit(rb.corr, rb.offsets, rb.is_inlier, 0)
    cd = oracle.reprojection_cost(Hd, rb.corr, rb.offsets, rb.is_inlier)
    assert np.all(cg <= cd * (1 + 1e-6))


def test_refit_full_size_512_pairs():
    # the batched-RANSAC workload at full size (512 pairs, N log-uniform in
    # [200, 8000]); masks = the generated inliers; the launches the bench
    # times (10 LM steps, and the DLT alone)
    rb = workloads.ransac_batch(P=512, seed=0)
    H, n_used, rms = _gpu_refit(rb.corr, rb.offsets, rb.is_inlier, 10)
    ref, used = _gate(H, rb.corr, rb.offsets, rb.is_inlier, 200, "refit LM 10 steps (512 pairs)")
    assert np.array_equal(n_used, used)
    _cost_gate(H, ref, rb.corr, rb.offsets, rb.is_inlier, "512 pairs")
    Hd, nd, _ = _gpu_refit(rb.corr, rb.offsets, rb.is_inlier, 0)
    _gate(Hd, rb.corr, rb.offsets, rb.is_inlier, 0, "refit DLT (512 pairs)")
    assert np.array_equal(nd, used)


def test_refit_dlt_on_contaminated_sets():
    # the DLT over every point of pairs with 10-60 % outliers (mask = None):
    # the smallest eigenvalue of the normal matrix is no longer small against
    # the next one, so the eigenvector refinement contracts slowly; the
    # result must still meet the gate
    probs = [workloads.ransac_problem(n, eps, 1.0, seed=40 + i)
             for i, (n, eps) in enumerate([(300, 0.9), (800, 0.7), (1500, 0.55), (4000, 0.4), (6000, 0.6)])]
    corr = np.concatenate([q.corr for q in probs])
    offsets = np.concatenate([[0], np.cumsum([len(q.corr) for q in probs])]).astype(np.int64)
    allpts = np.ones(len(corr), bool)
    H, n_used, _ = _gpu_refit(corr, offsets, None, 0)
    ref, used = _gate(H, corr, offsets, allpts, 0, "refit DLT, contaminated (5 problems)")
    assert np.array_equal(n_used, used)
    H10, _, _ = _gpu_refit(corr, offsets, None, 10)
    ref10, _ = _gate(H10, corr, offsets, allpts, 200, "refit LM 10 steps, contaminated (5 problems)")


def test_refit_noise_free_recovers_the_true_map():
    rp = workloads.ransac_problem(500, 0.6, 0.0, seed=31)
    for iters in (0, 10):
        H, n_used, _ = _gpu_refit(rp.corr, np.array([0, 500]), rp.is_inlier, iters)
        Ht = oracle.normalize_frob(rp.H_true.reshape(9))
        assert n_used[0] == rp.is_inlier.sum()
        assert unit_aligned_err(H, Ht)[0] < 2e-5


def test_refit_edge_cases():
    rp = workloads.ransac_problem(400, 0.8, 1.0, seed=32)
    c = rp.corr
    # problems: empty, 3 used points, exactly 4, 5, all 400 with no mask below
    sizes = [0, 50, 40, 40, 270]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    mask = rp.is_inlier[:400].copy()
    seg = [np.arange(offsets[i], offsets[i + 1]) for i in range(5)]
    mask[seg[1]] = False
    mask[seg[1][np.flatnonzero(rp.is_inlier[seg[1]])[:3]]] = True
    for i, k in ((2, 4), (3, 5)):
        keep = seg[i][np.flatnonzero(rp.is_inlier[seg[i]])[:k]]
        mask[seg[i]] = False
        mask[keep] = True
    H, n_used, rms = _gpu_refit(c, offsets, mask, 10)
    ref, used = oracle.refit(c, offsets, mask, 200)
    assert np.array_equal(n_used, used)
    assert list(used[:4]) == [0, 3, 4, 5]
    assert np.all(H[:2] == 0) and np.all(rms[:2] == 0)
    # 4 points: the exact interpolant (the minimal solution), residual ~ 0
    assert unit_aligned_err(H[2:3], ref[2:3])[0] < 1e-4 and rms[2] < 1e-3
    assert unit_aligned_err(H[3:], ref[3:]).max() < 1e-4
    # mask = None uses every point
    Ha, na, _ = _gpu_refit(c, offsets, None, 10)
    refa, useda = oracle.refit(c, offsets, np.ones(400, bool), 200)
    assert np.array_equal(na, useda)
    assert unit_aligned_err(Ha[1:], refa[1:]).max() < 1e-3


def test_refit_is_deterministic_and_validates_arguments(batch48):
    rb = batch48
    a = _gpu_refit(rb.corr, rb.offsets, rb.is_inlier, 10)
    b = _gpu_refit(rb.corr, rb.offsets, rb.is_inlier, 10)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    c, o = cuda(rb.corr), cuda(rb.offsets)
    H = torch.empty((48, 9), device="cuda")
    with pytest.raises(AcaError):
        _lib.aca_refit(c, o, H, lm_iters=-1)
    with pytest.raises(AcaError):
        _lib.aca_refit(c, o, H, lm_iters=10001)
    flat = torch.zeros(4 * 100 + 1, device="cuda")
    mis = flat[1:].view(100, 4)          # 4-byte offset: misaligned corr
    with pytest.raises(AcaError):
        _lib.aca_refit(mis, cuda(np.array([0, 100])), torch.empty((1, 9), device="cuda"))
    _lib.aca_refit(c, cuda(np.array([0], np.int64)), H)       # P = 0 is a no-op
    torch.cuda.synchronize()


def test_ransac_plan_with_refit_in_a_cuda_graph():
    rb = workloads.ransac_batch(P=32, seed=8, n_max=2000, cap=1024)
    tot = int(rb.n_hyp.sum())
    plan = api.RansacPlan(cuda(rb.corr), cuda(rb.offsets), cuda(rb.n_hyp), 3.0, 5, tot, refit_iters=10)
    eager = plan.run()
    e = {k: getattr(eager, k).clone() for k in ("best_H", "best_count", "inlier_mask", "refit_H", "refit_rms")}
    plan.capture()
    rep = plan.replay()
    torch.cuda.synchronize()
    for k, v in e.items():
        assert torch.equal(v, getattr(rep, k)), k
    # the refit stage is aca_refit on the RANSAC inlier mask
    H2 = torch.empty_like(rep.refit_H)
    _lib.aca_refit(plan.corr, plan.offsets, H2, mask=rep.inlier_mask, lm_iters=10)
    torch.cuda.synchronize()
    assert torch.equal(H2, rep.refit_H)
    # every masked point is within 3 px of the RANSAC H; the refit minimises the cost
    assert float(rep.refit_rms.max()) < 3.0


def test_refit_many_small_problems_beyond_the_ordering_limit():
    # more problems than the longest-first ordering ranks (natural order
    # above 65536): per-problem results do not depend on the order, so a
    # subset refit alone must give bit-identical outputs
    P, k = 70000, 6
    rp = workloads.ransac_problem(P * k, 1.0, 0.5, seed=33)
    corr = rp.corr
    offsets = np.arange(P + 1, dtype=np.int64) * k
    H, n_used, rms = _gpu_refit(corr, offsets, None, 10)
    assert np.all(n_used == k)
    sub = 1000
    Hs, ns, rs = _gpu_refit(corr[:sub * k], offsets[:sub + 1], None, 10)
    assert np.array_equal(Hs, H[:sub]) and np.array_equal(rs, rms[:sub])
    idx = np.arange(0, P, 7001)
    sel = np.concatenate([np.arange(i * k, (i + 1) * k) for i in idx])
    _gate(H[idx], corr[sel], np.arange(idx.size + 1) * k, np.ones(sel.size, bool), 200, "70000 problems, sampled")


def test_refit_sizes_around_the_shared_copy():
    # the refit keeps the first points of each pair in shared memory (4096 on
    # GB300, fewer where an SM has less of it) and reads the rest from global
    # memory on every pass: pairs just below, at and above the copy's size
    sizes = [3839, 3840, 3841, 4095, 4096, 4097, 9001]
    probs = [workloads.ransac_problem(n, 0.7, 1.0, seed=60 + i) for i, n in enumerate(sizes)]
    corr = np.concatenate([q.corr for q in probs])
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    mask = np.concatenate([q.is_inlier for q in probs])
    for iters, oracle_iters in ((0, 0), (10, 200)):
        H, n_used, _ = _gpu_refit(corr, offsets, mask, iters)
        ref, used = _gate(H, corr, offsets, mask, oracle_iters, f"refit {iters} LM steps, pairs around the copy size")
        assert np.array_equal(n_used, used)
