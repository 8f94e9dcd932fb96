"""Pins of the oracle's online adaptive stop (Sec. 6.2: the loop count follows
from the inlier ratio at 99% confidence that one 4-point sample is all
inliers, capped): the paper's printed sample numbers, the stop conditions
restated with numpy prefix maxima, monotonicity and special cases."""
import os

import numpy as np

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table8():
    rows, cap = [], None
    for line in open(os.path.join(GOLDEN, "table8_sample_counts.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "CAP":
            cap = (int(line[1]), int(line[2]))
        else:
            rows.append((int(line[0]), int(line[1])))
    return rows, cap


def test_required_hypotheses_reproduce_the_papers_sample_numbers():
    rows, cap = _table8()
    N = 100000
    for samples, outlier_pct in rows[1:]:
        # whole-percent outlier ratios in the paper: bracket by +-0.5 %
        c_hi = int(round((1 - (outlier_pct - 0.5) / 100) * N))
        c_lo = int(round((1 - (outlier_pct + 0.5) / 100) * N))
        assert oracle.adaptive_k(c_hi, N, 10**9) <= samples <= oracle.adaptive_k(c_lo, N, 10**9)
    k26 = oracle.adaptive_k(cap[1], 100, 10**9)
    assert abs(k26 - cap[0]) / cap[0] < 0.05          # "roughly 26%" for the 1000-loop cap
    assert oracle.adaptive_k(N, N, 1000) == 1          # all inliers: one sample suffices
    assert oracle.adaptive_k(0, N, 1000) == 1000 and oracle.adaptive_k(-1, N, 1000) == 1000
    assert oracle.adaptive_k(1, N, 1000) == 1000       # w^4 = 1e-20 vanishes next to 1: the cap


def test_required_hypotheses_do_not_increase_with_the_count():
    N = 3000
    ks = [oracle.adaptive_k(c, N, 16384) for c in range(0, N + 1, 7)]
    assert all(a >= b for a, b in zip(ks, ks[1:]))


def _stop_conditions(counts, N, i_star):
    # B(i) = max of counts[0..i-1]; the loop stops at the first i with
    # i >= K(B(i)), or at the cap
    k = len(counts)
    B = np.maximum.accumulate(np.r_[-1, counts])[:k + 1]        # B[i] for i = 0..k
    K = np.array([oracle.adaptive_k(int(b), N, k) for b in B])
    stop_ok = i_star == k or i_star >= K[i_star]
    earlier = all(i < K[i] for i in range(1, i_star))
    return stop_ok and earlier and 1 <= i_star <= k


def test_stop_index_satisfies_the_stop_conditions():
    rng = np.random.default_rng(0)
    for trial in range(300):
        N = int(rng.integers(8, 3000))
        k = int(rng.integers(1, 600))
        eps = rng.uniform(0.05, 1.0)
        counts = rng.binomial(N, eps, size=k) * (rng.random(k) < 0.3)
        counts[rng.random(k) < 0.05] = -1                   # degenerate samples
        i_star = oracle.adaptive_stop(counts, N)
        assert _stop_conditions(counts.astype(np.int64), N, i_star), (trial, i_star)


def test_stop_index_never_increases_with_larger_counts_and_special_cases():
    rng = np.random.default_rng(1)
    for _ in range(100):
        N, k = 2000, 500
        counts = rng.integers(-1, N // 2, size=k)
        bump = counts + rng.integers(0, 50, size=k)
        assert oracle.adaptive_stop(bump, N) <= oracle.adaptive_stop(counts, N)
    assert oracle.adaptive_stop(np.zeros(700, np.int32), 100) == 700       # never a valid count
    assert oracle.adaptive_stop(np.full(700, 100, np.int32), 100) == 1      # all inliers at once
    assert oracle.adaptive_stop(np.array([-1, -1, 100], np.int32), 100) == 3


def test_adaptive_ransac_stops_early_on_clean_data_and_matches_fixed_ransac():
    rp = workloads.ransac_problem(400, 0.8, 1.0, seed=41)
    r = oracle.ransac_adaptive(rp.corr, [0, 400], [4000], 3.0, 9)
    ne = int(r["n_eval"][0])
    assert ne == oracle.adaptive_stop(r["hyp_counts"], 400)
    assert 1 <= ne < 100                                  # eps = 0.8: K(0.8) = 9 at best
    f = oracle.ransac(rp.corr, [0, 400], [ne], 3.0, 9)
    assert f["best_hyp"][0] == r["best_hyp"][0] and f["best_count"][0] == r["best_count"][0]
    assert np.array_equal(f["best_H"], r["best_H"])
    # pure outliers: no count reaches a usable ratio, the cap is reached
    rq = workloads.ransac_problem(300, 0.0, 1.0, seed=42)
    r2 = oracle.ransac_adaptive(rq.corr, [0, 300], [500], 3.0, 9)
    assert r2["n_eval"][0] == 500
