"""Pins of the oracle's RANSAC parts: Philox4x32-10 against cuRAND's
implementation of the same published generator, the distinct-index sampler
against a direct remaining-list definition, uniformity, the paper's
sample-count rule (Sec. 6.2, 6.4), and scoring properties that brute force
fixes (noise-free inliers, degenerate problems, ties)."""
import os
import random
import shutil
import subprocess
import tempfile
from collections import Counter

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

_CURAND_PROBE = r"""
#define QUALIFIERS static inline __host__ __device__
#include <curand_philox4x32_x.h>
#include <cstdio>
int main() {
  unsigned a, b, c, d, k0, k1;
  while (std::scanf("%u %u %u %u %u %u", &a, &b, &c, &d, &k0, &k1) == 6) {
    uint4 ctr = make_uint4(a, b, c, d);
    uint2 key = make_uint2(k0, k1);
    uint4 r = curand_Philox4x32_10(ctr, key);
    std::printf("%u %u %u %u\n", r.x, r.y, r.z, r.w);
  }
  return 0;
}
"""


def _curand_philox(rows):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.cu")
        exe = os.path.join(d, "p")
        open(src, "w").write(_CURAND_PROBE)
        subprocess.check_call([nvcc, "-O1", "-o", exe, src])
        inp = "\n".join(" ".join(str(v) for v in r) for r in rows) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    return [tuple(int(x) for x in line.split()) for line in out.strip().splitlines()]


def test_philox_matches_curand_host_implementation():
    rnd = random.Random(31)
    rows = [(0, 0, 0, 0, 0, 0), (0xFFFFFFFF,) * 6]
    rows += [tuple(rnd.getrandbits(32) for _ in range(6)) for _ in range(300)]
    rows += [(h, p, 0, 0, 12345, 0) for h in range(20) for p in range(3)]
    ref = _curand_philox(rows)
    for r, e in zip(rows, ref):
        got = tuple(int(v) for v in oracle.philox4x32_10(r[:4], r[4:]))
        assert got == e


def _remaining_list(js, N):
    rem = list(range(N))
    return [rem.pop(j) for j in js]


def test_sample4_equals_rank_of_remaining_definition():
    for N in (4, 5, 7, 100, 2000, 1 << 20):
        for hyp in range(50):
            seed, prob = 0xC0FFEE + N, 3
            u = oracle.philox4x32_10([hyp, prob, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])
            js = [(int(u[k]) * (N - k)) >> 32 for k in range(4)]
            idx = oracle.sample4(seed, prob, hyp, N)
            assert list(idx) == _remaining_list(js, N)
            assert len(set(idx)) == 4 and min(idx) >= 0 and max(idx) < N


def test_sample4_is_uniform_over_ordered_tuples():
    N = 5
    cnt = Counter(tuple(oracle.sample4(7, 0, h, N)) for h in range(24000))
    assert len(cnt) == 120
    exp = 24000 / 120
    chi2 = sum((c - exp) ** 2 / exp for c in cnt.values())
    assert chi2 < 180          # 119 dof, p ~ 3e-4


def _read_table8():
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


def test_adaptive_count_reproduces_the_papers_sample_numbers():
    rows, cap = _read_table8()
    for samples, outlier_pct in rows[1:]:
        # the paper rounds the outlier ratio to a whole percent: the sample
        # count must fall between the counts at the two neighbouring ratios
        lo = workloads.adaptive_hypotheses(1 - (outlier_pct - 0.5) / 100, cap=10**9)
        hi = workloads.adaptive_hypotheses(1 - (outlier_pct + 0.5) / 100, cap=10**9)
        assert lo <= samples <= hi, (samples, outlier_pct, lo, hi)
    assert workloads.adaptive_hypotheses(1.0) == 1
    k26 = workloads.adaptive_hypotheses(cap[1] / 100, cap=10**9)
    assert abs(k26 - cap[0]) / cap[0] < 0.05
    assert workloads.adaptive_hypotheses(0.05) == 16384


def test_noise_free_inlier_hypotheses_count_all_inliers():
    rp = workloads.ransac_problem(300, 0.6, 0.0, seed=5)
    cnt, _, _ = oracle.score_problem(rp.corr, 400, 1.0, seed=11)
    n_in = int(rp.is_inlier.sum())
    for h in range(400):
        idx = oracle.sample4(11, 0, h, 300)
        if rp.is_inlier[idx].all() and cnt[h] >= 0:
            assert cnt[h] >= n_in
            assert cnt[h] <= n_in + 2      # an outlier may land within 1 px by chance
    r = oracle.ransac(rp.corr, [0, 300], [400], 1.0, 11, want_mask=True)
    assert r["best_count"][0] >= n_in
    assert int(r["inlier_mask"].sum()) == r["best_count"][0]
    Ht = rp.H_true.reshape(9) / np.linalg.norm(rp.H_true)
    Ht = Ht * np.sign(Ht[8])
    assert np.max(np.abs(r["best_H"][0] - Ht)) < 1e-5


def test_collinear_problem_has_no_valid_hypothesis():
    x = np.linspace(0, 600, 50)
    corr = np.stack([x, 2 * x + 1, x + 3, 0.5 * x], axis=1).astype(np.float32)
    r = oracle.ransac(corr, [0, 50], [64], 3.0, 1, want_mask=True)
    assert r["best_hyp"][0] == -1 and r["best_count"][0] == 0
    assert np.all(r["hyp_counts"] == -1)
    assert r["inlier_mask"].sum() == 0


def test_too_few_points_and_zero_hypotheses():
    corr = np.zeros((3, 4), dtype=np.float32)
    r = oracle.ransac(corr, [0, 3, 3], [5, 0], 3.0, 1)
    assert list(r["best_hyp"]) == [-1, -1] and list(r["best_count"]) == [0, 0]


def test_argmax_takes_the_lowest_index_among_ties():
    rp = workloads.ransac_problem(200, 0.9, 0.0, seed=6)
    r = oracle.ransac(rp.corr, [0, 200], [256], 1.0, 3)
    c = r["hyp_counts"]
    best = c.max()
    assert r["best_hyp"][0] == int(np.nonzero(c == best)[0][0])
    assert r["best_count"][0] == best


def test_scoring_matches_direct_residuals_of_oracle_hypotheses():
    rp = workloads.ransac_problem(120, 0.5, 1.0, seed=7)
    cnt, b_in, b_out = oracle.score_problem(rp.corr, 64, 3.0, seed=2, band_px=1e-3)
    c64 = rp.corr.astype(np.float64)
    for h in range(64):
        idx = oracle.sample4(2, 0, h, 120)
        s = np.concatenate([c64[idx, :2].ravel(), c64[idx, 2:].ravel()])
        if oracle.sample_degenerate(s):
            assert cnt[h] == -1 and b_in[h] == 0 and b_out[h] == 0
            continue
        H = oracle.aca(s.reshape(16, 1)).reshape(3, 3)
        X = np.stack([c64[:, 0], c64[:, 1], np.ones(120)])
        U = H @ X
        ok = U[2] != 0
        r = np.hypot(c64[:, 2] - U[0] / U[2], c64[:, 3] - U[1] / U[2])
        inl = ok & (r <= 3.0)
        assert cnt[h] == int(np.sum(inl))
        # the band is per point: the fixed band, widened by the FP32 test's
        # derived bound; split by the exact decision
        amb = oracle.score_band(s, rp.corr, 3.0, band_px=1e-3).astype(bool)
        assert np.all(amb[ok & (np.abs(r - 3.0) < 1e-3)])
        assert b_in[h] == int(np.sum(amb & inl)) and b_out[h] == int(np.sum(amb & ~inl))


def test_ambiguity_band_is_the_fixed_band_united_with_the_derived_fp32_band():
    rp = workloads.ransac_problem(400, 0.6, 1.0, seed=8)
    c0, i0, o0 = oracle.score_problem(rp.corr, 128, 3.0, seed=4, band_px=0.0)      # derived band alone
    c1, i1, o1 = oracle.score_problem(rp.corr, 128, 3.0, seed=4, band_px=1e-3)
    c2, i2, o2 = oracle.score_problem(rp.corr, 128, 3.0, seed=4, band_px=1e-1)
    assert np.array_equal(c0, c1) and np.array_equal(c1, c2)
    assert np.all(i0 <= i1) and np.all(i1 <= i2) and np.all(o0 <= o1) and np.all(o1 <= o2)
    assert (i2 + o2).sum() > (i0 + o0).sum()
    # per point, the derived band is exactly where |E| <= the FP32 bound
    for h in range(0, 128, 16):
        idx = oracle.sample4(4, 0, h, 400)
        s = np.concatenate([rp.corr[idx, :2].astype(np.float64).ravel(), rp.corr[idx, 2:].astype(np.float64).ravel()])
        if oracle.sample_degenerate(s):
            continue
        E, B = oracle.score_bound_E(s, rp.corr, 3.0)
        amb = oracle.score_band(s, rp.corr, 3.0, band_px=0.0).astype(bool)
        assert np.array_equal(amb, ~(np.abs(E) > B))
    # a noise-free problem: residuals of all-inlier hypotheses are ~0, far
    # from the threshold, so nothing is ambiguous for most of them
    rq = workloads.ransac_problem(300, 1.0, 0.0, seed=9)
    c, bi, bo = oracle.score_problem(rq.corr, 64, 3.0, seed=1, band_px=1e-4)
    assert np.mean((bi + bo)[c == 300] == 0) > 0.9


def test_each_collinear_triple_alone_makes_a_sample_degenerate():
    # reading 10: a sample is degenerate when, on either side, any of its
    # triples (M,N,P), (M,Q,P), (M,N,Q), (N,P,Q) has sine of the angle at
    # its first point at most 1e-3; one triple made collinear at a time
    ms = workloads.minimal_sets(4, seed=8)
    base = oracle.sets_aos(ms.pts)
    for b in base:
        assert not oracle.sample_degenerate(b)
        for side in (0, 8):
            P = {k: b[side + 2 * i: side + 2 * i + 2].copy() for i, k in enumerate("MNPQ")}
            for moved, a, c in (("P", "M", "N"), ("Q", "M", "P"), ("Q", "M", "N"), ("Q", "N", "P")):
                t = b.copy()
                i = "MNPQ".index(moved)
                t[side + 2 * i: side + 2 * i + 2] = P[a] + 1.7 * (P[c] - P[a])
                assert oracle.sample_degenerate(t), (side, moved, a, c)


def test_degenerate_sample_threshold_is_a_sine_of_1e3():
    # the angle at M between MN and MP just below and just above sine 1e-3
    ms = workloads.minimal_sets(1, seed=9)
    b = oracle.sets_aos(ms.pts)[0]
    M, N = b[0:2], b[2:4]
    u = (N - M) / np.linalg.norm(N - M)
    v = np.array([-u[1], u[0]])
    assert not oracle.sample_degenerate(b)
    for sine, expect in ((0.9e-3, True), (1.1e-3, False)):
        t = b.copy()
        t[4:6] = M + 200.0 * (np.sqrt(1 - sine * sine) * u + sine * v)
        assert oracle.sample_degenerate(t) == expect, sine


def test_inlier_test_is_inclusive_at_the_threshold():
    # reading 11: the oracle's test is ||x2 - pi(H x1)|| <= thr, inclusive.
    # Seven small integer points moved by an integer translation, and one
    # point moved 3 px further along x: every hypothesis drawn from four of
    # the seven is that translation, with integer entries small enough that
    # FP64 holds every product of the chain exactly, so every residual is
    # exact; it counts the eighth point at thr = 3 but not a hair below.
    src = np.array([[1, 2], [17, 3], [4, 15], [19, 12], [9, 8], [14, 18], [2, 11], [12, 1]], dtype=np.float32)
    dst = src + np.array([5, -2], dtype=np.float32)
    dst[7, 0] += 3
    corr = np.ascontiguousarray(np.c_[src, dst], dtype=np.float32)
    exact = [h for h in range(400) if 7 not in oracle.sample4(5, 0, h, 8)]
    assert len(exact) > 50
    for thr, count in ((3.0, 8), (2.999, 7)):
        c = oracle.ransac(corr, [0, 8], [400], thr, 5, band_px=0.0)["hyp_counts"]
        assert all(int(c[h]) == count for h in exact), (thr, sorted(set(int(c[h]) for h in exact)))


def test_a_sample_with_a_non_finite_coordinate_is_degenerate():
    ms = workloads.minimal_sets(8, seed=3)
    s = oracle.sets_aos(ms.pts)
    assert not any(oracle.sample_degenerate(s[i]) for i in range(8))
    for k, v in ((0, np.nan), (5, np.inf), (9, -np.inf), (15, -np.nan)):
        t = s[k % 8].copy()
        t[k] = v
        assert oracle.sample_degenerate(t)
