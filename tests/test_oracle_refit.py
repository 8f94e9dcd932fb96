"""Pins of the oracle's refit on all inliers (the global optimisation after
RANSAC, Sec. 6.2 stage 5): normalised DLT, then Levenberg-Marquardt.  Each
pin checks the oracle against something other than itself: exact recovery
from noise-free data, the ACA minimal solution on four points, the
similarity covariance that only a correctly normalised DLT has, MINPACK's
LM (scipy) on the pixel-frame residuals, and central differences of the
cost."""
import numpy as np
import pytest

import oracle
import workloads


def _problem(N=300, eps=0.7, sigma=1.0, seed=12):
    rp = workloads.ransac_problem(N, eps, sigma, seed=seed)
    return rp, np.array([0, N])


def test_hartley_normalization_centroid_and_mean_distance():
    xy = np.random.default_rng(0).uniform(0, 640, (57, 2))
    T = oracle.hartley_normalization(xy)
    q = (T @ np.c_[xy, np.ones(57)].T).T
    assert np.allclose(q[:, 2], 1.0)
    assert np.allclose(q[:, :2].mean(axis=0), 0.0, atol=1e-12)
    assert abs(np.mean(np.hypot(q[:, 0], q[:, 1])) - np.sqrt(2.0)) < 1e-12
    assert T[0, 0] == T[1, 1] and T[0, 1] == 0 and T[1, 0] == 0     # isotropic


def test_dlt_recovers_the_exact_map_from_noise_free_inliers():
    rp, off = _problem(sigma=0.0)
    H, used = oracle.refit_dlt(rp.corr, off, rp.is_inlier)
    Ht = oracle.normalize_frob(rp.H_true.reshape(9))[0]
    assert used[0] == rp.is_inlier.sum()
    assert np.max(np.abs(H[0] - Ht)) < 1e-6      # float32 rounding of the points only


def test_dlt_of_exactly_four_points_is_the_minimal_solution():
    ms = workloads.minimal_sets(20, seed=13)
    s = oracle.sets_aos(ms.pts)
    for i in range(20):
        corr = np.stack([s[i, 0:8:2], s[i, 1:8:2], s[i, 8:16:2], s[i, 9:16:2]], axis=1).astype(np.float32)
        H, _ = oracle.refit_dlt(corr, [0, 4], np.ones(4, bool))
        Ha = oracle.normalize_frob(oracle.aca(ms.pts[:, i:i + 1]))[0]
        assert np.max(np.abs(H[0] - Ha)) < 1e-8


def test_dlt_is_covariant_under_similarities_of_either_image():
    # The normalised DLT commutes with similarities (the unnormalised one does
    # not): fit(S2 X <- S1 x) = S2 H S1^-1.
    rp, off = _problem(sigma=2.0, seed=21)
    H, _ = oracle.refit_dlt(rp.corr, off, rp.is_inlier)
    rng = np.random.default_rng(5)

    def sim():
        a, s = rng.uniform(0, 2 * np.pi), rng.uniform(0.5, 2.0)
        return np.array([[s * np.cos(a), -s * np.sin(a), rng.uniform(-300, 300)],
                         [s * np.sin(a), s * np.cos(a), rng.uniform(-300, 300)], [0, 0, 1.0]])

    S1, S2 = sim(), sim()
    c = rp.corr.astype(np.float64)
    a = (S1 @ np.c_[c[:, :2], np.ones(len(c))].T).T
    b = (S2 @ np.c_[c[:, 2:], np.ones(len(c))].T).T
    corr2 = np.c_[a[:, :2], b[:, :2]]
    # float64 points: compare with the oracle's own float32 rounding removed
    H2, _ = oracle.refit_dlt(corr2.astype(np.float32), off, rp.is_inlier)
    expect = oracle.normalize_frob((S2 @ H[0].reshape(3, 3) @ np.linalg.inv(S1)).reshape(9))[0]
    assert np.max(np.abs(H2[0] - expect)) < 2e-5   # float32 rounding of the moved points


def test_refit_is_invariant_to_point_order_and_ignores_unmasked_points():
    rp, off = _problem(200, 0.6, 1.0, seed=14)
    H1, u1 = oracle.refit(rp.corr, off, rp.is_inlier)
    perm = np.random.default_rng(0).permutation(200)
    H2, u2 = oracle.refit(rp.corr[perm], off, rp.is_inlier[perm])
    assert u1[0] == u2[0] and np.max(np.abs(H1 - H2)) < 1e-10
    few, used = oracle.refit(rp.corr, off, np.arange(200) < 3)
    assert used[0] == 3 and np.all(few == 0)


def test_lm_converges_to_the_exact_map_from_a_perturbed_start():
    rp, off = _problem(sigma=0.0, seed=15)
    Ht = oracle.normalize_frob(rp.H_true.reshape(9))[0]
    start = Ht * (1 + 0.05 * np.random.default_rng(1).standard_normal(9))
    H = oracle.refit_lm(rp.corr, off, rp.is_inlier, start[None], iters=100)
    assert np.max(np.abs(H[0] - Ht)) < 1e-6
    assert oracle.reprojection_cost(H, rp.corr, off, rp.is_inlier)[0] < 1e-6


@pytest.mark.parametrize("seed,sigma", [(16, 0.5), (17, 1.0), (18, 2.0)])
def test_lm_optimum_matches_minpack(seed, sigma):
    opt = pytest.importorskip("scipy.optimize")
    rp, off = _problem(400, 0.6, sigma, seed=seed)
    H, _ = oracle.refit(rp.corr, off, rp.is_inlier)
    Hd, _ = oracle.refit_dlt(rp.corr, off, rp.is_inlier)
    sel = rp.corr[rp.is_inlier].astype(np.float64)

    def res(h8):
        h = np.append(h8, 1.0)
        w = h[6] * sel[:, 0] + h[7] * sel[:, 1] + h[8]
        return np.r_[(h[0] * sel[:, 0] + h[1] * sel[:, 1] + h[2]) / w - sel[:, 2],
                     (h[3] * sel[:, 0] + h[4] * sel[:, 1] + h[5]) / w - sel[:, 3]]

    r = opt.least_squares(res, (Hd[0] / Hd[0, 8])[:8], method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15,
                          x_scale="jac")
    Hm = oracle.normalize_frob(np.append(r.x, 1.0))[0]
    # MINPACK works on the badly scaled pixel-frame parameters and stops a
    # little short (its cost is never below the oracle's): agreement to 1e-8
    assert np.max(np.abs(H[0] - Hm)) < 1e-8
    cost = oracle.reprojection_cost(np.stack([H[0], Hd[0], Hm]), np.r_[rp.corr, rp.corr, rp.corr],
                                    np.array([0, 400, 800, 1200]), np.r_[rp.is_inlier, rp.is_inlier, rp.is_inlier])
    assert cost[0] <= cost[1]                       # LM never worse than its DLT start
    assert cost[0] <= cost[2] * (1 + 1e-12)

def _minpack(sel, h8_start):
    opt = pytest.importorskip("scipy.optimize")

    def res(h8):
        h = np.append(h8, 1.0)
        w = h[6] * sel[:, 0] + h[7] * sel[:, 1] + h[8]
        return np.r_[(h[0] * sel[:, 0] + h[1] * sel[:, 1] + h[2]) / w - sel[:, 2],
                     (h[3] * sel[:, 0] + h[4] * sel[:, 1] + h[5]) / w - sel[:, 3]]

    r = opt.least_squares(res, h8_start, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, x_scale="jac")
    return oracle.normalize_frob(np.append(r.x, 1.0))[0]


@pytest.mark.parametrize("seed,n,eps", [(2004, 10, 0.6), (2007, 6, 0.5)])
def test_lm_from_a_poor_start_rejects_its_first_trial_and_reaches_minpacks_optimum(seed, n, eps):
    # every point of a small contaminated set: the DLT is far from the
    # minimiser, the nearly undamped first trial (mu0 = 1e-6 max diag) is
    # rejected, and the damping restarts at the poor-start value
    from oracle import inlier_refit as ir
    rp = workloads.ransac_problem(n, eps, 1.0, seed=seed)
    off, m = np.array([0, n]), np.ones(n, bool)
    Hd, _ = oracle.refit_dlt(rp.corr, off, m)
    sel = rp.corr.astype(np.float64)
    T1, T2, x, X = ir._frame(sel)
    Hn = T2 @ Hd[0].reshape(3, 3) @ np.linalg.inv(T1)
    start = (Hn / Hn[2, 2]).reshape(9)[:8]
    assert np.array_equal(ir._lm(start, x, X, 1), start)
    H, _ = oracle.refit(rp.corr, off, m)
    Hm = _minpack(sel, (Hd[0] / Hd[0, 8])[:8])
    cost = oracle.reprojection_cost(np.stack([H[0], Hm]), np.r_[rp.corr, rp.corr], np.array([0, n, 2 * n]),
                                    np.r_[m, m])
    assert cost[0] <= cost[1] * (1 + 1e-9)
    assert np.max(np.abs(H[0] - Hm)) < 1e-5


def test_lm_on_a_degenerate_set_ends_without_error_and_never_above_its_start():
    # 8 points, half of them outliers: LM walks towards an H that sends the
    # points to infinity, where J^T J vanishes and J^T J + mu I becomes
    # numerically singular; those trials are rejected, mu grows until it is
    # no longer finite, and the result is finite
    rp = workloads.ransac_problem(8, 0.5, 1.0, seed=2005)
    off, m = np.array([0, 8]), np.ones(8, bool)
    H, used = oracle.refit(rp.corr, off, m)
    Hd, _ = oracle.refit_dlt(rp.corr, off, m)
    assert used[0] == 8 and np.all(np.isfinite(H))
    c = oracle.reprojection_cost(np.stack([H[0], Hd[0]]), np.r_[rp.corr, rp.corr], np.array([0, 8, 16]), np.r_[m, m])
    assert c[0] <= c[1]


def test_lm_optimum_is_stationary_under_central_differences():
    rp, off = _problem(300, 0.8, 1.5, seed=19)
    H, _ = oracle.refit(rp.corr, off, rp.is_inlier)
    h = H[0] / H[0, 8]
    f0 = oracle.reprojection_cost(h[None], rp.corr, off, rp.is_inlier)[0]
    for k in range(8):
        step = 1e-6 * max(abs(h[k]), 1e-3)
        hp, hm = h.copy(), h.copy()
        hp[k] += step
        hm[k] -= step
        fp = oracle.reprojection_cost(hp[None], rp.corr, off, rp.is_inlier)[0]
        fm = oracle.reprojection_cost(hm[None], rp.corr, off, rp.is_inlier)[0]
        curv = (fp - 2 * f0 + fm) / step ** 2
        grad = (fp - fm) / (2 * step)
        # relative to the curvature scale: the stationary point is within a
        # tiny fraction of a step
        assert abs(grad) <= 1e-5 * curv * step + 1e-9 * f0 / step, (k, grad, curv)
