"""FP64 refit of a homography on all inliers of each problem: TEST
INFRASTRUCTURE ONLY (see the package docstring).

The paper's RANSAC pipeline ends with a global optimisation on all inliers
(Sec. 6.2, stage 5): a Levenberg-Marquardt (LM) minimisation of the
reprojection error, started from a linear fit.  This module writes both steps
out plainly, per problem, in float64:

1. Linear fit: the normalised DLT.  Each side is translated to its centroid
   and scaled so the mean distance to it is sqrt(2) (Hartley normalisation);
   each point contributes the two rows of Eq. 2; h is the right singular
   vector of the smallest singular value (numpy's SVD).
2. LM on F(h) = 1/2 sum_i ||pi(H x_i) - X_i||^2 over the eight entries of the
   normalised H with h33 = 1, with the damping schedule of Madsen, Nielsen &
   Tingleff, "Methods for non-linear least squares problems" (2004), Alg. 3.16:
   mu0 = tau max diag(J^T J) with tau = 1e-6, their value for a start believed
   close to the minimiser (the DLT of the same points); a step solves (J^T J + mu I) d = -J^T r; the gain
   ratio rho = (F(h) - F(h + d)) / (1/2 d^T (mu d - g)) accepts (rho > 0, mu
   scaled by max(1/3, 1 - (2 rho - 1)^3), nu = 2) or rejects (mu *= nu,
   nu *= 2) it; every trial step counts as one iteration.  When the first
   trial is rejected the start was not close, and mu becomes their value for
   a poorer start, 1e-3 max diag(J^T J), with nu unchanged.  A numerically
   singular J^T J + mu I (H sends the points to infinity and J vanishes) is a
   rejected trial; LM ends when mu is no longer finite.

The target normalisation is a similarity, so F in the normalised frame is the
pixel reprojection error times a constant: both have the same minimiser.
"""
from __future__ import annotations

import numpy as np

from . import normalize_frob

SQRT2 = np.sqrt(2.0)


def hartley_normalization(xy) -> np.ndarray:
    """3x3 T with T (x, y, 1): centroid at the origin, mean distance sqrt(2)."""
    xy = np.asarray(xy, dtype=np.float64)
    mu = xy.mean(axis=0)
    d = np.mean(np.hypot(xy[:, 0] - mu[0], xy[:, 1] - mu[1]))
    sc = SQRT2 / d
    return np.array([[sc, 0.0, -sc * mu[0]], [0.0, sc, -sc * mu[1]], [0.0, 0.0, 1.0]])


def _problems(corr, offsets, mask):
    c = np.asarray(corr, dtype=np.float32).astype(np.float64)
    off = np.asarray(offsets, dtype=np.int64)
    m = np.asarray(mask).astype(bool)
    for p in range(off.size - 1):
        yield p, c[off[p]:off[p + 1]][m[off[p]:off[p + 1]]]


def _homog(xy):
    return np.c_[xy, np.ones(len(xy))]


def _dlt_normalized(x, X) -> np.ndarray:
    """Smallest right singular vector of the Eq. 2 rows of normalised points."""
    A = np.zeros((max(2 * len(x), 9), 9))     # a zero row keeps 9 singular vectors for n = 4
    xh = _homog(x)
    A[0:2 * len(x):2, 0:3] = xh
    A[0:2 * len(x):2, 6:9] = -X[:, 0:1] * xh
    A[1:2 * len(x):2, 3:6] = -xh
    A[1:2 * len(x):2, 6:9] = X[:, 1:2] * xh
    return np.linalg.svd(A, full_matrices=False)[2][-1].reshape(3, 3)


def _frame(sel):
    T1, T2 = hartley_normalization(sel[:, :2]), hartley_normalization(sel[:, 2:])
    x = (T1 @ _homog(sel[:, :2]).T).T[:, :2]
    X = (T2 @ _homog(sel[:, 2:]).T).T[:, :2]
    return T1, T2, x, X


def refit_dlt(corr, offsets, mask):
    """Normalised DLT on the masked points of each problem.  Returns (P, 9)
    unit-Frobenius sign-fixed H (zeros with fewer than 4 points) and the
    number of points used."""
    P = np.asarray(offsets).size - 1
    out = np.zeros((P, 9))
    used = np.zeros(P, dtype=np.int64)
    for p, sel in _problems(corr, offsets, mask):
        used[p] = len(sel)
        if len(sel) < 4:
            continue
        T1, T2, x, X = _frame(sel)
        H = np.linalg.inv(T2) @ _dlt_normalized(x, X) @ T1
        out[p] = normalize_frob(H.reshape(9))[0]
    return out, used


def _residuals(h8, x, X):
    """r (2n) and J (2n x 8) of pi(H x) - X with H = [h8, 1]."""
    h = np.append(h8, 1.0)
    u_ = h[0] * x[:, 0] + h[1] * x[:, 1] + h[2]
    v_ = h[3] * x[:, 0] + h[4] * x[:, 1] + h[5]
    w = h[6] * x[:, 0] + h[7] * x[:, 1] + h[8]
    u, v = u_ / w, v_ / w
    r = np.empty(2 * len(x))
    r[0::2] = u - X[:, 0]
    r[1::2] = v - X[:, 1]
    J = np.zeros((2 * len(x), 8))
    J[0::2, 0] = x[:, 0] / w
    J[0::2, 1] = x[:, 1] / w
    J[0::2, 2] = 1.0 / w
    J[0::2, 6] = -u * x[:, 0] / w
    J[0::2, 7] = -u * x[:, 1] / w
    J[1::2, 3] = x[:, 0] / w
    J[1::2, 4] = x[:, 1] / w
    J[1::2, 5] = 1.0 / w
    J[1::2, 6] = -v * x[:, 0] / w
    J[1::2, 7] = -v * x[:, 1] / w
    return r, J


def _lm(h8, x, X, iters, tau=1e-6, tau_poor=1e-3, eps2=1e-12):
    r, J = _residuals(h8, x, X)
    A, g, F = J.T @ J, J.T @ r, 0.5 * r @ r
    mu, nu = tau * np.max(np.diag(A)), 2.0
    mu_poor = tau_poor * np.max(np.diag(A))
    for trial in range(iters):
        if not (np.isfinite(mu) and mu > 0.0):
            break
        try:
            d = np.linalg.solve(A + mu * np.eye(8), -g)
        except np.linalg.LinAlgError:           # numerically singular: a rejected trial
            d = None
        if d is not None and np.linalg.norm(d) <= eps2 * (np.linalg.norm(h8) + eps2):
            break
        rho = -1.0
        if d is not None:
            hn = h8 + d
            rn, Jn = _residuals(hn, x, X)
            Fn = 0.5 * rn @ rn
            with np.errstate(invalid="ignore"):
                rho = (F - Fn) / (0.5 * d @ (mu * d - g))
        if rho > 0:
            h8, A, g, F = hn, Jn.T @ Jn, Jn.T @ rn, Fn
            mu *= max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3)
            nu = 2.0
        elif trial == 0:
            mu = mu_poor
        else:
            mu *= nu
            nu *= 2.0
    return h8


def refit_lm(corr, offsets, mask, H_start, iters: int = 200):
    """LM on the masked points of each problem from H_start (P, 9), in the
    normalised frames.  Returns (P, 9) unit-Frobenius sign-fixed H; problems
    with fewer than 4 points, or whose normalised start has |h33| below 1e-3
    of its norm, keep H_start."""
    H_start = np.asarray(H_start, dtype=np.float64).reshape(-1, 9)
    out = H_start.copy()
    for p, sel in _problems(corr, offsets, mask):
        if len(sel) < 4:
            continue
        T1, T2, x, X = _frame(sel)
        Hn = T2 @ H_start[p].reshape(3, 3) @ np.linalg.inv(T1)
        if abs(Hn[2, 2]) < 1e-3 * np.linalg.norm(Hn):
            continue
        h8 = _lm((Hn / Hn[2, 2]).reshape(9)[:8], x, X, iters)
        H = np.linalg.inv(T2) @ np.append(h8, 1.0).reshape(3, 3) @ T1
        out[p] = normalize_frob(H.reshape(9))[0]
    return out


def refit(corr, offsets, mask, lm_iters: int = 200):
    """Normalised DLT, then LM for lm_iters trial steps (0: DLT only)."""
    H, used = refit_dlt(corr, offsets, mask)
    if lm_iters > 0:
        H = refit_lm(corr, offsets, mask, H, lm_iters)
    return H, used


def reprojection_cost(H, corr, offsets, mask) -> np.ndarray:
    """Per-problem sum of squared pixel reprojection errors of the masked
    points, sum ||pi(H x) - X||^2, in float64 (inf when a point maps to
    infinity)."""
    H = np.asarray(H, dtype=np.float64).reshape(-1, 9)
    out = np.zeros(H.shape[0])
    for p, sel in _problems(corr, offsets, mask):
        if len(sel) == 0:
            continue
        q = H[p].reshape(3, 3) @ _homog(sel[:, :2]).T
        with np.errstate(divide="ignore", invalid="ignore"):
            e = (q[0] / q[2] - sel[:, 2]) ** 2 + (q[1] / q[2] - sel[:, 3]) ** 2
        out[p] = np.sum(e) if np.all(np.isfinite(e)) else np.inf
    return out


def refit_tolerance(corr, offsets, mask, lm_iters: int = 200, draws: int = 4, rel: float = 16 * 2.0 ** -24,
                    seed: int = 0) -> np.ndarray:
    """Per-problem conditioning of the refit: the largest entry-wise movement
    of the unit-Frobenius H when every input coordinate is moved by `rel`
    relative (random signs, `draws` draws, rounded back to float32).  An FP32
    evaluation is backward stable with errors of a few units of 2^-24 in the
    normalised coordinates, so its distance from the float64 result is of
    the order of this movement."""
    c = np.asarray(corr, dtype=np.float32)
    H0, _ = refit(c, offsets, mask, lm_iters)
    rng = np.random.default_rng(seed)
    out = np.zeros(H0.shape[0])
    for _ in range(draws):
        s = rng.choice([-1.0, 1.0], size=c.shape)
        cp = (c.astype(np.float64) * (1.0 + rel * s)).astype(np.float32)
        H1, _ = refit(cp, offsets, mask, lm_iters)
        out = np.maximum(out, np.max(np.abs(H1 - H0), axis=1))
    return out
