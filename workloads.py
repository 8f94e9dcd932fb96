"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the CPU oracle's tests and by the CUDA path's tests
and benchmark.  It draws random numbers and maps points through randomly drawn
ground-truth homographies; it holds none of the ACA / SKS / RANSAC arithmetic
that the library or the oracle implement.

Layouts (all float32, generated in float64 and rounded once):

* minimal sets: SoA ``pts[16, ld]``; plane ``p = side*8 + point*2 + coord``
  with side 0 = source, 1 = target, point 0..3 = M, N, P, Q and coord 0/1 =
  x/y (the paper's anchor naming, Sec. 4.2: M, N, P are the three anchor
  points and Q the fourth correspondence);
* RANSAC correspondences: AoS ``corr[total, 4]`` = (x1, y1, x2, y2) per point,
  problems concatenated, ``offsets[P+1]`` (int64) in points;
* rectangle workloads: ``tgt[8, ld]`` = target corners M2, N2, P2, Q2 (x, y)
  for a fixed source rectangle (M upper-left, N upper-right, Q lower-right,
  P lower-left: the paper's clockwise order of Sec. 5.3).

Images are 640x480 as in the paper's RANSAC experiment (Sec. 6.2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

WIDTH = 640.0
HEIGHT = 480.0
CHUNK = 1 << 18          # sets per generator chunk (fixes the prefix property)
MIN_ALTITUDE_PX = 5.0    # sets with any triple closer to collinear are redrawn
NEAR_DEGENERATE_PX = 0.5


def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, *stream])))


def random_homographies(rng: np.random.Generator, m: int) -> np.ndarray:
    """Ground-truth homographies H = C * G * C^-1, shape (m, 3, 3), float64.

    G = [[s cos t, -s sin t, tx], [s sin t, s cos t, ty], [g, h, 1]] with
    t ~ U[-30, 30] deg, s ~ U[0.7, 1.4], tx, ty ~ U[-50, 50] px,
    g, h ~ U[-1e-3, 1e-3]; C translates the origin to the image centre so the
    projective depth stays within [0.44, 1.56] over the image.
    """
    th = np.deg2rad(rng.uniform(-30.0, 30.0, m))
    s = rng.uniform(0.7, 1.4, m)
    tx = rng.uniform(-50.0, 50.0, m)
    ty = rng.uniform(-50.0, 50.0, m)
    g = rng.uniform(-1e-3, 1e-3, m)
    h = rng.uniform(-1e-3, 1e-3, m)
    G = np.zeros((m, 3, 3))
    G[:, 0, 0] = s * np.cos(th)
    G[:, 0, 1] = -s * np.sin(th)
    G[:, 0, 2] = tx
    G[:, 1, 0] = s * np.sin(th)
    G[:, 1, 1] = s * np.cos(th)
    G[:, 1, 2] = ty
    G[:, 2, 0] = g
    G[:, 2, 1] = h
    G[:, 2, 2] = 1.0
    cx, cy = WIDTH / 2, HEIGHT / 2
    C = np.array([[1, 0, cx], [0, 1, cy], [0, 0, 1.0]])
    Ci = np.array([[1, 0, -cx], [0, 1, -cy], [0, 0, 1.0]])
    return C @ G @ Ci


def apply_h(H: np.ndarray, x: np.ndarray, y: np.ndarray):
    """Map points (x, y) (shape (m, k)) by per-row homographies H (m, 3, 3)."""
    u = H[:, 0, 0, None] * x + H[:, 0, 1, None] * y + H[:, 0, 2, None]
    v = H[:, 1, 0, None] * x + H[:, 1, 1, None] * y + H[:, 1, 2, None]
    w = H[:, 2, 0, None] * x + H[:, 2, 1, None] * y + H[:, 2, 2, None]
    return u / w, v / w, w


def _min_altitude(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Smallest point-to-line distance over the 4 triples of 4 points (m, 4)."""
    out = np.full(x.shape[0], np.inf)
    for a, b, c in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
        abx, aby = x[:, b] - x[:, a], y[:, b] - y[:, a]
        acx, acy = x[:, c] - x[:, a], y[:, c] - y[:, a]
        bcx, bcy = x[:, c] - x[:, b], y[:, c] - y[:, b]
        area2 = np.abs(abx * acy - aby * acx)
        longest = np.sqrt(np.maximum(np.maximum(abx**2 + aby**2, acx**2 + acy**2), bcx**2 + bcy**2))
        out = np.minimum(out, np.where(longest > 0, area2 / np.where(longest > 0, longest, 1), 0.0))
    return out


def _chunk_sets(seed: int, chunk: int, degenerate_frac: float):
    rng = _rng(seed, 0x5E75, chunk)
    m = CHUNK
    src_x = np.empty((m, 4))
    src_y = np.empty((m, 4))
    H = np.empty((m, 3, 3))
    todo = np.arange(m)
    while todo.size:
        k = todo.size
        sx = rng.uniform(0.0, WIDTH, (k, 4))
        sy = rng.uniform(0.0, HEIGHT, (k, 4))
        Hk = random_homographies(rng, k)
        tx, ty, _ = apply_h(Hk, sx, sy)
        ok = (_min_altitude(sx, sy) >= MIN_ALTITUDE_PX) & (_min_altitude(tx, ty) >= MIN_ALTITUDE_PX)
        src_x[todo[ok]] = sx[ok]
        src_y[todo[ok]] = sy[ok]
        H[todo[ok]] = Hk[ok]
        todo = todo[~ok]
    near = np.zeros(m, dtype=bool)
    if degenerate_frac > 0:
        near = rng.random(m) < degenerate_frac
        idx = np.nonzero(near)[0]
        # Move P1 to within U[0, 0.5] px of the line M1 N1 (random side).
        mx, my = src_x[idx, 0], src_y[idx, 0]
        dx, dy = src_x[idx, 1] - mx, src_y[idx, 1] - my
        L = np.hypot(dx, dy)
        ux, uy = dx / L, dy / L
        px, py = src_x[idx, 2] - mx, src_y[idx, 2] - my
        along = px * ux + py * uy
        d = rng.uniform(0.0, NEAR_DEGENERATE_PX, idx.size) * np.where(rng.random(idx.size) < 0.5, -1.0, 1.0)
        src_x[idx, 2] = mx + along * ux - d * uy
        src_y[idx, 2] = my + along * uy + d * ux
    tgt_x, tgt_y, _ = apply_h(H, src_x, src_y)
    return src_x, src_y, tgt_x, tgt_y, near, H


@dataclass
class MinimalSets:
    pts: np.ndarray        # float32 (16, ld)
    n: int
    near_degenerate: np.ndarray  # bool (n,) ground-truth label
    H_true: np.ndarray     # float64 (n, 3, 3)


def _chunk_job(args):
    seed, c, frac = args
    sx, sy, tx, ty, nr, H = _chunk_sets(seed, c, frac)
    return (np.concatenate([sx, sy, tx, ty], axis=1).astype(np.float32), nr, H)


def minimal_sets(n: int, seed: int = 0, degenerate_frac: float = 0.0, ld: int | None = None,
                 keep_truth: bool = True, workers: int = 1) -> MinimalSets:
    """n minimal 4-point sets: source U[0,640]x[0,480], target = H(source).

    Sets in which any triple of the 4 points (on either side) is within 5 px
    of collinear are redrawn.  A fraction ``degenerate_frac`` then gets its P1
    moved to within 0.5 px of the line M1 N1 (labelled in ``near_degenerate``).
    The first k sets do not depend on n (chunked generation).
    """
    if ld is None:
        ld = n
    assert ld >= n
    pts = np.zeros((16, ld), dtype=np.float32)
    near = np.zeros(n, dtype=bool)
    H_true = np.zeros((n, 3, 3)) if keep_truth else np.zeros((0, 3, 3))
    nchunks = (n + CHUNK - 1) // CHUNK
    jobs = [(seed, c, degenerate_frac) for c in range(nchunks)]
    if workers > 1 and nchunks > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, nchunks)) as pool:
            results = pool.imap(_chunk_job, jobs)
            _fill(results, n, pts, near, H_true, keep_truth)
    else:
        _fill(map(_chunk_job, jobs), n, pts, near, H_true, keep_truth)
    return MinimalSets(pts=pts, n=n, near_degenerate=near, H_true=H_true)


def _fill(results, n, pts, near, H_true, keep_truth):
    # columns of a chunk: src x (4), src y (4), tgt x (4), tgt y (4)
    for c, (cols, nr, H) in enumerate(results):
        lo = c * CHUNK
        hi = min(n, lo + CHUNK)
        k = hi - lo
        for pnt in range(4):
            pts[2 * pnt, lo:hi] = cols[:k, pnt]
            pts[2 * pnt + 1, lo:hi] = cols[:k, 4 + pnt]
            pts[8 + 2 * pnt, lo:hi] = cols[:k, 8 + pnt]
            pts[8 + 2 * pnt + 1, lo:hi] = cols[:k, 12 + pnt]
        near[lo:hi] = nr[:k]
        if keep_truth:
            H_true[lo:hi] = H[:k]


# --------------------------------------------------------------------------
# RANSAC workloads
# --------------------------------------------------------------------------

def adaptive_hypotheses(inlier_ratio: float, confidence: float = 0.99, cap: int = 16384) -> int:
    """Standard RANSAC sample count for a 4-point solver.

    k = ceil(log(1 - confidence) / log(1 - eps^4)), the rule the paper uses to
    relate sample numbers to outlier ratios at 99% confidence (Sec. 6.2 and
    Sec. 6.4), capped at ``cap``.
    """
    e4 = inlier_ratio ** 4
    if e4 >= 1.0:
        return 1
    if e4 <= 0.0:
        return cap
    k = math.ceil(math.log(1.0 - confidence) / math.log(1.0 - e4))
    return int(max(1, min(cap, k)))


@dataclass
class RansacProblem:
    corr: np.ndarray       # float32 (N, 4): x1, y1, x2, y2
    is_inlier: np.ndarray  # bool (N,)
    H_true: np.ndarray     # float64 (3, 3)


def ransac_problem(N: int, inlier_ratio: float, sigma: float, seed: int, stream: int = 0) -> RansacProblem:
    """One image pair: N correspondences in 640x480.

    round(eps*N) inliers: target = H(source) + N(0, sigma^2) per coordinate;
    the rest are outliers with source and target independent U[image].  The
    order is a seeded random permutation.
    """
    rng = _rng(seed, 0x4A45, stream)
    H = random_homographies(rng, 1)
    n_in = int(round(inlier_ratio * N))
    sx = rng.uniform(0.0, WIDTH, N)
    sy = rng.uniform(0.0, HEIGHT, N)
    tx, ty, _ = apply_h(H, sx[None, :], sy[None, :])
    tx = tx[0] + rng.normal(0.0, sigma, N)
    ty = ty[0] + rng.normal(0.0, sigma, N)
    ox = rng.uniform(0.0, WIDTH, N)
    oy = rng.uniform(0.0, HEIGHT, N)
    inl = np.zeros(N, dtype=bool)
    inl[:n_in] = True
    tx = np.where(inl, tx, ox)
    ty = np.where(inl, ty, oy)
    perm = rng.permutation(N)
    corr = np.stack([sx, sy, tx, ty], axis=1)[perm].astype(np.float32)
    return RansacProblem(corr=np.ascontiguousarray(corr), is_inlier=inl[perm], H_true=H[0])


@dataclass
class RansacBatch:
    corr: np.ndarray       # float32 (total, 4)
    offsets: np.ndarray    # int64 (P+1,)
    n_hyp: np.ndarray      # int32 (P,)
    inlier_ratio: np.ndarray
    sigma: np.ndarray
    is_inlier: np.ndarray  # bool (total,): the point was generated from the true H


def ransac_batch(P: int = 512, seed: int = 0, n_min: int = 200, n_max: int = 8000,
                 eps_lo: float = 0.1, eps_hi: float = 0.9, sigma_lo: float = 0.5,
                 sigma_hi: float = 2.0, cap: int = 16384) -> RansacBatch:
    """P uneven image pairs: N log-uniform in [n_min, n_max], eps ~ U[eps_lo,
    eps_hi], sigma ~ U[sigma_lo, sigma_hi]; hypothesis counts from the 99%
    confidence rule, capped."""
    rng = _rng(seed, 0xBA7C)
    Ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), P)).round().astype(np.int64)
    eps = rng.uniform(eps_lo, eps_hi, P)
    sig = rng.uniform(sigma_lo, sigma_hi, P)
    probs = [ransac_problem(int(Ns[p]), float(eps[p]), float(sig[p]), seed, stream=p + 1) for p in range(P)]
    parts = [pr.corr for pr in probs]
    offsets = np.zeros(P + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(Ns)
    n_hyp = np.array([adaptive_hypotheses(float(e), cap=cap) for e in eps], dtype=np.int32)
    return RansacBatch(corr=np.ascontiguousarray(np.concatenate(parts, axis=0)), offsets=offsets,
                       n_hyp=n_hyp, inlier_ratio=eps, sigma=sig,
                       is_inlier=np.concatenate([pr.is_inlier for pr in probs]))


# --------------------------------------------------------------------------
# Rectangle (4-point offset regression) workloads
# --------------------------------------------------------------------------

@dataclass
class RectBatch:
    rect: tuple            # (x0, y0, w, r): upper-left corner, width, aspect ratio w/h
    src_corners: np.ndarray  # float64 (4, 2): M, N, P, Q
    tgt: np.ndarray        # float32 (8, ld): M2, N2, P2, Q2 target corners
    tgt_gt: np.ndarray     # float32 (8, ld): second offset draw (ground truth)


def rect_corners(x0: float, y0: float, w: float, h: float) -> np.ndarray:
    """Corners in the anchor order M (upper-left), N (upper-right),
    P (lower-left), Q (lower-right)."""
    return np.array([[x0, y0], [x0 + w, y0], [x0, y0 + h], [x0 + w, y0 + h]], dtype=np.float64)


def rect_batch(B: int, seed: int = 0, x0: float = 32.0, y0: float = 32.0, w: float = 128.0,
               h: float = 128.0, max_offset: float = 32.0, gt_sigma: float = 2.0,
               ld: int | None = None) -> RectBatch:
    """Target corners = source corners + U[-max_offset, max_offset] per
    coordinate; the ground truth adds N(0, gt_sigma^2) to those offsets."""
    if ld is None:
        ld = B
    rng = _rng(seed, 0x7EC7)
    src = rect_corners(x0, y0, w, h)
    off = rng.uniform(-max_offset, max_offset, (B, 4, 2))
    off_gt = off + rng.normal(0.0, gt_sigma, (B, 4, 2))
    tgt = np.zeros((8, ld), dtype=np.float32)
    tgt_gt = np.zeros((8, ld), dtype=np.float32)
    for k in range(4):
        for c in range(2):
            tgt[2 * k + c, :B] = src[k, c] + off[:, k, c]
            tgt_gt[2 * k + c, :B] = src[k, c] + off_gt[:, k, c]
    return RectBatch(rect=(x0, y0, w, w / h), src_corners=src, tgt=tgt, tgt_gt=tgt_gt)


def grid_points(x0: float, y0: float, w: float, h: float, k: int = 8) -> np.ndarray:
    """A k x k grid spanning the patch, edges included, shape (k*k, 2)."""
    xs = np.linspace(x0, x0 + w, k)
    ys = np.linspace(y0, y0 + h, k)
    gx, gy = np.meshgrid(xs, ys, indexing="xy")
    return np.stack([gx.ravel(), gy.ravel()], axis=1)
