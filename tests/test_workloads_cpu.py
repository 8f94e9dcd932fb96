"""The seeded input generators match the recipe they state: minimal sets
(image bounds, the 5 px collinearity rejection, the 0.5 px near-degenerate
fraction, target = H(source), bounded projective depth, prefix property,
worker-count invariance), RANSAC pairs (N range, inlier fraction, noise,
hypothesis counts from the 99 % rule) and rectangle offsets.  Distances are
recomputed here from the generated points, independently of the
generator's own helpers."""
import math

import numpy as np
import pytest

import workloads


def _altitudes(x, y):
    """Point-to-line distance of every point of every triple, (m, 12)."""
    out = []
    for a, b, c in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
        for p, q, r in ((a, b, c), (b, c, a), (c, a, b)):   # distance of r from line p q
            dx, dy = x[:, q] - x[:, p], y[:, q] - y[:, p]
            ex, ey = x[:, r] - x[:, p], y[:, r] - y[:, p]
            out.append(np.abs(dx * ey - dy * ex) / np.hypot(dx, dy))
    return np.stack(out, axis=1)


def _sides(ms, n):
    p = ms.pts[:, :n].astype(np.float64)
    return p[0:8:2].T, p[1:8:2].T, p[8:16:2].T, p[9:16:2].T   # (n, 4) each: M N P Q


@pytest.fixture(scope="module")
def sets():
    return workloads.minimal_sets(20000, seed=3, degenerate_frac=0.01)


def test_minimal_sets_recipe(sets):
    n = 20000
    sx, sy, tx, ty = _sides(sets, n)
    ok = ~sets.near_degenerate
    # sources in the image (a near-degenerate set's P1 is moved next to the
    # line M1 N1, which can take it a little outside)
    assert sx[ok].min() >= 0 and sx[ok].max() <= 640 and sy[ok].min() >= 0 and sy[ok].max() <= 480
    # the longest-side altitude used by the rejection is at least the smallest
    # point-to-line distance; every triple is >= 5 px from collinear (both sides)
    assert _altitudes(sx[ok], sy[ok]).max(axis=1).min() >= 5.0 - 1e-3
    tri = lambda x, y: np.min([np.abs((x[:, b] - x[:, a]) * (y[:, c] - y[:, a]) - (y[:, b] - y[:, a]) *
                                      (x[:, c] - x[:, a])) /
                               np.max([np.hypot(x[:, b] - x[:, a], y[:, b] - y[:, a]),
                                       np.hypot(x[:, c] - x[:, a], y[:, c] - y[:, a]),
                                       np.hypot(x[:, c] - x[:, b], y[:, c] - y[:, b])], axis=0)
                               for a, b, c in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3))], axis=0)
    assert tri(sx[ok], sy[ok]).min() >= 5.0 - 1e-3 and tri(tx[ok], ty[ok]).min() >= 5.0 - 1e-3
    # target = H(source), up to the float32 rounding of the coordinates
    H = sets.H_true
    w = H[:, 2, 0, None] * sx + H[:, 2, 1, None] * sy + H[:, 2, 2, None]
    u = (H[:, 0, 0, None] * sx + H[:, 0, 1, None] * sy + H[:, 0, 2, None]) / w
    v = (H[:, 1, 0, None] * sx + H[:, 1, 1, None] * sy + H[:, 1, 2, None]) / w
    assert np.abs(u - tx).max() < 1e-3 and np.abs(v - ty).max() < 1e-3
    # projective depth over the image corners stays in [0.44, 1.56]
    cx = np.array([0, 640, 0, 640.0])
    cy = np.array([0, 0, 480, 480.0])
    wc = H[:, 2, 0, None] * cx + H[:, 2, 1, None] * cy + H[:, 2, 2, None]
    assert wc.min() > 0.43 and wc.max() < 1.57


def test_near_degenerate_sets(sets):
    near = sets.near_degenerate
    k = int(near.sum())
    assert abs(k - 200) < 4 * math.sqrt(200 * 0.99)          # binomial(20000, 0.01)
    sx, sy, _, _ = _sides(sets, 20000)
    # P1 lies within 0.5 px of the line M1 N1 (source side), up to rounding
    dx, dy = sx[near, 1] - sx[near, 0], sy[near, 1] - sy[near, 0]
    ex, ey = sx[near, 2] - sx[near, 0], sy[near, 2] - sy[near, 0]
    d = np.abs(dx * ey - dy * ex) / np.hypot(dx, dy)
    assert d.max() <= 0.5 + 1e-3
    assert d.mean() > 0.15                                      # U[0, 0.5]: mean 0.25


def test_minimal_sets_are_seeded_and_prefix_stable(sets):
    head = workloads.minimal_sets(100, seed=3, degenerate_frac=0.01)
    assert np.array_equal(head.pts, sets.pts[:, :100])
    assert np.array_equal(head.near_degenerate, sets.near_degenerate[:100])
    other = workloads.minimal_sets(100, seed=4, degenerate_frac=0.01)
    assert not np.array_equal(other.pts, head.pts)
    padded = workloads.minimal_sets(100, seed=3, degenerate_frac=0.01, ld=104)
    assert np.array_equal(padded.pts[:, :100], head.pts) and np.all(padded.pts[:, 100:] == 0)


def test_parallel_generation_gives_the_same_sets():
    n = workloads.CHUNK + 37
    one = workloads.minimal_sets(n, seed=9, keep_truth=False, workers=1)
    two = workloads.minimal_sets(n, seed=9, keep_truth=False, workers=2)
    assert np.array_equal(one.pts, two.pts)


def test_sample_count_rule():
    # k = ceil(log(1 - 0.99) / log(1 - eps^4)), capped
    assert workloads.adaptive_hypotheses(0.5) == 72
    assert workloads.adaptive_hypotheses(0.9) == 5
    assert workloads.adaptive_hypotheses(0.1) == 16384
    assert workloads.adaptive_hypotheses(0.1, cap=100000) == 46050
    assert workloads.adaptive_hypotheses(1.0) == 1 and workloads.adaptive_hypotheses(0.0) == 16384


def test_ransac_batch_recipe():
    rb = workloads.ransac_batch(P=64, seed=5)
    N = np.diff(rb.offsets)
    assert rb.offsets[0] == 0 and rb.offsets[-1] == rb.corr.shape[0] == rb.is_inlier.size
    assert N.min() >= 200 and N.max() <= 8000
    assert np.all((rb.inlier_ratio >= 0.1) & (rb.inlier_ratio <= 0.9))
    assert np.all((rb.sigma >= 0.5) & (rb.sigma <= 2.0))
    assert np.array_equal(rb.n_hyp, [workloads.adaptive_hypotheses(float(e)) for e in rb.inlier_ratio])
    c = rb.corr.astype(np.float64)
    assert c[:, 0].min() >= 0 and c[:, 0].max() <= 640 and c[:, 1].min() >= 0 and c[:, 1].max() <= 480
    for p in range(64):
        a, b = rb.offsets[p], rb.offsets[p + 1]
        inl = rb.is_inlier[a:b]
        assert inl.sum() == int(round(rb.inlier_ratio[p] * (b - a)))


def test_ransac_problem_noise_and_outliers():
    rp = workloads.ransac_problem(20000, 0.6, 1.5, seed=8)
    H = rp.H_true
    c = rp.corr.astype(np.float64)
    w = H[2, 0] * c[:, 0] + H[2, 1] * c[:, 1] + H[2, 2]
    u = (H[0, 0] * c[:, 0] + H[0, 1] * c[:, 1] + H[0, 2]) / w
    v = (H[1, 0] * c[:, 0] + H[1, 1] * c[:, 1] + H[1, 2]) / w
    r = np.concatenate([(c[:, 2] - u)[rp.is_inlier], (c[:, 3] - v)[rp.is_inlier]])
    assert abs(r.std() - 1.5) < 0.05 and abs(r.mean()) < 0.05          # N(0, 1.5^2) per coordinate
    out = ~rp.is_inlier
    assert abs(c[out, 2].mean() - 320) < 10 and abs(c[out, 3].mean() - 240) < 10   # U[image]
    assert rp.is_inlier.sum() == 12000 and not np.all(rp.is_inlier[:12000])        # permuted


def test_rect_batch_recipe():
    rb = workloads.rect_batch(4096, seed=2)
    src = rb.src_corners
    assert np.array_equal(src, [[32, 32], [160, 32], [32, 160], [160, 160]])
    off = rb.tgt.astype(np.float64).T.reshape(-1, 4, 2) - src
    assert off.min() >= -32 - 1e-4 and off.max() <= 32 + 1e-4 and abs(off.mean()) < 0.5
    gt = rb.tgt_gt.astype(np.float64) - rb.tgt.astype(np.float64)
    assert abs(gt.std() - 2.0) < 0.05
    assert rb.rect == (32.0, 32.0, 128.0, 1.0)
