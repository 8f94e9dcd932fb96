"""Pins of the oracle's rounding-error bounds (oracle/fp32_bounds.c), the
tolerance model of the parity tests.  The bounds are derived, not chosen:
a first-order sum over every rounding event of the library's stated FP32
evaluation order, each event bounded by a published rule.  They are pinned
here against arithmetic other than their own:

1. every rule against exact rational arithmetic: the FP32 operation is
   emulated exactly (Fractions rounded to nearest even binary32) on random
   and cancellation-heavy operands, and its error never exceeds the rule's
   bound (Kahan's determinant: Jeannerod, Louvet and Muller 2013);
2. the whole ACA and SKS chains against a host build of the library's FP32
   arithmetic (the solver header compiled for the CPU with explicit
   roundings, which gives the kernels' bits): on every set, per entry and at
   unit Frobenius norm, the FP32 result lies within the bound; the bound is
   not vacuous (the largest error reaches a tenth of it); the chains' exact
   values are the H of the paper's ACA and SKS up to scale;
3. the inlier test: the host's FP32 test value lies within the bound of the
   exact E = w^2 (r^2 - thr^2) at every point, and every point decided
   otherwise than by the exact test lies inside the derived band;
4. the bound as a worst case over the set of rounding corners (every event
   at plus or minus its bound): the chains re-run at the corner the reverse
   sweep names as the worst land on the first-order bound to within the
   allowance for products of events, so a wrong partial derivative, a
   dropped path or a bound scaled up fails; and, for the inlier test at an
   exact FP32 H, an exhaustive enumeration of all 2^17 corners of its own
   17 rounding events, in an evaluation written out here, never exceeds the
   bound and comes within a few percent of it, so a dropped event or a bound
   too narrow or too wide fails."""
import ctypes
import os
import shutil
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import workloads

U = 2.0 ** -24
HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- exact FP32
def rn32(q):
    """Round a rational to the nearest binary32 value, ties to even (normal
    range only)."""
    q = Fr(q)
    if q == 0:
        return Fr(0)
    sgn = 1 if q > 0 else -1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fr(2) ** e > a:
        e -= 1
    while Fr(2) ** (e + 1) <= a:
        e += 1
    ulp = Fr(2) ** (e - 23)
    m = a / ulp
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fr(1, 2) or (rem == Fr(1, 2) and fl % 2 == 1):
        fl += 1
    return sgn * fl * ulp


def test_rn32_agrees_with_numpy_float32():
    rng = np.random.default_rng(0)
    for x in rng.standard_normal(500) * 10.0 ** rng.integers(-6, 7, 500):
        assert rn32(Fr(float(x))) == Fr(float(np.float32(x)))


def _kahan(a, b, c, d):
    w = rn32(b * c)
    e = rn32(-b * c + w)
    f = rn32(a * d - w)
    return rn32(f + e)


def _diff(a, b):
    """Exact difference as value + remainder (TwoSum on a and -b)."""
    d = rn32(a - b)
    bv = rn32(d - a)
    av = rn32(d - bv)
    return d, rn32(rn32(a - av) + rn32(-b - bv))


def _cross2x(u, v):
    """cross(u, v) of exact differences u = (ux, uy), v = (vx, vy), each a
    (value, remainder) pair: Kahan's determinant of the values plus the four
    first-order remainder products, in the library's order."""
    (uxh, uxl), (uyh, uyl) = u
    (vxh, vxl), (vyh, vyl) = v
    w = rn32(uyh * vxh)
    e = rn32(-uyh * vxh + w)
    f = rn32(uxh * vyh - w)
    c = rn32(uxh * vyl + rn32(uxl * vyh + rn32(-uyh * vxl + rn32(-uyl * vxh))))
    return rn32(f + rn32(e + c))


def _df_prod_mul_round(a, b, c):
    p = rn32(a * b)
    lo = rn32(a * b - p)
    q = rn32(p * c)
    ql = rn32(lo * c + rn32(p * c - q))
    return rn32(q + ql)


def _two_prod(a, b):
    p = rn32(a * b)
    return p, rn32(a * b - p)


def _df_add(x, y):
    s = rn32(x[0] + y[0])
    bv = rn32(s - x[0])
    av = rn32(s - bv)
    e = rn32(rn32(x[0] - av) + rn32(y[0] - bv))
    return s, rn32(e + rn32(x[1] + y[1]))


def _cross2x_df(u, v):
    """cross(u, v) of exact differences kept as a double-float, in the
    library's order: exact products of the values, their difference by
    TwoSum, plus the four remainder products."""
    (uxh, uxl), (uyh, uyl) = u
    (vxh, vxl), (vyh, vyl) = v
    a, b = _two_prod(uxh, vyh), _two_prod(uyh, vxh)
    s = _df_add(a, (-b[0], -b[1]))
    c = rn32(uxh * vyl + rn32(uxl * vyh + rn32(-uyh * vxl + rn32(-uyl * vxh))))
    return s[0], rn32(s[1] + c)


def _det2_df(a, b, c, d):
    """a d - b c of four double-floats (value, low part), rounded once, in
    the library's order: Kahan's determinant of the values plus the low
    parts' first-order terms."""
    w = rn32(b[0] * c[0])
    e = rn32(-b[0] * c[0] + w)
    f = rn32(a[0] * d[0] - w)
    r = rn32(a[0] * d[1] + rn32(a[1] * d[0] + rn32(-b[0] * c[1] + rn32(-b[1] * c[0]))))
    return rn32(f + rn32(e + r))


def _df_mul_round(x, y):
    p = rn32(x[0] * y[0])
    e = rn32(x[0] * y[1] + rn32(x[1] * y[0] + rn32(x[0] * y[0] - p)))
    return rn32(p + e)


def _dot2x_df(u, v):
    """u . v of exact differences as a double-float, in the library's order."""
    (uxh, uxl), (uyh, uyl) = u
    (vxh, vxl), (vyh, vyl) = v
    s = _df_add(_two_prod(uxh, vxh), _two_prod(uyh, vyh))
    c = rn32(uxh * vxl + rn32(uxl * vxh + rn32(uyh * vyl + rn32(uyl * vyh))))
    return s[0], rn32(s[1] + c)


def _sks_side(M, N, P, Q):
    """One side of the SKS kernel up to n7x, n7y (Eq. 6-11), in the library's
    order: ON = MN / 2 and the edges as exact differences, f_S, P3, Q3 and
    cross(ON, QP) as double-floats, then n7x as a determinant and n7y as a
    product of double-floats, each rounded once."""
    half = Fr(1, 2)
    onx = tuple(half * x for x in _diff(N[0], M[0]))
    ony = tuple(half * x for x in _diff(N[1], M[1]))
    on = (onx, ony)
    mp = (_diff(P[0], M[0]), _diff(P[1], M[1]))
    mq = (_diff(Q[0], M[0]), _diff(Q[1], M[1]))
    qp = (_diff(P[0], Q[0]), _diff(P[1], Q[1]))
    fS = _dot2x_df(on, on)
    P3y, Q3y = _cross2x_df(on, mp), _cross2x_df(on, mq)
    d = _dot2x_df(on, mp)
    P3x = _df_add(d, (-fS[0], -fS[1]))
    d = _dot2x_df(on, mq)
    Q3x = _df_add(d, (-fS[0], -fS[1]))
    cQP = _cross2x_df(on, qp)
    return _det2_df(Q3x, P3x, Q3y, P3y), _df_mul_round(fS, cQP)


def _side_points(rng, i):
    p = _f32(rng, 8, 0, 640)
    if i % 3 == 1:        # P close to the line MN: P3.y small against its terms
        t = rng.uniform(-1, 2)
        q = p[0:2] + t * (p[2:4] - p[0:2])
        p[4:6] = (q + rng.uniform(-0.5, 0.5, 2)).astype(np.float32)
    if i % 3 == 2:        # Q close to the line through O (the midpoint of MN) and P: P3, Q3
        o = 0.5 * (p[0:2].astype(np.float64) + p[2:4])      # nearly parallel, n7x cancels
        q = o + rng.uniform(0.3, 2.0) * (p[4:6] - o)
        p[6:8] = (q + rng.uniform(-1e-3, 1e-3, 2)).astype(np.float32)
    return p


def _f32(rng, n, lo=-700.0, hi=700.0):
    return rng.uniform(lo, hi, n).astype(np.float32)


def _check_rule(op, args, emulated):
    v, b = oracle.fp32_rule_bound(op, args)
    assert abs(float(emulated) - v) <= b * (1 + 1e-12) + 1e-300, (op, args, float(emulated), v, b)
    return abs(float(emulated) - v) / b if b > 0 else 0.0


def test_rounded_operations_within_their_rule():
    rng = np.random.default_rng(1)
    a, b, c = _f32(rng, 300), _f32(rng, 300), _f32(rng, 300)
    b[:100] = -a[:100] * np.float32(1 + 1e-6)             # cancellation
    for x, y, z in zip(a, b, c):
        X, Y, Z = Fr(float(x)), Fr(float(y)), Fr(float(z))
        _check_rule(0, [x, y], rn32(X + Y))
        _check_rule(1, [x, y], rn32(X * Y))
        _check_rule(2, [x, y, z], rn32(X * Y + Z))
        if y != 0:
            _check_rule(3, [x, y], rn32(X / Y))


def test_kahan_determinant_within_2u_even_under_cancellation():
    rng = np.random.default_rng(2)
    worst = 0.0
    for i in range(600):
        a, b, c = _f32(rng, 3)
        d = np.float32(float(b) * float(c) / float(a))     # a d close to b c
        if i % 3 == 0:
            d = np.float32(rng.uniform(-700, 700))
        A, B, C, D = (Fr(float(t)) for t in (a, b, c, d))
        if A * D - B * C == 0:
            continue
        worst = max(worst, _check_rule(4, [a, b, c, d], _kahan(A, B, C, D)))
    assert worst > 0.25          # the 2u bound is approached


def test_cross_product_of_exact_differences_within_its_rule():
    rng = np.random.default_rng(3)
    worst = 0.0
    for i in range(600):
        p = _f32(rng, 6, 0, 640)
        if i % 2 == 0:           # third point within a fraction of a pixel of the line
            t = rng.uniform(-2, 2)
            n = np.array([-(p[3] - p[1]), p[2] - p[0]], np.float64)
            n /= np.linalg.norm(n)
            q = p[:2] + t * (p[2:4] - p[:2]) + n * rng.uniform(-1e-2, 1e-2)
            p[4:6] = q.astype(np.float32)
        # u = N - M, v = P - M
        M, N, P = (Fr(float(p[0])), Fr(float(p[1]))), (Fr(float(p[2])), Fr(float(p[3]))), (Fr(float(p[4])), Fr(float(p[5])))
        u = (_diff(N[0], M[0]), _diff(N[1], M[1]))
        v = (_diff(P[0], M[0]), _diff(P[1], M[1]))
        got = _cross2x(u, v)
        worst = max(worst, _check_rule(5, [p[2], p[0], p[3], p[1], p[4], p[0], p[5], p[1]], got))
    assert worst > 0.1


def test_double_float_product_within_its_rule():
    rng = np.random.default_rng(4)
    for _ in range(400):
        a, b, c = _f32(rng, 3, -3e3, 3e3)
        _check_rule(6, [a, b, c], _df_prod_mul_round(Fr(float(a)), Fr(float(b)), Fr(float(c))))


def test_sks_n7_of_double_float_sides_within_their_rules():
    # n7x = Q3.x P3.y - P3.x Q3.y and n7y = f_S cross(ON, QP) of one side,
    # formed in the library's order from the double-float sides, on random
    # and cancellation-heavy point sets
    rng = np.random.default_rng(7)
    worst = [0.0, 0.0]
    for i in range(900):
        p = _side_points(rng, i)
        F = [Fr(float(x)) for x in p]
        n7x, n7y = _sks_side((F[0], F[1]), (F[2], F[3]), (F[4], F[5]), (F[6], F[7]))
        for k, (op, got) in enumerate(((7, n7x), (8, n7y))):
            v, b = oracle.fp32_rule_bound(op, p)
            if v == 0:
                continue
            assert abs(float(got) - v) <= b * (1 + 1e-12), (i, op, float(got), v, b)
            worst[k] = max(worst[k], abs(float(got) - v) / b)
    print(f"n7x worst error / bound {worst[0]:.3f}, n7y {worst[1]:.3f}")
    assert min(worst) > 0.1


def test_cross_product_kept_as_a_double_float_within_its_rule():
    # P3.y, Q3.y, cross(ON, QP) of the SKS kernel: the pair's value against
    # the exact cross product of the exact differences
    rng = np.random.default_rng(9)
    for i in range(600):
        p = _f32(rng, 6, 0, 640)
        if i % 2 == 0:
            t = rng.uniform(-2, 2)
            n = np.array([-(p[3] - p[1]), p[2] - p[0]], np.float64)
            n /= np.linalg.norm(n)
            q = p[:2] + t * (p[2:4] - p[:2]) + n * rng.uniform(-1e-2, 1e-2)
            p[4:6] = q.astype(np.float32)
        M, N, P = (Fr(float(p[0])), Fr(float(p[1]))), (Fr(float(p[2])), Fr(float(p[3]))), (Fr(float(p[4])), Fr(float(p[5])))
        u = (_diff(N[0], M[0]), _diff(N[1], M[1]))
        w = (_diff(P[0], M[0]), _diff(P[1], M[1]))
        h, lo = _cross2x_df(u, w)
        v, b = oracle.fp32_rule_bound(9, [p[2], p[0], p[3], p[1], p[4], p[0], p[5], p[1]])
        assert abs(float(h + lo - Fr(v))) <= b * (1 + 1e-12) + 1e-300, (i, float(h + lo), v, b)


# ---------------------------------------------------------------- whole chains
@pytest.fixture(scope="module")
def host():
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, f"libhost_fp32_{os.getpid()}.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                           os.path.join(HERE, "host_fp32.cpp"), "-o", so])
    L = ctypes.CDLL(so)
    os.remove(so)
    fp = ctypes.POINTER(ctypes.c_float)
    L.host_aca.argtypes = [fp, fp, ctypes.c_int64]
    L.host_sks.argtypes = [fp, fp, ctypes.c_int64]
    L.host_test_e.argtypes = [fp, fp, ctypes.c_int64, ctypes.c_float, fp, fp]
    return L


def _host_solve(L, name, pts):
    a = np.ascontiguousarray(pts.T.astype(np.float32))
    H = np.empty((a.shape[0], 9), np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    getattr(L, name)(a.ctypes.data_as(fp), H.ctypes.data_as(fp), a.shape[0])
    return H.astype(np.float64)


def _unit_err(a, b):
    a = a / np.linalg.norm(a, axis=1, keepdims=True)
    b = b / np.linalg.norm(b, axis=1, keepdims=True)
    a = a * np.sign(np.sum(a * b, axis=1, keepdims=True))
    return np.abs(a - b).max(axis=1)


@pytest.mark.parametrize("solver", ["aca", "sks"])
@pytest.mark.parametrize("seed,n,frac", [(0, 4096, 0.0), (11, 1 << 15, 0.01)])
def test_chain_bound_covers_the_fp32_evaluation(host, solver, seed, n, frac):
    ms = workloads.minimal_sets(n, seed=seed, degenerate_frac=frac)
    bound = oracle.aca_fp32_bound if solver == "aca" else oracle.sks_fp32_bound
    beta, Hv, He = bound(ms.pts, per_entry=True)
    ref = oracle.aca(ms.pts) if solver == "aca" else oracle.sks(ms.pts)
    assert _unit_err(Hv, ref).max() < 1e-8            # the chain computes the paper's H
    Hh = _host_solve(host, "host_" + solver, ms.pts)
    ent = np.abs(Hh - Hv)
    assert np.all(ent <= He * (1 + 1e-6)), float(np.max(ent / He))
    err = _unit_err(Hh, ref)
    assert np.all(err <= beta + beta ** 2), float(np.max(err / beta))
    ratio = err / beta
    print(f"{solver} seed {seed}: max err {err.max():.2e}, max bound {beta.max():.2e}, "
          f"max err/bound {ratio.max():.3f}, p99 {np.quantile(ratio, 0.99):.3f}")
    assert ratio.max() > 0.1
    if frac == 0.0:
        assert err.max() < 1e-4            # the library's FP32 arithmetic meets 1e-4 on every config-0 set


def test_inlier_test_bound_covers_the_fp32_evaluation(host):
    rp = workloads.ransac_problem(2000, 0.6, 1.0, seed=0)
    c = np.ascontiguousarray(rp.corr, np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    thr = 3.0
    flips = amb = tests = 0
    worst = 0.0
    for h in range(384):
        idx = oracle.sample4(2024, 0, h, 2000)
        s = np.concatenate([c[idx, :2].astype(np.float64).ravel(), c[idx, 2:].astype(np.float64).ravel()])
        if oracle.sample_degenerate(s):
            continue
        s32 = s.astype(np.float32)
        Hs = np.empty(9, np.float32)
        e = np.empty(2000, np.float32)
        host.host_test_e(s32.ctypes.data_as(fp), c.ctypes.data_as(fp), 2000, ctypes.c_float(thr),
                         Hs.ctypes.data_as(fp), e.ctypes.data_as(fp))
        E, B = oracle.score_bound_E(s, c, thr)
        _, Hv, _ = oracle.aca_fp32_bound(s.reshape(16, 1), per_entry=True)
        k = int(np.argmax(np.abs(Hv[0])))
        scale = 2.0 ** np.round(np.log2(abs(float(Hs[k]) / Hv[0, k])))      # exact power of two
        d = np.abs(e.astype(np.float64) / scale ** 2 - E)
        assert np.all(d <= B), (h, float(np.max(d / B)))
        worst = max(worst, float(np.max(d / B)))
        flip = (e < 0) != (E < 0)
        a = oracle.score_band(s, c, thr, band_px=0.0).astype(bool)
        assert not np.any(flip & ~a), h
        flips += int(flip.sum())
        amb += int(a.sum())
        tests += 2000
    print(f"inlier test: {tests} tests, {flips} FP32 decisions differ, {amb} in the derived band, "
          f"max error/bound {worst:.3f}")
    assert worst > 0.1
    assert amb < 1e-4 * tests


def _host_test_case(host, corr, s, thr):
    fp = ctypes.POINTER(ctypes.c_float)
    c = np.ascontiguousarray(corr, np.float32)
    s32 = np.asarray(s, np.float64).astype(np.float32)
    Hs = np.empty(9, np.float32)
    e = np.empty(c.shape[0], np.float32)
    host.host_test_e(s32.ctypes.data_as(fp), c.ctypes.data_as(fp), c.shape[0], ctypes.c_float(thr),
                     Hs.ctypes.data_as(fp), e.ctypes.data_as(fp))
    E, B = oracle.score_bound_E(s, c, thr)
    _, Hv, _ = oracle.aca_fp32_bound(np.asarray(s, np.float64).reshape(16, 1), per_entry=True)
    k = int(np.argmax(np.abs(Hv[0])))
    scale = 2.0 ** np.round(np.log2(abs(float(Hs[k]) / Hv[0, k])))
    return e.astype(np.float64) / scale ** 2, E, B


def test_inlier_test_bound_at_a_sample_point_near_the_vanishing_line(host):
    # pair 4 of this batch, hypotheses 226 and 227: the sample point M1 lies
    # next to the line that H maps to infinity (w' ~ 5e-8 at H's scale), so
    # E = -thr^2 w^2 is itself of second order; without the squares of the
    # errors of du, dv, w' in the bound, the FP32 test there is decided the
    # other way by more than the first-order bound
    rb = workloads.ransac_batch(P=16, seed=6, n_max=3000, cap=512)
    a, b = int(rb.offsets[4]), int(rb.offsets[5])
    c = rb.corr[a:b]
    for h in (226, 227):
        idx = oracle.sample4(99, 4, h, b - a)
        s = np.concatenate([c[idx, :2].astype(np.float64).ravel(), c[idx, 2:].astype(np.float64).ravel()])
        e, E, B = _host_test_case(host, c, s, 3.0)
        assert np.all(np.abs(e - E) <= B), h
        flip = (e < 0) != (E < 0)
        assert flip.any()                                   # FP32 does decide a point the other way
        assert np.all(oracle.score_band(s, c, 3.0, band_px=0.0).astype(bool)[flip])


def test_band_in_pixels_near_the_threshold():
    # the derived band converted to pixels of |r - thr| at points near the
    # threshold: a few 1e-4 px at image coordinates up to 640 (the FP32
    # rounding of u, v, w there is about 4e-5 px each)
    rp = workloads.ransac_problem(2000, 0.6, 1.0, seed=0)
    px = []
    for h in range(64):
        idx = oracle.sample4(2024, 0, h, 2000)
        s = np.concatenate([rp.corr[idx, :2].astype(np.float64).ravel(), rp.corr[idx, 2:].astype(np.float64).ravel()])
        if oracle.sample_degenerate(s):
            continue
        H = oracle.aca(s.reshape(16, 1))[0]
        x, y = rp.corr[:, 0].astype(np.float64), rp.corr[:, 1].astype(np.float64)
        w = H[6] * x + H[7] * y + H[8]
        r = np.hypot(rp.corr[:, 2] - (H[0] * x + H[1] * y + H[2]) / w, rp.corr[:, 3] - (H[3] * x + H[4] * y + H[5]) / w)
        near = np.abs(r - 3.0) < 0.5
        px.append(oracle.score_band_px(s, rp.corr, 3.0)[near])
    px = np.concatenate(px)
    med = float(np.median(px))
    print(f"band near the threshold: median {med:.2e} px, p99 {np.quantile(px, 0.99):.2e} px")
    assert 1e-5 < med < 1e-3


# ------------------------------------------------- the worst rounding corner
def _config0_sets(n):
    ms = workloads.minimal_sets(n, seed=0)
    return ms.pts


@pytest.mark.parametrize("solver", ["aca", "sks"])
def test_chain_bound_is_attained_at_its_worst_corner(solver):
    # F = sum g_i H_i for random g: re-running the chain with every event at
    # the sign of its weight times its bound moves F by the first-order bound
    # b1, up to the products of events (at most bound - b1); never beyond
    pts = _config0_sets(384)
    rng = np.random.default_rng(5)
    worst = 0.0
    for i in range(pts.shape[1]):
        b1, dev, bound = oracle.fp32_chain_corner(solver, pts[:, i], rng.standard_normal(9))
        assert abs(dev - b1) <= bound - b1, (i, dev / b1)
        assert dev <= bound
        worst = max(worst, abs(dev / b1 - 1))
    print(f"{solver}: worst corner within {worst:.1e} of the first-order bound")


def test_inlier_test_bound_is_attained_at_its_worst_corner():
    # the test with its hypothesis's solve: the solve's events and then the
    # test's at the signs of their weights move e by at most the bound B and
    # by at least 0.9 B (the rest of B is the token and the squares of the
    # bounds of du, dv, w')
    rp = workloads.ransac_problem(2000, 0.6, 1.0, seed=0)
    c = np.ascontiguousarray(rp.corr, np.float32)
    ratios = []
    for h in range(48):
        idx = oracle.sample4(2024, 0, h, 2000)
        s = np.concatenate([c[idx, :2].astype(np.float64).ravel(), c[idx, 2:].astype(np.float64).ravel()])
        if oracle.sample_degenerate(s):
            continue
        _, B = oracle.score_bound_E(s, c[::40], 3.0)
        for j, i in enumerate(range(0, 2000, 40)):
            b1, dev, _ = oracle.score_corner(s, c[i], 3.0)
            assert abs(dev) <= B[j], (h, i, dev / B[j])
            ratios.append(dev / B[j])
    ratios = np.asarray(ratios)
    print(f"inlier test worst corner / bound: min {ratios.min():.4f}, max {ratios.max():.6f}")
    assert ratios.min() > 0.9


def _test_corners(H, thr, c, d):
    """The inlier test's FP32 evaluation order (Sec. 6.2 test, threshold
    folded in) with each of its 17 roundings replaced by a factor (1 + d_k):
    d (17, m) holds m corners.  The inputs (H, thr, the point) are exact."""
    x, y, X, Y = (float(v) for v in c)
    rt = (1.0 / thr) * (1 + d[0])
    Xs, Ys = X * rt * (1 + d[1]), Y * rt * (1 + d[2])
    G6, G7, G8 = thr * H[6] * (1 + d[3]), thr * H[7] * (1 + d[4]), thr * H[8] * (1 + d[5])
    w = (G6 * x + (G7 * y + G8) * (1 + d[6])) * (1 + d[7])
    nu = (-H[0] * x + (-H[1] * y - H[2]) * (1 + d[8])) * (1 + d[9])
    nv = (-H[3] * x + (-H[4] * y - H[5]) * (1 + d[10])) * (1 + d[11])
    du, dv = (Xs * w + nu) * (1 + d[12]), (Ys * w + nv) * (1 + d[13])
    p = (w * -w) * (1 + d[14])
    return (du * du + (dv * dv + p) * (1 + d[15])) * (1 + d[16])


def test_inlier_test_bound_covers_every_corner_of_its_own_events():
    k = 17
    bits = (np.arange(1 << k)[None, :] >> np.arange(k)[:, None]) & 1
    d = (2.0 * bits - 1.0) * U                       # all 2^17 corners, (17, 2^17)
    zero = np.zeros((k, 1))
    rp = workloads.ransac_problem(2000, 0.6, 1.0, seed=0)
    c = np.ascontiguousarray(rp.corr, np.float32)
    x, y = c[:, 0].astype(np.float64), c[:, 1].astype(np.float64)
    near, other = [], []
    for h in range(8):
        idx = oracle.sample4(2024, 0, h, 2000)
        s = np.concatenate([c[idx, :2].astype(np.float64).ravel(), c[idx, 2:].astype(np.float64).ravel()])
        if oracle.sample_degenerate(s):
            continue
        H = oracle.aca(s.reshape(16, 1))[0]
        H = (H / np.abs(H).max()).astype(np.float32).astype(np.float64)       # an exact FP32 H
        _, B = oracle.score_bound_E_fixed(H, c, 3.0)
        w = H[6] * x + H[7] * y + H[8]
        r = np.hypot(c[:, 2] - (H[0] * x + H[1] * y + H[2]) / w, c[:, 3] - (H[3] * x + H[4] * y + H[5]) / w)
        order = np.argsort(np.abs(r - 3.0))
        rest = np.random.default_rng(h).choice(2000, 12, replace=False)
        for j, i in enumerate(list(order[:12]) + list(rest)):
            E = _test_corners(H, 3.0, c[i], zero)[0]
            m = float(np.max(np.abs(_test_corners(H, 3.0, c[i], d) - E)))
            assert m <= B[i], (h, i, m / B[i])
            (near if j < 12 else other).append(m / B[i])
    print(f"all corners / bound: near the threshold min {min(near):.4f}, elsewhere min {min(other):.4f}, "
          f"max {max(near + other):.7f}")
    assert min(near + other) > 0.9
