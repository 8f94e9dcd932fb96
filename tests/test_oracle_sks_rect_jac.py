"""Pins of the oracle's SKS (Sec. 3, Eq. 4-14), rectangle path (Sec. 5.3,
Eq. 39-42, Algorithm 1) and analytic Jacobian."""
import itertools
import random
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from oracle import exact
import workloads
from tests.test_oracle_aca import random_integer_sets


def _unit(H):
    H = np.asarray(H, dtype=np.float64).reshape(-1, 9)
    H = H / np.linalg.norm(H, axis=1, keepdims=True)
    return H * np.where(H[:, 8:9] < 0, -1.0, 1.0)


def _sks_defined(s):
    try:
        exact.sks(s)
        return True
    except ZeroDivisionError:
        return False


@pytest.mark.parametrize("s", [s for s in random_integer_sets(50, seed=21) if _sks_defined(s)][:40])
def test_exact_sks_proportional_to_exact_dlt(s):
    assert exact.proportional(exact.sks(s), exact.dlt(s))


@pytest.mark.parametrize("s", [s for s in random_integer_sets(30, seed=22) if _sks_defined(s)][:20])
def test_prop1_kernel_fixes_canonical_two_anchor_points(s):
    K = exact.sks_kernel(s)
    # Eq. 9 structure: k21 = k23 = 0, k11 = k33, k13 = k31 (Appendix A)
    assert K[3] == 0 and K[5] == 0 and K[0] == K[8] and K[2] == K[6]
    for x in (-1, 1):
        u, v, w = exact.apply(K, F(x), F(0))
        assert v == 0 and u == x * w


def test_fp64_oracle_sks_matches_dlt_on_workload():
    ms = workloads.minimal_sets(4096, seed=0)
    Hs = _unit(oracle.sks(ms.pts))
    Hd = _unit(oracle.dlt(ms.pts))
    assert np.max(np.abs(Hs - Hd)) < 1e-8


def _rect_sets(k, seed):
    rnd = random.Random(seed)
    out = []
    while len(out) < k:
        x0, y0 = rnd.randint(-50, 300), rnd.randint(-50, 300)
        w, h = rnd.randint(1, 200), rnd.randint(1, 200)
        src = [x0, y0, x0 + w, y0, x0, y0 + h, x0 + w, y0 + h]   # M, N, P, Q
        tgt = [src[i] + rnd.randint(-40, 40) for i in range(8)]
        s = src + tgt
        from tests.test_oracle_aca import _general_position
        if _general_position(s):
            out.append((s, (x0, y0, w, F(w, h))))
    return out


@pytest.mark.parametrize("s,rect", _rect_sets(30, 23))
def test_rect_eq42_proportional_to_general_aca(s, rect):
    H42 = exact.rect_eq42(s[8:], *rect)
    assert exact.proportional(H42, exact.aca(s))


def test_rect_alg1_and_eq42_agree_in_fp64():
    rb = workloads.rect_batch(1000, seed=3)
    H42 = oracle.aca_rect(rb.tgt, rb.rect)
    Ha1 = oracle.aca_rect_alg1(rb.tgt, rb.rect)
    pts = np.concatenate([np.repeat(rb.src_corners.reshape(8, 1), 1000, axis=1), rb.tgt], axis=0)
    Hg = oracle.aca(pts)
    assert np.max(np.abs(_unit(H42) - _unit(Ha1))) < 1e-12
    assert np.max(np.abs(_unit(H42) - _unit(Hg))) < 1e-12
    # Algorithm 1 as operations returns -H of Eq. 42 (its comments' signs aside)
    assert np.allclose(Ha1, -H42, rtol=1e-12, atol=1e-9 * np.abs(H42).max())


def test_oracle_rect_forms_on_rectangles_of_any_aspect_and_offset():
    # the C oracle's Eq. 42 and Algorithm 1 against its general ACA on
    # rectangles of every aspect ratio and offset (the 4-point-offset patch
    # of the differentiable workload is square, where the r and y0 terms of
    # Eq. 42 would go unseen)
    for s, (x0, y0, w, r) in _rect_sets(30, 31):
        tgt = np.array(s[8:], dtype=np.float64).reshape(8, 1)
        rect = (float(x0), float(y0), float(w), float(r))
        Hg = _unit(oracle.aca(np.array(s, dtype=np.float64).reshape(16, 1)))
        assert np.max(np.abs(_unit(oracle.aca_rect(tgt, rect)) - Hg)) < 1e-10, rect
        assert np.max(np.abs(_unit(oracle.aca_rect_alg1(tgt, rect)) - Hg)) < 1e-10, rect


def test_all_24_rectangle_corner_orders_give_the_same_h():
    # Appendix B: a pivot-free elimination fails for 8 of the 24 orders of a
    # rectangle's corners; ACA must give one H for all of them.
    for s, _ in _rect_sets(5, 24):
        base = exact.aca(s)
        for perm in itertools.permutations(range(4)):
            t = []
            for side in range(2):
                for k in perm:
                    t += [s[8 * side + 2 * k], s[8 * side + 2 * k + 1]]
            assert exact.proportional(exact.aca(t), base)


def _stencil_derivative(f, s, k, h=F(1, 3)):
    """Exact derivative of a polynomial of degree <= 4 in coordinate k."""
    def at(d):
        t = list(s)
        t[k] = t[k] + d
        return f(t)
    fp2, fp1, fm1, fm2 = at(2 * h), at(h), at(-h), at(-2 * h)
    return [(-fp2[i] + 8 * fp1[i] - 8 * fm1[i] + fm2[i]) / (12 * h) for i in range(9)]


def test_aca_jacobian_exact_against_polynomial_stencil():
    sets = random_integer_sets(6, seed=25)
    pts = np.array(sets, dtype=np.float64).T.copy()
    J = oracle.aca_jacobian(pts)
    for n, s in enumerate(sets):
        sF = [F(v) for v in s]
        for k in range(8):
            d = _stencil_derivative(exact.aca, sF, 8 + k)
            ref = np.array([float(x) for x in d])
            scale = max(1.0, np.abs(ref).max())
            assert np.max(np.abs(J[n, :, k] - ref)) <= 1e-13 * scale


def test_h_is_cubic_in_each_target_coordinate():
    # degree <= 3 per target coordinate: the 4th finite difference vanishes
    s = [F(v) for v in random_integer_sets(1, seed=26)[0]]
    for k in range(8, 16):
        vals = []
        for d in range(5):
            t = list(s)
            t[k] += d
            vals.append(exact.aca(t))
        fourth = [vals[4][i] - 4 * vals[3][i] + 6 * vals[2][i] - 4 * vals[1][i] + vals[0][i] for i in range(9)]
        assert all(x == 0 for x in fourth)


def test_rect_jacobian_exact_against_polynomial_stencil():
    for s, rect in _rect_sets(4, 27):
        tgt = np.array(s[8:], dtype=np.float64).reshape(8, 1)
        J = oracle.aca_rect_jacobian(tgt, [float(v) for v in rect])[0]
        f = lambda t: exact.rect_eq42(t, *rect)
        for k in range(8):
            d = _stencil_derivative(f, [F(v) for v in s[8:]], k)
            ref = np.array([float(x) for x in d])
            assert np.max(np.abs(J[:, k] - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


def test_aca_jacobian_matches_fp64_central_differences():
    ms = workloads.minimal_sets(64, seed=4)
    J = oracle.aca_jacobian(ms.pts)
    base = oracle.sets_aos(ms.pts)
    step = 1e-6
    for k in range(8):
        p = base.copy()
        m = base.copy()
        p[:, 8 + k] += step
        m[:, 8 + k] -= step
        Hp = oracle.aca(p.T.copy())
        Hm = oracle.aca(m.T.copy())
        fd = (Hp - Hm) / (2 * step)
        scale = np.abs(J).max(axis=(1, 2))[:, None]
        assert np.max(np.abs(fd - J[:, :, k]) / scale) < 1e-6


def test_source_jacobian_matches_fp64_central_differences():
    ms = workloads.minimal_sets(64, seed=12)
    J = oracle.aca_jacobian_src(ms.pts)
    base = oracle.sets_aos(ms.pts)
    step = 1e-6
    for k in range(8):
        p, m = base.copy(), base.copy()
        p[:, k] += step
        m[:, k] -= step
        fd = (oracle.aca(p.T.copy()) - oracle.aca(m.T.copy())) / (2 * step)
        scale = np.abs(J).max(axis=(1, 2))[:, None]
        assert np.max(np.abs(fd - J[:, :, k]) / scale) < 1e-6


def test_condition_number_bounds_and_is_attained_by_worst_sign_perturbation():
    ms = workloads.minimal_sets(200, seed=13)
    kap = oracle.aca_condition(ms.pts)
    s = oracle.sets_aos(ms.pts)
    H0 = oracle.aca(ms.pts)
    H0 = H0 / np.linalg.norm(H0, axis=1, keepdims=True)
    J = np.concatenate([oracle.aca_jacobian_src(ms.pts), oracle.aca_jacobian(ms.pts)], axis=2)
    delta = 1e-7
    rng = np.random.default_rng(0)
    for i in range(200):
        nrm = np.linalg.norm(oracle.aca(s[i].reshape(16, 1)))
        dhat = (J[i] - np.outer(H0[i], H0[i] @ J[i])) / nrm          # (9, 16)
        r = int(np.argmax(np.abs(dhat) @ np.abs(s[i])))
        worst = s[i] * (1 + delta * np.sign(dhat[r] * s[i]))          # relative perturbation
        Hw = oracle.aca(worst.reshape(16, 1))[0]
        Hw = Hw / np.linalg.norm(Hw) * np.sign(Hw @ H0[i])
        moved = abs(Hw[r] - H0[i][r])
        kd = kap[i] * delta          # first order; the rest is O(kd^2)
        assert abs(moved - kd) <= 1e-3 * kd + 10 * kd ** 2 + 1e-14
        rnd = s[i] * (1 + delta * rng.choice([-1.0, 1.0], 16))
        Hr = oracle.aca(rnd.reshape(16, 1))[0]
        Hr = Hr / np.linalg.norm(Hr) * np.sign(Hr @ H0[i])
        assert np.abs(Hr - H0[i]).max() <= kd * (1 + 1e-3) + 10 * kd ** 2 + 1e-14
