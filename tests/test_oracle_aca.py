"""Pins of the oracle's ACA (Sec. 4, Eq. 20-32) against what the paper and
the mathematics fix: uniqueness of the minimal solution (independent exact
DLT), the defining invariant x2 x (H x1) = 0, Prop. 4, special cases (Eq. 38,
identity), the division-form core (Eq. 26), the polynomial form (Eq. 30-32)
and correspondence-order invariance."""
import itertools
import random
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from oracle import exact
import workloads


def _general_position(s):
    pts1 = [(s[2 * k], s[2 * k + 1]) for k in range(4)]
    pts2 = [(s[8 + 2 * k], s[9 + 2 * k]) for k in range(4)]
    for pts in (pts1, pts2):
        for a, b, c in itertools.combinations(pts, 3):
            if (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]) == 0:
                return False
    return True


def random_integer_sets(k, seed=1, lo=0, hi=640):
    rnd = random.Random(seed)
    out = []
    while len(out) < k:
        s = [rnd.randint(lo, hi) for _ in range(16)]
        if _general_position(s):
            out.append(s)
    return out


def cross3(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


@pytest.mark.parametrize("s", random_integer_sets(60))
def test_exact_aca_proportional_to_exact_dlt(s):
    Ha = exact.aca(s)
    Hd = exact.dlt(s)
    assert Hd is not None
    assert exact.proportional(Ha, Hd)


@pytest.mark.parametrize("s", random_integer_sets(30, seed=2))
def test_exact_aca_maps_all_four_correspondences(s):
    H = exact.aca(s)
    assert any(h != 0 for h in H)
    for k in range(4):
        x1 = [F(s[2 * k]), F(s[2 * k + 1]), F(1)]
        x2 = [F(s[8 + 2 * k]), F(s[9 + 2 * k]), F(1)]
        Hx = list(exact.apply(H, x1[0], x1[1]))
        assert cross3(x2, Hx) == [0, 0, 0]


def test_exact_aca_invariant_under_24_orders():
    for s in random_integer_sets(6, seed=3):
        base = exact.aca(s)
        for perm in itertools.permutations(range(4)):
            t = []
            for side in range(2):
                for k in perm:
                    t += [s[8 * side + 2 * k], s[8 * side + 2 * k + 1]]
            assert exact.proportional(exact.aca(t), base)


@pytest.mark.parametrize("s", random_integer_sets(20, seed=4))
def test_prop4_core_fixes_canonical_anchor_points_and_maps_q3_to_q4(s):
    p = exact.aca_parts(s)
    c11, c22, c33 = p["c11"], p["c22"], p["c33"]
    HC = [c11, 0, 0, 0, c22, 0, c11 - c33, c22 - c33, c33]
    for (x, y) in ((0, 0), (1, 0), (0, 1)):
        u, v, w = exact.apply(HC, F(x), F(y))
        assert w != 0 and (u / w, v / w) == (x, y)
    # H_A1 sends M1, N1, P1 to the canonical HAP (Eq. 20)
    for k, (x, y) in zip(range(3), ((0, 0), (1, 0), (0, 1))):
        u, v, w = exact.apply(p["HA1"], F(s[2 * k]), F(s[2 * k + 1]))
        assert (u / w, v / w) == (x, y)
    # Q3 -> Q4 under H_C (Eq. 25-29)
    q3 = [p["Q3"][0], p["Q3"][1], p["fA1"]]
    q4 = [p["Q4"][0], p["Q4"][1], p["fA2"]]
    hq = [sum(HC[3 * i + j] * q3[j] for j in range(3)) for i in range(3)]
    assert cross3(hq, q4) == [0, 0, 0]


def test_affine_target_gives_identity_core():
    rnd = random.Random(5)
    for _ in range(20):
        src = random_integer_sets(1, seed=rnd.randint(0, 10**6))[0][:8]
        A = [rnd.randint(-5, 5) for _ in range(4)] + [rnd.randint(-50, 50), rnd.randint(-50, 50)]
        if A[0] * A[3] - A[1] * A[2] == 0:
            continue
        tgt = []
        for k in range(4):
            x, y = src[2 * k], src[2 * k + 1]
            tgt += [A[0] * x + A[1] * y + A[4], A[2] * x + A[3] * y + A[5]]
        s = src + tgt
        p = exact.aca_parts(s)
        assert p["c11"] == p["c22"] == p["c33"] != 0      # H_C = c I (Eq. 38)
        H = exact.aca(s)
        assert H[6] == 0 and H[7] == 0 and H[8] != 0


def test_identity_target_gives_multiple_of_identity():
    for s in random_integer_sets(10, seed=6):
        t = s[:8] + s[:8]
        H = exact.aca(t)
        assert exact.proportional(H, [1, 0, 0, 0, 1, 0, 0, 0, 1])


@pytest.mark.parametrize("s", random_integer_sets(20, seed=7))
def test_division_form_core_matches_division_free_core(s):
    p = exact.aca_parts(s)
    (Q3x, Q3y), (Q4x, Q4y) = p["Q3"], p["Q4"]
    if 0 in (Q3x, Q3y, p["t2"]):
        pytest.skip("division form undefined")
    aC = p["t1"] * Q4x / (p["t2"] * Q3x)
    bC = p["t1"] * Q4y / (p["t2"] * Q3y)
    c11, c22, c33 = p["c11"], p["c22"], p["c33"]
    assert exact.proportional([aC, 0, 0, 0, bC, 0, aC - 1, bC - 1, 1],
                              [c11, 0, 0, 0, c22, 0, c11 - c33, c22 - c33, c33])


def test_polynomial_form_eq30_with_corrected_third_column_and_degrees():
    sympy = pytest.importorskip("sympy")
    names = "M1x M1y N1x N1y P1x P1y Q1x Q1y M2x M2y N2x N2y P2x P2y Q2x Q2y"
    v = sympy.symbols(names)
    M1x, M1y, N1x, N1y, P1x, P1y, Q1x, Q1y, M2x, M2y, N2x, N2y, P2x, P2y, Q2x, Q2y = v
    # c11, c22, c33 as symbols (Eq. 25-29); the printed coefficient matrix
    # below is the independent part of this pin
    MN1x, MN1y, MP1x, MP1y = N1x - M1x, N1y - M1y, P1x - M1x, P1y - M1y
    MN2x, MN2y, MP2x, MP2y = N2x - M2x, N2y - M2y, P2x - M2x, P2y - M2y
    fA1 = MN1x * MP1y - MN1y * MP1x
    fA2 = MN2x * MP2y - MN2y * MP2x
    MQ1x, MQ1y, MQ2x, MQ2y = Q1x - M1x, Q1y - M1y, Q2x - M2x, Q2y - M2y
    Q3x, Q3y = MQ1x * MP1y - MQ1y * MP1x, MN1x * MQ1y - MN1y * MQ1x
    Q4x, Q4y = MQ2x * MP2y - MQ2y * MP2x, MN2x * MQ2y - MN2y * MQ2x
    t1, t2 = fA1 - Q3x - Q3y, fA2 - Q4x - Q4y
    c = sympy.Matrix([t1 * Q3y * Q4x, t1 * Q3x * Q4y, t2 * Q3x * Q3y])
    # The oracle's (Fraction) ACA evaluated at random rationals must equal
    # the printed polynomial form, with the c33 coefficients of h13, h23,
    # h33 read as f3 = N1.x P1.y - N1.y P1.x (the print shows f_A1 there).
    f1 = P1x * M1y - P1y * M1x
    f2 = M1x * N1y - M1y * N1x
    f3 = N1x * P1y - N1y * P1x
    Cm = sympy.Matrix([
        [N2x * (P1y - M1y), P2x * (M1y - N1y), M2x * (N1y - P1y)],
        [N2y * (P1y - M1y), P2y * (M1y - N1y), M2y * (N1y - P1y)],
        [(P1y - M1y), (M1y - N1y), (N1y - P1y)],
        [N2x * (M1x - P1x), P2x * (N1x - M1x), M2x * (P1x - N1x)],
        [N2y * (M1x - P1x), P2y * (N1x - M1x), M2y * (P1x - N1x)],
        [(M1x - P1x), (N1x - M1x), (P1x - N1x)],
        [N2x * f1, P2x * f2, M2x * f3],
        [N2y * f1, P2y * f2, M2y * f3],
        [f1, f2, f3]])
    col = Cm * c          # column-major h11 h21 h31 h12 h22 h32 h13 h23 h33
    rnd = random.Random(8)
    for _ in range(5):
        vals = [F(rnd.randint(-300, 300), rnd.randint(1, 7)) for _ in range(16)]
        H = exact.aca(vals)
        sub = dict(zip(v, vals))
        colv = [F(str(sympy.nsimplify(e.subs(sub)))) for e in col]
        rowmajor = [colv[0], colv[3], colv[6], colv[1], colv[4], colv[7], colv[2], colv[5], colv[8]]
        assert rowmajor == H
    # degrees of Eq. 32 (row-major): [[8,8,9],[8,8,9],[7,7,8]]
    degs = [sympy.Poly(sympy.expand(e), *v).total_degree() for e in col]
    assert degs == [8, 8, 7, 8, 8, 7, 9, 9, 8]
    # the printed c33 coefficient (f_A1 = M1N1 x M1P1 on h33) differs from f3
    assert sympy.expand(fA1 - f3) != 0


def test_exact_inverse_consistency():
    for s in random_integer_sets(10, seed=9):
        Hf = exact.aca(s)
        Hb = exact.aca(s[8:] + s[:8])
        P = exact._mm(Hb, Hf)
        assert exact.proportional(P, [1, 0, 0, 0, 1, 0, 0, 0, 1])


def _unit(H):
    H = np.asarray(H, dtype=np.float64).reshape(-1, 9)
    H = H / np.linalg.norm(H, axis=1, keepdims=True)
    return H * np.where(H[:, 8:9] < 0, -1.0, 1.0)


def test_fp64_oracle_aca_matches_exact_dlt_on_integer_sets():
    sets = random_integer_sets(40, seed=10)
    pts = np.array(sets, dtype=np.float64).T.copy()
    Ha = _unit(oracle.aca(pts))
    Hd = _unit(np.array([[float(x) for x in exact.dlt(s)] for s in sets]))
    assert np.max(np.abs(Ha - Hd)) < 1e-12


def test_fp64_oracle_aca_vs_dlt_and_divform_on_workload():
    ms = workloads.minimal_sets(4096, seed=0)
    Ha = _unit(oracle.aca(ms.pts))
    Hd = _unit(oracle.dlt(ms.pts))
    Hv = _unit(oracle.aca_divform(ms.pts))
    Ht = _unit(ms.H_true.reshape(-1, 9))
    assert np.max(np.abs(Ha - Hd)) < 1e-9
    assert np.max(np.abs(Ha - Hv)) < 1e-9
    # the generator's ground truth, up to the float32 rounding of the points
    # (clustered sets amplify the 3e-5 px input rounding to ~1e-3 of |H|)
    assert np.max(np.abs(Ha - Ht)) < 1e-2
    assert np.median(np.abs(Ha - Ht).max(axis=1)) < 1e-5


def test_fp64_oracle_reprojects_the_four_points():
    ms = workloads.minimal_sets(2048, seed=3)
    H = oracle.aca(ms.pts).reshape(-1, 3, 3)
    s = oracle.sets_aos(ms.pts)
    for k in range(4):
        x = np.stack([s[:, 2 * k], s[:, 2 * k + 1], np.ones(len(s))], axis=1)
        y = np.einsum("nij,nj->ni", H, x)
        err = np.hypot(y[:, 0] / y[:, 2] - s[:, 8 + 2 * k], y[:, 1] / y[:, 2] - s[:, 9 + 2 * k])
        assert err.max() < 1e-8


def _affine_sets(k, seed):
    rnd = random.Random(seed)
    out = []
    while len(out) < k:
        s = [rnd.randint(0, 640) for _ in range(12)]
        a = ((s[2] - s[0]) * (s[5] - s[1]) - (s[3] - s[1]) * (s[4] - s[0]))
        b = ((s[8] - s[6]) * (s[11] - s[7]) - (s[9] - s[7]) * (s[10] - s[6]))
        if a != 0 and b != 0:
            out.append(s)
    return out


@pytest.mark.parametrize("s", _affine_sets(20, 41))
def test_exact_affine_maps_the_three_points_and_equals_eq38_second_form(s):
    H = exact.affine(s)
    assert H[6] == 0 and H[7] == 0 and H[8] != 0
    for k in range(3):
        u, v, w = exact.apply(H, F(s[2 * k]), F(s[2 * k + 1]))
        assert (u / w, v / w) == (s[6 + 2 * k], s[7 + 2 * k])
    # Eq. 38 second form: [N2 P2 M2; 1 1 1] [N1 P1 M1; 1 1 1]^-1
    A2 = [s[8], s[10], s[6], s[9], s[11], s[7], 1, 1, 1]
    A1 = [s[2], s[4], s[0], s[3], s[5], s[1], 1, 1, 1]
    assert exact.proportional(H, exact._mm(A2, exact.inverse3(A1)))


def test_affine_equals_aca_for_an_affine_fourth_point():
    for s in _affine_sets(10, 42):
        H = exact.affine(s)
        # fourth correspondence Q consistent with the affine map
        q = (F(s[0] + s[2]) / 3 + 7, F(s[1] + s[5]) / 5 - 3)
        u, v, w = exact.apply(H, q[0], q[1])
        s16 = s[0:6] + [q[0], q[1]] + s[6:12] + [u / w, v / w]
        assert exact.proportional(exact.aca(s16), H)


def test_fp64_affine_oracle_matches_exact():
    sets = _affine_sets(50, 43)
    pts = np.array(sets, dtype=np.float64).T.copy()
    Ho = oracle.aca_affine(pts)
    for k, s in enumerate(sets):
        He = np.array([float(x) for x in exact.affine(s)])
        assert np.max(np.abs(Ho[k] - He)) <= 1e-12 * np.abs(He).max()
