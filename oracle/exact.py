"""Exact-rational (fractions.Fraction) versions of the solvers, used by the
oracle's pins.  TEST INFRASTRUCTURE ONLY (same rule as the rest of oracle/).

Each follows the same paper passage as its FP64 twin in oracle.c; over the
rationals there is no rounding, so the uniqueness of the minimal solution
(Sec. 2.1) makes ACA, SKS and the DLT agree exactly up to scale.
A set is a list of 16 numbers: M1 N1 P1 Q1 M2 N2 P2 Q2, (x, y) each.
"""
from __future__ import annotations

from fractions import Fraction as F


def _mm(A, B):
    return [sum(A[3 * i + k] * B[3 * k + j] for k in range(3)) for i in range(3) for j in range(3)]


def _mv(A, x):
    return [A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2] for i in range(3)]


def aca(s):
    """ACA, Eq. 20-29 (division-free core Eq. 28-29), unnormalised."""
    s = [F(v) for v in s]
    M1x, M1y, N1x, N1y, P1x, P1y, Q1x, Q1y, M2x, M2y, N2x, N2y, P2x, P2y, Q2x, Q2y = s
    MN1x, MN1y, MP1x, MP1y = N1x - M1x, N1y - M1y, P1x - M1x, P1y - M1y
    MN2x, MN2y, MP2x, MP2y = N2x - M2x, N2y - M2y, P2x - M2x, P2y - M2y
    fA1 = MN1x * MP1y - MN1y * MP1x
    fA2 = MN2x * MP2y - MN2y * MP2x
    MQ1x, MQ1y, MQ2x, MQ2y = Q1x - M1x, Q1y - M1y, Q2x - M2x, Q2y - M2y
    Q3x = MQ1x * MP1y - MQ1y * MP1x
    Q3y = MN1x * MQ1y - MN1y * MQ1x
    Q4x = MQ2x * MP2y - MQ2y * MP2x
    Q4y = MN2x * MQ2y - MN2y * MQ2x
    t1 = fA1 - Q3x - Q3y
    t2 = fA2 - Q4x - Q4y
    c11, c22, c33 = t1 * Q3y * Q4x, t1 * Q3x * Q4y, t2 * Q3x * Q3y
    HC = [c11, 0, 0, 0, c22, 0, c11 - c33, c22 - c33, c33]
    HA1 = _mm([MP1y, -MP1x, 0, -MN1y, MN1x, 0, 0, 0, fA1], [1, 0, -M1x, 0, 1, -M1y, 0, 0, 1])
    HA2inv = [MN2x, MP2x, M2x, MN2y, MP2y, M2y, 0, 0, 1]
    return _mm(_mm(HA2inv, HC), HA1)


def aca_parts(s):
    """Intermediate quantities of ACA (Eq. 20-29) for the special-case pins."""
    s = [F(v) for v in s]
    M1x, M1y, N1x, N1y, P1x, P1y, Q1x, Q1y, M2x, M2y, N2x, N2y, P2x, P2y, Q2x, Q2y = s
    MN1x, MN1y, MP1x, MP1y = N1x - M1x, N1y - M1y, P1x - M1x, P1y - M1y
    MN2x, MN2y, MP2x, MP2y = N2x - M2x, N2y - M2y, P2x - M2x, P2y - M2y
    fA1 = MN1x * MP1y - MN1y * MP1x
    fA2 = MN2x * MP2y - MN2y * MP2x
    MQ1x, MQ1y, MQ2x, MQ2y = Q1x - M1x, Q1y - M1y, Q2x - M2x, Q2y - M2y
    Q3x = MQ1x * MP1y - MQ1y * MP1x
    Q3y = MN1x * MQ1y - MN1y * MQ1x
    Q4x = MQ2x * MP2y - MQ2y * MP2x
    Q4y = MN2x * MQ2y - MN2y * MQ2x
    t1 = fA1 - Q3x - Q3y
    t2 = fA2 - Q4x - Q4y
    HA1 = _mm([MP1y, -MP1x, 0, -MN1y, MN1x, 0, 0, 0, fA1], [1, 0, -M1x, 0, 1, -M1y, 0, 0, 1])
    HA2inv = [MN2x, MP2x, M2x, MN2y, MP2y, M2y, 0, 0, 1]
    return dict(fA1=fA1, fA2=fA2, Q3=(Q3x, Q3y), Q4=(Q4x, Q4y), t1=t1, t2=t2,
                c11=t1 * Q3y * Q4x, c22=t1 * Q3x * Q4y, c33=t2 * Q3x * Q3y, HA1=HA1, HA2inv=HA2inv)


def dlt(s):
    """Eq. 2 stacked to the 8x8 inhomogeneous system (h33 = 1), Gaussian
    elimination with partial pivoting over the rationals.  None if singular."""
    s = [F(v) for v in s]
    A = []
    for k in range(4):
        x, y, X, Y = s[2 * k], s[2 * k + 1], s[8 + 2 * k], s[9 + 2 * k]
        A.append([x, y, F(1), F(0), F(0), F(0), -X * x, -X * y, X])
        A.append([F(0), F(0), F(0), -x, -y, F(-1), Y * x, Y * y, -Y])
    for c in range(8):
        piv = max(range(c, 8), key=lambda r: abs(A[r][c]))
        if A[piv][c] == 0:
            return None
        A[c], A[piv] = A[piv], A[c]
        for r in range(c + 1, 8):
            f = A[r][c] / A[c][c]
            for j in range(c, 9):
                A[r][j] -= f * A[c][j]
    h = [F(0)] * 8
    for r in range(7, -1, -1):
        acc = A[r][8] - sum(A[r][j] * h[j] for j in range(r + 1, 8))
        h[r] = acc / A[r][r]
    return h + [F(1)]


def sks(s):
    """SKS, Eq. 4-14."""
    s = [F(v) for v in s]
    M1x, M1y, N1x, N1y = s[0:4]
    M2x, M2y, N2x, N2y = s[8:12]
    half = F(1, 2)
    O1x, O1y = half * (M1x + N1x), half * (M1y + N1y)
    ON1x, ON1y = N1x - O1x, N1y - O1y
    O2x, O2y = half * (M2x + N2x), half * (M2y + N2y)
    ON2x, ON2y = N2x - O2x, N2y - O2y
    fS1 = ON1x ** 2 + ON1y ** 2
    fS2 = ON2x ** 2 + ON2y ** 2
    HS1 = _mm([ON1x, ON1y, 0, -ON1y, ON1x, 0, 0, 0, fS1], [1, 0, -O1x, 0, 1, -O1y, 0, 0, 1])
    HS2 = _mm([ON2x, ON2y, 0, -ON2y, ON2x, 0, 0, 0, fS2], [1, 0, -O2x, 0, 1, -O2y, 0, 0, 1])
    HS2inv = [ON2x, -ON2y, O2x, ON2y, ON2x, O2y, 0, 0, 1]
    P3 = _mv(HS1, [s[4], s[5], 1])
    Q3 = _mv(HS1, [s[6], s[7], 1])
    P4 = _mv(HS2, [s[12], s[13], 1])
    Q4 = _mv(HS2, [s[14], s[15], 1])
    P5 = (P3[0] / P3[1], P3[2] / P3[1])
    P6 = (P4[0] / P4[1], P4[2] / P4[1])
    Q7 = (Q3[0] / Q3[1] - P5[0], Q3[2] / Q3[1] - P5[1])
    Q8 = (Q4[0] / Q4[1] - P6[0], Q4[2] / Q4[1] - P6[1])
    det = Q7[0] ** 2 - Q7[1] ** 2
    aG = (Q8[0] * Q7[0] - Q8[1] * Q7[1]) / det
    bG = (Q8[1] * Q7[0] - Q8[0] * Q7[1]) / det
    uK = P6[0] - aG * P5[0] - bG * P5[1]
    vK = P6[1] - bG * P5[0] - aG * P5[1]
    HK = [aG, uK, bG, 0, 1, 0, bG, vK, aG]
    return _mm(_mm(HS2inv, HK), HS1)


def sks_kernel(s):
    """H_S2 * H * H_S1^-1 for the SKS H of a set: by Eq. 14 this is the kernel
    H_K of Eq. 9 up to scale (used by the Prop. 1 pin)."""
    s = [F(v) for v in s]
    H = sks(s)
    M1x, M1y, N1x, N1y = s[0:4]
    M2x, M2y, N2x, N2y = s[8:12]
    half = F(1, 2)
    O1x, O1y = half * (M1x + N1x), half * (M1y + N1y)
    ON1x, ON1y = N1x - O1x, N1y - O1y
    O2x, O2y = half * (M2x + N2x), half * (M2y + N2y)
    ON2x, ON2y = N2x - O2x, N2y - O2y
    HS1inv = [ON1x, -ON1y, O1x, ON1y, ON1x, O1y, 0, 0, 1]
    fS2 = ON2x ** 2 + ON2y ** 2
    HS2 = _mm([ON2x, ON2y, 0, -ON2y, ON2x, 0, 0, 0, fS2], [1, 0, -O2x, 0, 1, -O2y, 0, 0, 1])
    return _mm(_mm(HS2, H), HS1inv)


def rect_eq42(t, x0, y0, w, r):
    """Rectangle source, Eq. 42."""
    t = [F(v) for v in t]
    x0, y0, w, r = F(x0), F(y0), F(w), F(r)
    M2x, M2y, N2x, N2y, P2x, P2y, Q2x, Q2y = t
    MN2x, MN2y, MP2x, MP2y = N2x - M2x, N2y - M2y, P2x - M2x, P2y - M2y
    MQ2x, MQ2y = Q2x - M2x, Q2y - M2y
    fA2 = MN2x * MP2y - MN2y * MP2x
    Q4x = MQ2x * MP2y - MQ2y * MP2x
    Q4y = MN2x * MQ2y - MN2y * MQ2x
    t2 = fA2 - Q4x - Q4y
    A = [N2x, P2x, M2x, N2y, P2y, M2y, 1, 1, 1]
    B = [Q4x, 0, -Q4x * x0, 0, r * Q4y, -r * Q4y * y0, t2, r * t2, -t2 * (x0 + r * y0 + w)]
    return _mm(A, B)


def apply(H, x, y):
    """(u, v, w) = H (x, y, 1)."""
    return (H[0] * x + H[1] * y + H[2], H[3] * x + H[4] * y + H[5], H[6] * x + H[7] * y + H[8])


def proportional(A, B) -> bool:
    """A = lambda B for some nonzero rational lambda (exact)."""
    k = next(i for i in range(9) if B[i] != 0)
    if A[k] == 0:
        return False
    lam = F(A[k]) / F(B[k])
    return all(F(A[i]) == lam * F(B[i]) for i in range(9))


def affine(s12):
    """Eq. 38, first form: H_A2^-1 H_A1 (s12 = M1 N1 P1 M2 N2 P2)."""
    s12 = [F(v) for v in s12]
    M1x, M1y, N1x, N1y, P1x, P1y, M2x, M2y, N2x, N2y, P2x, P2y = s12
    MN1x, MN1y, MP1x, MP1y = N1x - M1x, N1y - M1y, P1x - M1x, P1y - M1y
    MN2x, MN2y, MP2x, MP2y = N2x - M2x, N2y - M2y, P2x - M2x, P2y - M2y
    fA1 = MN1x * MP1y - MN1y * MP1x
    HA1 = _mm([MP1y, -MP1x, 0, -MN1y, MN1x, 0, 0, 0, fA1], [1, 0, -M1x, 0, 1, -M1y, 0, 0, 1])
    return _mm([MN2x, MP2x, M2x, MN2y, MP2y, M2y, 0, 0, 1], HA1)


def inverse3(A):
    """Exact inverse of a 3x3 matrix (adjugate / determinant)."""
    a, b, c, d, e, f, g, h, i = [F(x) for x in A]
    det = a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g)
    adj = [e * i - f * h, c * h - b * i, b * f - c * e,
           f * g - d * i, a * i - c * g, c * d - a * f,
           d * h - e * g, b * g - a * h, a * e - b * d]
    return [x / det for x in adj]
