// FP32 minimal-solver arithmetic shared by the CUDA kernels of this library.
//
// ACA (Affine-Core-Affine, Sec. 4 of arXiv 2402.18008, Eq. 20-29) and SKS
// (Similarity-Kernel-Similarity, Sec. 3, Eq. 4-14) for one set of four
// correspondences M, N, P, Q (source side 1, target side 2), plus the
// rectangle-source form of Sec. 5.3 (Eq. 39-42).
//
// Numerical formulation (same H as the paper's, up to rounding):
//  * everything is computed in local frames anchored at M1 / M2 (ACA) or at
//    the midpoints O1 / O2 (SKS) and translated back at the end, i.e.
//    H = T(M2) * H_local * T(-M1); this is Eq. 24 regrouped by associativity;
//  * every 2x2 cross product uses Kahan's FMA determinant (fp32.cuh);
//  * t1 = f_A1 - Q3.x - Q3.y (Eq. 27) is evaluated as cross(N1P1, N1Q1), its
//    exact value (twice the signed area of N1 P1 Q1), so the sum does not
//    cancel; likewise t2;
//  * the core product (Eq. 28-29) and the local-frame composition (Eq. 24)
//    are carried in double-float and rounded once per entry (aca_compose).
// Unnormalised output (ACA_NORM_NONE) is the paper's division-free H of
// Eq. 24 with the scale of Eq. 28-29, the function the backward kernels
// differentiate.
// The ACA and SKS solves are written over a value type (fp32.cuh): float for
// one set, or packed pairs for two sets per instruction, with the same bits
// per lane.
#pragma once
#include <stdint.h>

#include "fp32.cuh"

namespace aca {

// One set (V = float) or two sets side by side (V = P2, see fp32.cuh).
template <class V>
struct SetT {
    V M1x, M1y, N1x, N1y, P1x, P1y, Q1x, Q1y;
    V M2x, M2y, N2x, N2y, P2x, P2y, Q2x, Q2y;
};
using Set = SetT<float>;

// Per-set flag bits (see include/aca.h).
enum : uint8_t {
    kFlagSrcAnchors = 1,   // source anchor triple M1 N1 P1 within 1 px of collinear
    kFlagTgtAnchors = 2,   // target anchor triple M2 N2 P2 within 1 px of collinear
    kFlagOtherTriple = 4,  // a triple containing Q within 1 px of collinear (either side)
    kFlagNonFinite = 8,    // a non-finite input or output
};

// Intermediates of the ACA chain kept for the flags and the backward pass.
template <class V>
struct AcaPartsT {
    V MN1x, MN1y, MP1x, MP1y, NP1x, NP1y;
    V MN2x, MN2y, MP2x, MP2y, MQ2x, MQ2y, NP2x, NP2y, NQ2x, NQ2y;
    V fA1, fA2, Q3x, Q3y, Q4x, Q4y, t1, t2;
    V MQ1x, MQ1y, NQ1x, NQ1y;
};
using AcaParts = AcaPartsT<float>;

// Eq. 20-27 (vectors, f_A, Q3, Q4, t1, t2) for one set.  Edge vectors are
// exact differences (value + remainder) and every cross product takes the
// remainders into account (cross2x), so f_A, Q3, Q4, t1, t2 are accurate to
// about one rounding of their exact values for the given inputs.
template <class V>
ACA_HD void aca_parts(const SetT<V> &s, AcaPartsT<V> &p)
{
    using Diff = DiffT<V>;
    const Diff mn1x = diff(s.N1x, s.M1x), mn1y = diff(s.N1y, s.M1y);
    const Diff mp1x = diff(s.P1x, s.M1x), mp1y = diff(s.P1y, s.M1y);
    const Diff mq1x = diff(s.Q1x, s.M1x), mq1y = diff(s.Q1y, s.M1y);
    const Diff np1x = diff(s.P1x, s.N1x), np1y = diff(s.P1y, s.N1y);
    const Diff nq1x = diff(s.Q1x, s.N1x), nq1y = diff(s.Q1y, s.N1y);
    const Diff mn2x = diff(s.N2x, s.M2x), mn2y = diff(s.N2y, s.M2y);
    const Diff mp2x = diff(s.P2x, s.M2x), mp2y = diff(s.P2y, s.M2y);
    const Diff mq2x = diff(s.Q2x, s.M2x), mq2y = diff(s.Q2y, s.M2y);
    const Diff np2x = diff(s.P2x, s.N2x), np2y = diff(s.P2y, s.N2y);
    const Diff nq2x = diff(s.Q2x, s.N2x), nq2y = diff(s.Q2y, s.N2y);
    p.MN1x = mn1x.h; p.MN1y = mn1y.h; p.MP1x = mp1x.h; p.MP1y = mp1y.h;
    p.MQ1x = mq1x.h; p.MQ1y = mq1y.h; p.NP1x = np1x.h; p.NP1y = np1y.h;
    p.NQ1x = nq1x.h; p.NQ1y = nq1y.h;
    p.MN2x = mn2x.h; p.MN2y = mn2y.h; p.MP2x = mp2x.h; p.MP2y = mp2y.h;
    p.MQ2x = mq2x.h; p.MQ2y = mq2y.h; p.NP2x = np2x.h; p.NP2y = np2y.h;
    p.NQ2x = nq2x.h; p.NQ2y = nq2y.h;
    p.fA1 = cross2x(mn1x, mn1y, mp1x, mp1y);   // Eq. 21
    p.fA2 = cross2x(mn2x, mn2y, mp2x, mp2y);
    p.Q3x = cross2x(mq1x, mq1y, mp1x, mp1y);   // Eq. 25
    p.Q3y = cross2x(mn1x, mn1y, mq1x, mq1y);
    p.Q4x = cross2x(mq2x, mq2y, mp2x, mp2y);
    p.Q4y = cross2x(mn2x, mn2y, mq2x, mq2y);
    p.t1 = cross2x(np1x, np1y, nq1x, nq1y);    // Eq. 27 (exact value)
    p.t2 = cross2x(np2x, np2y, nq2x, nq2y);
}

ACA_HD float fmax3_(float a, float b, float c);
ACA_HD float pow2_inv_scale(float x);

// Power-of-two factor bringing the largest of |a|, |b|, |c| into [1, 2).
ACA_HD float prescale_factor(float a, float b, float c) { return pow2_inv_scale(fmax3_(a, b, c)); }

// Core (Eq. 29) and composition (Eq. 24) from the parts, H row-major.
// The core c11, c22, c33 and the products of the local-frame homography
//   L = H_A2^-1(M2 frame) * H_C * H_A1(M1 frame)
// are carried in double-float and each entry of L is rounded once; the
// translation back, H = T(M2) L T(-M1), is plain FP32.  (Rounding c11, c22,
// c33 and the products c * M2N2 to FP32 instead roughly doubles the error of
// ill-conditioned sets; carrying the translation in double-float as well
// changes nothing measurable.)
// H_C * A1 rows with A1 = [[MP1.y, -MP1.x], [-MN1.y, MN1.x]] (Eq. 20); the
// third row is c11*a0 + c22*a1 + c33*(-NP1.y, NP1.x, f_A1), which equals
// (c11-c33)*a0 + (c22-c33)*a1 + c33*(0, 0, f_A1) of Eq. 28 exactly.  The
// left factor H_A2^-1 (Eq. 22) in the M2 frame is [[MN2.x, MP2.x],
// [MN2.y, MP2.y]].  With `prescale`, (c11, c22, c33) are first multiplied by
// a power of two (exact) so that the largest has magnitude in [1, 2): H
// changes by that exact factor only, and normalised outputs stay clear of
// overflow.
template <class V>
ACA_HD void aca_compose(const SetT<V> &s, const AcaPartsT<V> &p, bool prescale, V H[9])
{
    using DF = DFT<V>;
    DF c11 = df_mul(df_prod(p.t1, p.Q3y), p.Q4x);
    DF c22 = df_mul(df_prod(p.t1, p.Q3x), p.Q4y);
    DF c33 = df_mul(df_prod(p.t2, p.Q3x), p.Q3y);
    if (prescale) {
        const V sc = prescale_factor(c11.h, c22.h, c33.h);
        c11 = DF{vmul(c11.h, sc), vmul(c11.l, sc)};
        c22 = DF{vmul(c22.h, sc), vmul(c22.l, sc)};
        c33 = DF{vmul(c33.h, sc), vmul(c33.l, sc)};
    }
    const DF k0x = df_mul(c11, p.MN2x), k0y = df_mul(c11, p.MN2y);
    const DF k1x = df_mul(c22, p.MP2x), k1y = df_mul(c22, p.MP2y);
    const V L00 = df_round(df_sub(df_mul(k0x, p.MP1y), df_mul(k1x, p.MN1y)));
    const V L01 = df_round(df_sub(df_mul(k1x, p.MN1x), df_mul(k0x, p.MP1x)));
    const V L10 = df_round(df_sub(df_mul(k0y, p.MP1y), df_mul(k1y, p.MN1y)));
    const V L11 = df_round(df_sub(df_mul(k1y, p.MN1x), df_mul(k0y, p.MP1x)));
    const V L20 = df_round(df_sub(df_sub(df_mul(c11, p.MP1y), df_mul(c22, p.MN1y)), df_mul(c33, p.NP1y)));
    const V L21 = df_round(df_add(df_sub(df_mul(c22, p.MN1x), df_mul(c11, p.MP1x)), df_mul(c33, p.NP1x)));
    const V L22 = df_round(df_mul(c33, p.fA1));
    const V G02 = vneg(vfma(s.M1x, L00, vmul(s.M1y, L01)));
    const V G12 = vneg(vfma(s.M1x, L10, vmul(s.M1y, L11)));
    const V G22 = vfma(vneg(s.M1x), L20, vfma(vneg(s.M1y), L21, L22));
    H[0] = vfma(s.M2x, L20, L00);
    H[1] = vfma(s.M2x, L21, L01);
    H[2] = vfma(s.M2x, G22, G02);
    H[3] = vfma(s.M2y, L20, L10);
    H[4] = vfma(s.M2y, L21, L11);
    H[5] = vfma(s.M2y, G22, G12);
    H[6] = L20;
    H[7] = L21;
    H[8] = G22;
}

ACA_HD uint32_t f2u(float x)
{
#if defined(__CUDA_ARCH__)
    return __float_as_uint(x);
#else
    uint32_t u;
    __builtin_memcpy(&u, &x, 4);
    return u;
#endif
}

ACA_HD float u2f(uint32_t u)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(u);
#else
    float x;
    __builtin_memcpy(&x, &u, 4);
    return x;
#endif
}

// Power of two 2^-e where 2^e <= |x| < 2^(e+1), for normal finite x != 0
// (exact scale factor); 1 for 0, subnormal or non-finite x.
ACA_HD float pow2_inv_scale(float x)
{
    const int e = (int)((f2u(x) >> 23) & 0xffu) - 127;
    if (e == -127 || e == 128)
        return 1.0f;
    const int b = 127 - e;                 // in [0, 253]
    return b > 0 ? u2f((uint32_t)b << 23) : 1.0f;
}

ACA_HD float fabs_(float x) { return x < 0 ? -x : x; }

ACA_HD float fmax3_(float a, float b, float c)
{
    a = fabs_(a); b = fabs_(b); c = fabs_(c);
    const float m = a > b ? a : b;
    return m > c ? m : c;
}

// pow2_inv_scale lane by lane (one set, or each set of a packed pair).
ACA_HD float vpow2_inv_scale(float x) { return pow2_inv_scale(x); }
#if defined(__CUDACC__)
__device__ __forceinline__ P2 vpow2_inv_scale(P2 x)
{
    float a, b;
    vunpack(x, a, b);
    return vpack(pow2_inv_scale(a), pow2_inv_scale(b));
}
#endif

// Largest |entry| of H.
ACA_HD float max_abs9(const float H[9])
{
    float m = 0.0f;
    for (int i = 0; i < 9; ++i) { const float a = fabs_(H[i]); m = a > m ? a : m; }
    return m;
}

// Normalisations (Sec. 3.4: "generally based on h33", 1 division + 8 mults).
ACA_HD void normalize_h33(float H[9])
{
    const float r = F_DIV(1.0f, H[8]);
    for (int i = 0; i < 8; ++i) H[i] = F_MUL(H[i], r);
    H[8] = 1.0f;
}

// Unit Frobenius norm, sign so that h33 > 0 (or, when |h33| < 1e-6 |H|, so
// that the entry of largest magnitude is positive).  Pre-scaled by a power of
// two so the sum of squares cannot overflow.
ACA_HD void normalize_frob(float H[9])
{
    const float m = max_abs9(H);
    if (!(m > 0) || !(m < 3.0e38f)) return;
    const float sc = pow2_inv_scale(m);
    float h[9];
    float ss = 0.0f;
    int big = 0;
    for (int i = 0; i < 9; ++i) {
        h[i] = F_MUL(H[i], sc);
        ss = F_FMA(h[i], h[i], ss);
        if (fabs_(h[i]) > fabs_(h[big])) big = i;
    }
    const float nrm = F_SQRT(ss);
    const float inv = F_DIV(1.0f, nrm);
    const bool use33 = fabs_(h[8]) >= F_MUL(1e-6f, nrm);
    const float sgn = use33 ? (h[8] > 0 ? 1.0f : -1.0f) : (h[big] > 0 ? 1.0f : -1.0f);
    const float f = F_MUL(sgn, inv);
    for (int i = 0; i < 9; ++i) H[i] = F_MUL(h[i], f);
}

ACA_HD float sq2(float x, float y) { return F_FMA(x, x, F_MUL(y, y)); }

// |cross| < 1 px * longest side  <=>  cross^2 < max(|a|^2, |b|^2, |a-b|^2).
ACA_HD bool near_collinear(float cr, float la, float lb, float lc)
{
    float L = la > lb ? la : lb;
    L = L > lc ? L : lc;
    return F_MUL(cr, cr) < L;
}


// Flag bits 1, 2 and 4 (the near-collinear triples).
ACA_HD uint8_t aca_geom_flags(const Set &s, const AcaParts &p)
{
    uint8_t f = 0;
    const float lMN1 = sq2(p.MN1x, p.MN1y), lMP1 = sq2(p.MP1x, p.MP1y), lNP1 = sq2(p.NP1x, p.NP1y);
    const float lMQ1 = sq2(p.MQ1x, p.MQ1y), lNQ1 = sq2(p.NQ1x, p.NQ1y);
    const float PQ1x = F_SUB(s.Q1x, s.P1x), PQ1y = F_SUB(s.Q1y, s.P1y), lPQ1 = sq2(PQ1x, PQ1y);
    const float lMN2 = sq2(p.MN2x, p.MN2y), lMP2 = sq2(p.MP2x, p.MP2y), lNP2 = sq2(p.NP2x, p.NP2y);
    const float lMQ2 = sq2(p.MQ2x, p.MQ2y), lNQ2 = sq2(p.NQ2x, p.NQ2y);
    const float PQ2x = F_SUB(s.Q2x, s.P2x), PQ2y = F_SUB(s.Q2y, s.P2y), lPQ2 = sq2(PQ2x, PQ2y);
    if (near_collinear(p.fA1, lMN1, lMP1, lNP1)) f |= kFlagSrcAnchors;
    if (near_collinear(p.fA2, lMN2, lMP2, lNP2)) f |= kFlagTgtAnchors;
    if (near_collinear(p.Q3x, lMQ1, lMP1, lPQ1) || near_collinear(p.Q3y, lMN1, lMQ1, lNQ1) ||
        near_collinear(p.t1, lNP1, lNQ1, lPQ1) || near_collinear(p.Q4x, lMQ2, lMP2, lPQ2) ||
        near_collinear(p.Q4y, lMN2, lMQ2, lNQ2) || near_collinear(p.t2, lNP2, lNQ2, lPQ2))
        f |= kFlagOtherTriple;
    return f;
}

// All flag bits; bit 8 marks a non-finite input or output: x * 0 + z is z for
// every finite x and NaN otherwise, so one FMA per value decides it.
ACA_HD uint8_t aca_flags(const Set &s, const AcaParts &p, const float H[9])
{
    uint8_t f = aca_geom_flags(s, p);
    const float *sv = &s.M1x;
    float z = 0.0f;
    for (int i = 0; i < 16; ++i) z = F_FMA(sv[i], 0.0f, z);
    for (int i = 0; i < 9; ++i) z = F_FMA(H[i], 0.0f, z);
    if (!(z == 0.0f)) f |= kFlagNonFinite;
    return f;
}

// ---------------------------------------------------------------------------
// SKS (Sec. 3, Eq. 4-14).
//
// The steps of the paper, rewritten with identities that remove the
// cancellations an FP32 evaluation would suffer (all exact in real
// arithmetic; O = midpoint of MN, ON = MN / 2):
//   P3 = H_S1 P1 = (ON.(P1 - O1), ON x (P1 - O1), f_S1) with
//     ON x (P1 - O1) = ON x M1P1 and ON.(P1 - O1) = ON.M1P1 - f_S1 (Eq. 6-7);
//   P5 = (P3.x, f_S1) / P3.y, Q7 = (Q3.x, f_S1) / Q3.y - P5 (Eq. 10-11) with
//     Q7.x = (Q3.x P3.y - P3.x Q3.y) / (Q3.y P3.y),
//     Q7.y = f_S1 (P3.y - Q3.y) / (Q3.y P3.y), P3.y - Q3.y = ON x Q1P1;
//   a_K, b_K of Eq. 11 and u_K, v_K of Eq. 13 over their common
//   denominator: with Q7 = (n7x, n7y) / d7, Q8 = (n8x, n8y) / d8 (d7 =
//   Q3.y P3.y, d8 likewise), A = n8x n7x - n8y n7y, B = n8y n7x - n8x n7y,
//   m = n7x^2 - n7y^2, and P5, P6 the dehomogenised P3, P4, the kernel
//   H_K = [[a_K, u_K, b_K], [0, 1, 0], [b_K, v_K, a_K]] times
//   D = Q4.y P4.y m is
//     K = [[a3, u3, b3], [0, D, 0], [b3, v3, a3]],
//     a3 = Q3.y P3.y A,  b3 = Q3.y P3.y B,
//     u3 = P4.x Q4.y m - Q3.y (A P3.x + B f_S1),
//     v3 = f_S2 Q4.y m - Q3.y (B P3.x + A f_S1),
//   the same H up to scale without a single division.  m, the determinant
//   of Eq. 11, vanishes where the SKS parameterisation (not the map) is
//   singular; dividing by it there amplified the rounding of P3, Q3, while
//   in K it only enters as a term.  P3, Q3, f_S and ON x QP are kept as
//   double-floats, and n7, n8 are formed from them and rounded once: where
//   Q7 and Q8 are nearly parallel, B cancels to a small part of its terms
//   and magnifies the rounding of its inputs (on the set of the 4096-set
//   test workload where this is worst, 1.99e-4 of |H| with FP32 sides,
//   7.5e-5 with these).  The quantities of each side are scaled by one
//   power of two k (exact), n7 and n8 by k^2, so that f_S lies in [1, 2):
//   H_K is invariant under it and the products stay far from overflow;
//   H = H_S2^-1 K H_S1 (Eq. 14) composed in the M frames in FP32 (the
//   local map's two zero entries not formed), then translated back in FP32.
// Differences are exact (TwoSum) and dot / cross products of them carry
// their remainders.
// ---------------------------------------------------------------------------
template <class V>
struct SksSide {
    DiffT<V> onx, ony;       // ON = M N / 2
    DFT<V> fS2;              // |ON|^2
    DFT<V> P3x2, P3y2, Q3x2, Q3y2;
    DFT<V> cQP2;             // ON x Q P (= P3.y - Q3.y)
    V fS, P3x, P3y, Q3y;     // the same, rounded once
};

template <class V>
ACA_HD void sks_side(V Mx, V My, V Nx, V Ny, V Px, V Py, V Qx, V Qy, SksSide<V> &o)
{
    o.onx = half(diff(Nx, Mx));
    o.ony = half(diff(Ny, My));
    const DiffT<V> mpx = diff(Px, Mx), mpy = diff(Py, My);
    const DiffT<V> mqx = diff(Qx, Mx), mqy = diff(Qy, My);
    const DiffT<V> qpx = diff(Px, Qx), qpy = diff(Py, Qy);
    o.fS2 = dot2x_df(o.onx, o.ony, o.onx, o.ony);
    o.P3y2 = cross2x_df(o.onx, o.ony, mpx, mpy);
    o.Q3y2 = cross2x_df(o.onx, o.ony, mqx, mqy);
    o.P3x2 = df_sub(dot2x_df(o.onx, o.ony, mpx, mpy), o.fS2);
    o.Q3x2 = df_sub(dot2x_df(o.onx, o.ony, mqx, mqy), o.fS2);
    o.cQP2 = cross2x_df(o.onx, o.ony, qpx, qpy);
    o.fS = df_round(o.fS2);
    o.P3x = df_round(o.P3x2);
    o.P3y = df_round(o.P3y2);
    o.Q3y = df_round(o.Q3y2);
}

template <class V>
ACA_HD void sks_solve(const SetT<V> &s, V H[9])
{
    SksSide<V> a, b;
    sks_side(s.M1x, s.M1y, s.N1x, s.N1y, s.P1x, s.P1y, s.Q1x, s.Q1y, a);
    sks_side(s.M2x, s.M2y, s.N2x, s.N2y, s.P2x, s.P2y, s.Q2x, s.Q2y, b);
    // each side's P3, Q3, f_S scaled by one power of two k (H_K is
    // invariant); the unscaled f_S1 stays for H_S1 below
    const V ka = vpow2_inv_scale(a.fS), kb = vpow2_inv_scale(b.fS);
    const V ka2 = vmul(ka, ka), kb2 = vmul(kb, kb);
    const V aP3x = vmul(a.P3x, ka), aP3y = vmul(a.P3y, ka), aQ3y = vmul(a.Q3y, ka), afS = vmul(a.fS, ka);
    const V bP3x = vmul(b.P3x, kb), bP3y = vmul(b.P3y, kb), bQ3y = vmul(b.Q3y, kb), bfS = vmul(b.fS, kb);
    // Q7 = (n7x, n7y) / d7, Q8 = (n8x, n8y) / d8 (Eq. 10-11), of degree 2
    // in a side's quantities: each formed from the double-float sides,
    // rounded once, then scaled by k^2 (exact)
    const V n7x = vmul(det2_df(a.Q3x2, a.P3x2, a.Q3y2, a.P3y2), ka2), n7y = vmul(df_mul_round(a.fS2, a.cQP2), ka2);
    const V n8x = vmul(det2_df(b.Q3x2, b.P3x2, b.Q3y2, b.P3y2), kb2), n8y = vmul(df_mul_round(b.fS2, b.cQP2), kb2);
    // Eq. 11 and Eq. 13 over the common denominator Q4.y P4.y m
    const V A = det2(n8x, n8y, n7y, n7x), B = det2(n8y, n8x, n7y, n7x);
    const V m = vmul(vsub(n7x, n7y), vadd(n7x, n7y));
    const V q = vmul(aQ3y, aP3y), bm = vmul(bQ3y, m);
    const V aK = vmul(q, A), bK = vmul(q, B), dK = vmul(bP3y, bm);
    const V uK = vfma(bP3x, bm, vneg(vmul(aQ3y, vfma(A, aP3x, vmul(B, afS)))));
    const V vK = vfma(bfS, bm, vneg(vmul(aQ3y, vfma(B, aP3x, vmul(A, afS)))));
    // Eq. 14 in the M frames: H = T(M2) L T(-M1) with
    // L = T(ON2) R2^-1 K R1 T(-ON1), R1 = [[ONx, ONy, 0], [-ONy, ONx, 0], [0, 0, fS1]],
    // R2^-1 = [[ONx, -ONy, 0], [ONy, ONx, 0], [0, 0, 1]], K = [[aK, uK, bK], [0, dK, 0], [bK, vK, aK]].
    const V o1x = a.onx.h, o1y = a.ony.h, o2x = b.onx.h, o2y = b.ony.h;
    // K R1 (rows); row 1 of K R1 is dK (-o1y, o1x, 0).  The composition is
    // plain FP32: carried in double-float it changed no aggregate of the
    // error against the FP64 oracle (measured with FP32 sides: config 0 max
    // 1.97e-4 against 1.99e-4; 2^18 sets: the same 56 above 1e-4, max 1.87e-3
    // against 1.86e-3), whose size comes from the sides and the kernel.
    const V A00 = vfma(aK, o1x, vneg(vmul(uK, o1y)));
    const V A01 = vfma(aK, o1y, vmul(uK, o1x));
    const V A20 = vfma(bK, o1x, vneg(vmul(vK, o1y)));
    const V A21 = vfma(bK, o1y, vmul(vK, o1x));
    const V A22 = vmul(aK, a.fS);
    const V D1x = vmul(dK, o1x), D1y = vmul(dK, o1y);
    // R2^-1 (K R1), the first two columns
    const V L00 = vfma(A00, o2x, vmul(D1y, o2y));
    const V L01 = vfma(A01, o2x, vneg(vmul(D1x, o2y)));
    const V L10 = vfma(A00, o2y, vneg(vmul(D1y, o2x)));
    const V L11 = vfma(A01, o2y, vmul(D1x, o2x));
    // fold T(-ON1) on the right (column 3 -= ON1.x col 1 + ON1.y col 2) and
    // T(ON2) on the left (rows 1, 2 += ON2 * row 3).  J maps M1 to M2, the
    // origins of the two M frames, so its column 3 is (0, 0, J22): the first
    // two entries, differences of terms that cancel exactly, are not formed.
    const V j22 = vfma(vneg(A20), o1x, vfma(vneg(A21), o1y, A22));
    const V j00 = vfma(A20, o2x, L00), j01 = vfma(A21, o2x, L01);
    const V j10 = vfma(A20, o2y, L10), j11 = vfma(A21, o2y, L11);
    const V j20 = A20, j21 = A21;
    // then H = T(M2) J T(-M1) in FP32, as for ACA
    const V nM1x = vneg(s.M1x), nM1y = vneg(s.M1y);
    const V K02 = vfma(nM1x, j00, vmul(nM1y, j01));
    const V K12 = vfma(nM1x, j10, vmul(nM1y, j11));
    const V K22 = vfma(nM1x, j20, vfma(nM1y, j21, j22));
    H[0] = vfma(s.M2x, j20, j00);
    H[1] = vfma(s.M2x, j21, j01);
    H[2] = vfma(s.M2x, K22, K02);
    H[3] = vfma(s.M2y, j20, j10);
    H[4] = vfma(s.M2y, j21, j11);
    H[5] = vfma(s.M2y, K22, K12);
    H[6] = j20;
    H[7] = j21;
    H[8] = K22;
}

// ---------------------------------------------------------------------------
// Affine map from three correspondences (Sec. 5.2, Eq. 38): H_A = H_A2^-1
// H_A1, the ACA chain with the identity core.  In the anchor frames it is
// L = [[M2N2.x, M2P2.x], [M2N2.y, M2P2.y]] [[M1P1.y, -M1P1.x], [-M1N1.y,
// M1N1.x]] with f_A1 in the corner; each entry of L is a 2x2 determinant of
// exact differences (compensated), and the translation column
// M2 f_A1 - L M1 is summed in double-float.  Third row (0, 0, f_A1).
// ---------------------------------------------------------------------------
struct Set3 {
    float M1x, M1y, N1x, N1y, P1x, P1y;
    float M2x, M2y, N2x, N2y, P2x, P2y;
};

ACA_HD void affine_solve(const Set3 &s, float H[9])
{
    const Diff mn1x = diff(s.N1x, s.M1x), mn1y = diff(s.N1y, s.M1y);
    const Diff mp1x = diff(s.P1x, s.M1x), mp1y = diff(s.P1y, s.M1y);
    const Diff mn2x = diff(s.N2x, s.M2x), mn2y = diff(s.N2y, s.M2y);
    const Diff mp2x = diff(s.P2x, s.M2x), mp2y = diff(s.P2y, s.M2y);
    const float fA1 = cross2x(mn1x, mn1y, mp1x, mp1y);            // Eq. 21
    const float L00 = cross2x(mn2x, mp2x, mn1y, mp1y);            // MN2x MP1y - MP2x MN1y
    const float L01 = cross2x(mp2x, mn2x, mp1x, mn1x);            // MP2x MN1x - MN2x MP1x
    const float L10 = cross2x(mn2y, mp2y, mn1y, mp1y);
    const float L11 = cross2x(mp2y, mn2y, mp1x, mn1x);
    const DF t0 = df_sub(df_sub(df_prod(s.M2x, fA1), df_prod(s.M1x, L00)), df_prod(s.M1y, L01));
    const DF t1 = df_sub(df_sub(df_prod(s.M2y, fA1), df_prod(s.M1x, L10)), df_prod(s.M1y, L11));
    H[0] = L00;
    H[1] = L01;
    H[2] = df_round(t0);
    H[3] = L10;
    H[4] = L11;
    H[5] = df_round(t1);
    H[6] = 0.0f;
    H[7] = 0.0f;
    H[8] = fA1;
}

// ---------------------------------------------------------------------------
// Rectangle source (Sec. 5.3, Eq. 39-42): M1 = (x0, y0) upper-left corner,
// width w, aspect ratio r = width / height; target corners M2 N2 P2 Q2.
// ---------------------------------------------------------------------------
struct Rect {
    float x0, y0, w, r;
};

struct RectParts {
    float MN2x, MN2y, MP2x, MP2y, MQ2x, MQ2y, NP2x, NP2y, NQ2x, NQ2y;
    float fA2, Q4x, Q4y, t2;
};

ACA_HD void rect_parts(const float t[8], RectParts &p)
{
    p.MN2x = F_SUB(t[2], t[0]); p.MN2y = F_SUB(t[3], t[1]);
    p.MP2x = F_SUB(t[4], t[0]); p.MP2y = F_SUB(t[5], t[1]);
    p.MQ2x = F_SUB(t[6], t[0]); p.MQ2y = F_SUB(t[7], t[1]);
    p.NP2x = F_SUB(t[4], t[2]); p.NP2y = F_SUB(t[5], t[3]);
    p.NQ2x = F_SUB(t[6], t[2]); p.NQ2y = F_SUB(t[7], t[3]);
    p.fA2 = cross2(p.MN2x, p.MN2y, p.MP2x, p.MP2y);
    p.Q4x = cross2(p.MQ2x, p.MQ2y, p.MP2x, p.MP2y);
    p.Q4y = cross2(p.MN2x, p.MN2y, p.MQ2x, p.MQ2y);
    p.t2 = cross2(p.NP2x, p.NP2y, p.NQ2x, p.NQ2y);
}

// Eq. 42: H = [[N2x, P2x, M2x], [N2y, P2y, M2y], [1, 1, 1]] * B,
// B = [[Q4x, 0, -Q4x x0], [0, r Q4y, -r Q4y y0], [t2, r t2, -t2 (x0 + r y0 + w)]].
ACA_HD void rect_solve(const float t[8], const Rect &R, float H[9])
{
    RectParts p;
    rect_parts(t, p);
    const float rQ4y = F_MUL(R.r, p.Q4y), rt2 = F_MUL(R.r, p.t2);
    const float c0x = F_FMA(p.Q4x, t[2], F_MUL(p.t2, t[0]));   // column 1
    const float c0y = F_FMA(p.Q4x, t[3], F_MUL(p.t2, t[1]));
    const float c0w = F_ADD(p.Q4x, p.t2);
    const float c1x = F_FMA(rQ4y, t[4], F_MUL(rt2, t[0]));     // column 2
    const float c1y = F_FMA(rQ4y, t[5], F_MUL(rt2, t[1]));
    const float c1w = F_ADD(rQ4y, rt2);
    // column 3 = -(x0 col1 + y0 col2 + w t2 m2): the t2 m2 parts of x0 col1
    // and y0 col2 supply the remaining -t2 (x0 + r y0) m2 of Eq. 42
    const float t2w = F_MUL(p.t2, R.w);
    H[0] = c0x; H[3] = c0y; H[6] = c0w;
    H[1] = c1x; H[4] = c1y; H[7] = c1w;
    H[2] = -F_FMA(R.x0, c0x, F_FMA(R.y0, c1x, F_MUL(t2w, t[0])));
    H[5] = -F_FMA(R.x0, c0y, F_FMA(R.y0, c1y, F_MUL(t2w, t[1])));
    H[8] = -F_FMA(R.x0, c0w, F_FMA(R.y0, c1w, t2w));
}

}  // namespace aca
