// Explicitly rounded FP32 operations.
//
// Every arithmetic step of the solvers goes through these macros so that the
// compiler can neither contract a*b+c into an FMA nor reassociate: a given
// set of inputs produces the same bits in every kernel that inlines the same
// device function (the RANSAC scorer, its epilogue and the plain solver), and
// a host build of the same header reproduces the device results exactly
// (IEEE-754 binary32 with round-to-nearest-even throughout; division and
// square root are the correctly rounded IEEE operations).
#pragma once

#if defined(__CUDACC__)
#define ACA_HD __host__ __device__ __forceinline__
#else
#define ACA_HD inline
#endif

#if defined(__CUDA_ARCH__)
#define F_MUL(a, b) __fmul_rn((a), (b))
#define F_ADD(a, b) __fadd_rn((a), (b))
#define F_SUB(a, b) __fsub_rn((a), (b))
#define F_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#define F_DIV(a, b) __fdiv_rn((a), (b))
#define F_SQRT(a) __fsqrt_rn(a)
#else
#include <cmath>
// Host builds must use -ffp-contract=off so these stay single operations.
#define F_MUL(a, b) ((float)(a) * (float)(b))
#define F_ADD(a, b) ((float)(a) + (float)(b))
#define F_SUB(a, b) ((float)(a) - (float)(b))
#define F_FMA(a, b, c) std::fma((float)(a), (float)(b), (float)(c))
#define F_DIV(a, b) ((float)(a) / (float)(b))
#define F_SQRT(a) std::sqrt((float)(a))
#endif

namespace aca {

// ---------------------------------------------------------------------------
// Value types.  The arithmetic below is written once over a value type V:
//  * float: one FP32 value, the explicitly rounded operations above;
//  * P2 (device code only): two FP32 values in one 64-bit register, operated
//    on by the packed f32x2 instructions of sm_100 and later.  Each lane of
//    a packed add, sub, mul or fma is rounded to nearest even exactly like
//    the scalar instruction, so a function evaluated on pairs gives, lane by
//    lane, the bits it gives on floats, with half the instructions issued.
// Negation goes through vneg so that both types share one formula (on float
// it is the sign flip the compiler folds into the consuming instruction).
// ---------------------------------------------------------------------------
ACA_HD float vmul(float a, float b) { return F_MUL(a, b); }
ACA_HD float vadd(float a, float b) { return F_ADD(a, b); }
ACA_HD float vsub(float a, float b) { return F_SUB(a, b); }
ACA_HD float vfma(float a, float b, float c) { return F_FMA(a, b, c); }
ACA_HD float vdiv(float a, float b) { return F_DIV(a, b); }
ACA_HD float vneg(float a) { return -a; }

// the constant x in the value type of `like`
ACA_HD float vconst(float /*like*/, float x) { return x; }

#if defined(__CUDACC__)
struct P2 {
    unsigned long long v;
};

__device__ __forceinline__ P2 vpack(float a, float b)
{
    P2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void vunpack(P2 x, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ float vlo(P2 x)
{
    float a, b;
    vunpack(x, a, b);
    return a;
}
__device__ __forceinline__ float vhi(P2 x)
{
    float a, b;
    vunpack(x, a, b);
    return b;
}
__device__ __forceinline__ P2 vmul(P2 a, P2 b)
{
    P2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ P2 vadd(P2 a, P2 b)
{
    P2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ P2 vsub(P2 a, P2 b)
{
    P2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ P2 vfma(P2 a, P2 b, P2 c)
{
    P2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
// no packed divide: two correctly rounded scalar divisions
__device__ __forceinline__ P2 vdiv(P2 a, P2 b)
{
    return vpack(F_DIV(vlo(a), vlo(b)), F_DIV(vhi(a), vhi(b)));
}
__device__ __forceinline__ P2 vneg(P2 a) { return P2{a.v ^ 0x8000000080000000ull}; }
__device__ __forceinline__ P2 vconst(P2 /*like*/, float x) { return vpack(x, x); }
#endif

// a*d - b*c with Kahan's FMA algorithm (error analysis: Jeannerod, Louvet and
// Muller, "Further analysis of Kahan's algorithm for the accurate computation
// of 2x2 determinants", Math. Comp. 2013): w = b*c rounded, e = w - b*c
// exactly, result = (a*d - w) + e, within 2 ulp of the exact value even
// under cancellation.
template <class V>
ACA_HD V det2(V a, V b, V c, V d)
{
    const V w = vmul(b, c);
    const V e = vfma(vneg(b), c, w);
    const V f = vfma(a, d, vneg(w));
    return vadd(f, e);
}

// u.x*v.y - u.y*v.x
template <class V>
ACA_HD V cross2(V ux, V uy, V vx, V vy)
{
    return det2(ux, uy, vx, vy);
}

// Exact difference: a - b = d + e exactly (Knuth's TwoSum on a and -b).
template <class V>
struct DiffT {
    V h, l;
};
using Diff = DiffT<float>;

template <class V>
ACA_HD DiffT<V> diff(V a, V b)
{
    const V d = vsub(a, b);
    const V bv = vsub(d, a);       // the part of d that came from -b
    const V av = vsub(d, bv);      // the part of d that came from a
    const V er = vadd(vsub(a, av), vsub(vneg(b), bv));
    return DiffT<V>{d, er};
}

// cross(u, v) of two exact differences u = uh + ul, v = vh + vl: Kahan's
// determinant of the leading parts plus the first-order remainder terms
// (the dropped ul*vl terms are ~u^2 relative).  Close to the correctly
// rounded cross product of the exact input differences, so a near-collinear
// triple loses no accuracy to the rounding of its edge vectors.
template <class V>
ACA_HD V cross2x(DiffT<V> ux, DiffT<V> uy, DiffT<V> vx, DiffT<V> vy)
{
    const V nuyh = vneg(uy.h);
    const V w = vmul(uy.h, vx.h);
    const V e = vfma(nuyh, vx.h, w);
    const V f = vfma(ux.h, vy.h, vneg(w));
    const V c = vfma(ux.h, vy.l, vfma(ux.l, vy.h, vfma(nuyh, vx.l, vmul(vneg(uy.l), vx.h))));
    return vadd(f, vadd(e, c));
}

// Double-float arithmetic (value = h + l, |l| <= ulp(h) roughly): products
// by TwoProduct (one FMA recovers the rounding error exactly), sums by
// TwoSum; the low parts are accumulated without renormalisation, which keeps
// ~45 significant bits through the short chains used here.
template <class V>
struct DFT {
    V h, l;
};
using DF = DFT<float>;

template <class V>
ACA_HD DFT<V> df_prod(V a, V b)
{
    const V p = vmul(a, b);
    return DFT<V>{p, vfma(a, b, vneg(p))};
}

// (x.h + x.l) * b
template <class V>
ACA_HD DFT<V> df_mul(DFT<V> x, V b)
{
    const V p = vmul(x.h, b);
    return DFT<V>{p, vfma(x.l, b, vfma(x.h, b, vneg(p)))};
}

template <class V>
ACA_HD DFT<V> df_add(DFT<V> x, DFT<V> y)
{
    const V s = vadd(x.h, y.h);
    const V bv = vsub(s, x.h);
    const V av = vsub(s, bv);
    const V e = vadd(vsub(x.h, av), vsub(y.h, bv));
    return DFT<V>{s, vadd(e, vadd(x.l, y.l))};
}

template <class V>
ACA_HD DFT<V> df_neg(DFT<V> x) { return DFT<V>{vneg(x.h), vneg(x.l)}; }

template <class V>
ACA_HD DFT<V> df_sub(DFT<V> x, DFT<V> y) { return df_add(x, df_neg(y)); }

template <class V>
ACA_HD V df_round(DFT<V> x) { return vadd(x.h, x.l); }

// u . v of two exact differences (value + remainder), as a double-float:
// exact products of the leading parts plus first-order remainder terms.
template <class V>
ACA_HD DFT<V> dot2x_df(DiffT<V> ux, DiffT<V> uy, DiffT<V> vx, DiffT<V> vy)
{
    const DFT<V> a = df_prod(ux.h, vx.h), b = df_prod(uy.h, vy.h);
    const DFT<V> s = df_add(a, b);
    const V c = vfma(ux.h, vx.l, vfma(ux.l, vx.h, vfma(uy.h, vy.l, vmul(uy.l, vy.h))));
    return DFT<V>{s.h, vadd(s.l, c)};
}

// cross(u, v) of two exact differences as a double-float: the exact
// products of the leading parts, their difference by TwoSum, plus the
// first-order remainder terms (what cross2x rounds, kept unrounded).
template <class V>
ACA_HD DFT<V> cross2x_df(DiffT<V> ux, DiffT<V> uy, DiffT<V> vx, DiffT<V> vy)
{
    const DFT<V> s = df_sub(df_prod(ux.h, vy.h), df_prod(uy.h, vx.h));
    const V nuyh = vneg(uy.h);
    const V c = vfma(ux.h, vy.l, vfma(ux.l, vy.h, vfma(nuyh, vx.l, vmul(vneg(uy.l), vx.h))));
    return DFT<V>{s.h, vadd(s.l, c)};
}

// a*d - b*c of four double-floats, rounded once: Kahan's determinant of the
// leading parts plus the first-order terms of the low parts.
template <class V>
ACA_HD V det2_df(DFT<V> a, DFT<V> b, DFT<V> c, DFT<V> d)
{
    const V nbh = vneg(b.h);
    const V w = vmul(b.h, c.h);
    const V e = vfma(nbh, c.h, w);
    const V f = vfma(a.h, d.h, vneg(w));
    const V r = vfma(a.h, d.l, vfma(a.l, d.h, vfma(nbh, c.l, vmul(vneg(b.l), c.h))));
    return vadd(f, vadd(e, r));
}

// x * y of two double-floats, rounded once (TwoProduct of the leading parts
// plus the first-order terms of the low parts).
template <class V>
ACA_HD V df_mul_round(DFT<V> x, DFT<V> y)
{
    const V p = vmul(x.h, y.h);
    const V e = vfma(x.h, y.l, vfma(x.l, y.h, vfma(x.h, y.h, vneg(p))));
    return vadd(p, e);
}

template <class V>
ACA_HD DiffT<V> half(DiffT<V> d)
{
    const V k = vconst(d.h, 0.5f);
    return DiffT<V>{vmul(k, d.h), vmul(k, d.l)};
}

}  // namespace aca
