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

// a*d - b*c with Kahan's FMA algorithm (error analysis: Jeannerod, Louvet and
// Muller, "Further analysis of Kahan's algorithm for the accurate computation
// of 2x2 determinants", Math. Comp. 2013): w = b*c rounded, e = w - b*c
// exactly, result = (a*d - w) + e, within 2 ulp of the exact value even
// under cancellation.
ACA_HD float det2(float a, float b, float c, float d)
{
    const float w = F_MUL(b, c);
    const float e = F_FMA(-b, c, w);
    const float f = F_FMA(a, d, -w);
    return F_ADD(f, e);
}

// u.x*v.y - u.y*v.x
ACA_HD float cross2(float ux, float uy, float vx, float vy)
{
    return det2(ux, uy, vx, vy);
}

// Exact difference: a - b = d + e exactly (Knuth's TwoSum on a and -b).
struct Diff {
    float h, l;
};

ACA_HD Diff diff(float a, float b)
{
    const float d = F_SUB(a, b);
    const float bv = F_SUB(d, a);       // the part of d that came from -b
    const float av = F_SUB(d, bv);      // the part of d that came from a
    const float er = F_ADD(F_SUB(a, av), F_SUB(-b, bv));
    return Diff{d, er};
}

// cross(u, v) of two exact differences u = uh + ul, v = vh + vl: Kahan's
// determinant of the leading parts plus the first-order remainder terms
// (the dropped ul*vl terms are ~u^2 relative).  Close to the correctly
// rounded cross product of the exact input differences, so a near-collinear
// triple loses no accuracy to the rounding of its edge vectors.
ACA_HD float cross2x(Diff ux, Diff uy, Diff vx, Diff vy)
{
    const float w = F_MUL(uy.h, vx.h);
    const float e = F_FMA(-uy.h, vx.h, w);
    const float f = F_FMA(ux.h, vy.h, -w);
    const float c = F_FMA(ux.h, vy.l, F_FMA(ux.l, vy.h, F_FMA(-uy.h, vx.l, F_MUL(-uy.l, vx.h))));
    return F_ADD(f, F_ADD(e, c));
}

// Double-float arithmetic (value = h + l, |l| <= ulp(h) roughly): products
// by TwoProduct (one FMA recovers the rounding error exactly), sums by
// TwoSum; the low parts are accumulated without renormalisation, which keeps
// ~45 significant bits through the short chains used here.
struct DF {
    float h, l;
};

ACA_HD DF df_prod(float a, float b)
{
    const float p = F_MUL(a, b);
    return DF{p, F_FMA(a, b, -p)};
}

// (x.h + x.l) * b
ACA_HD DF df_mul(DF x, float b)
{
    const float p = F_MUL(x.h, b);
    return DF{p, F_FMA(x.l, b, F_FMA(x.h, b, -p))};
}

ACA_HD DF df_add(DF x, DF y)
{
    const float s = F_ADD(x.h, y.h);
    const float bv = F_SUB(s, x.h);
    const float av = F_SUB(s, bv);
    const float e = F_ADD(F_SUB(x.h, av), F_SUB(y.h, bv));
    return DF{s, F_ADD(e, F_ADD(x.l, y.l))};
}

ACA_HD DF df_neg(DF x) { return DF{-x.h, -x.l}; }

ACA_HD DF df_sub(DF x, DF y) { return df_add(x, df_neg(y)); }

ACA_HD float df_round(DF x) { return F_ADD(x.h, x.l); }

// u . v of two exact differences (value + remainder), as a double-float:
// exact products of the leading parts plus first-order remainder terms.
ACA_HD DF dot2x_df(Diff ux, Diff uy, Diff vx, Diff vy)
{
    const DF a = df_prod(ux.h, vx.h), b = df_prod(uy.h, vy.h);
    const DF s = df_add(a, b);
    const float c = F_FMA(ux.h, vx.l, F_FMA(ux.l, vx.h, F_FMA(uy.h, vy.l, F_MUL(uy.l, vy.h))));
    return DF{s.h, F_ADD(s.l, c)};
}

ACA_HD Diff half(Diff d) { return Diff{F_MUL(0.5f, d.h), F_MUL(0.5f, d.l)}; }

}  // namespace aca
