/*
 * First-order rounding-error bounds for the FP32 evaluation orders that the
 * CUDA library documents for its ACA and SKS minimal solvers and for its
 * division-free RANSAC inlier test.  TEST INFRASTRUCTURE ONLY: this is the
 * tolerance model of the parity tests (how far an FP32 result may lie from
 * the exact one), not a solver; the library never calls it and it includes
 * nothing of the library.
 *
 * Method: first-order rounding-error analysis (Wilkinson, "Rounding Errors
 * in Algebraic Processes", 1963; Higham, "Accuracy and Stability of
 * Numerical Algorithms", 2nd ed., 2002, Ch. 2-3).  An FP32 evaluation is
 * recorded on a tape: every quantity q carries its exact value v (computed
 * here in FP64, whose own rounding, ~1e-16 relative, is neglected against
 * u = 2^-24) and the size C of its own rounding event, fl(q) = q + eps with
 * |eps| <= u C, the events independent.  A reverse sweep gives dout/d(event)
 * for every event, and the bound on |fl(out) - out| is u sum |dout/d(event)| C:
 * the worst case over the events to first order, which keeps the
 * cancellations between correlated errors that absolute values taken at
 * every step would lose.  Event sizes (u = 2^-24, round to nearest, no
 * underflow or overflow):
 *   exact FP32 input, exact difference (TwoSum pair)   C = 0
 *   rounded + - * fma /                                C = |v|
 *   Kahan's FMA determinant ad - bc                    C = 2 |v|
 *       (Jeannerod, Louvet and Muller, Math. Comp. 82, 2013: relative
 *       error at most 2u for exact operands)
 *   cross product of two exact differences given as value + remainder,
 *   evaluated as Kahan's determinant of the values plus the four
 *   first-order remainder products          C = 2 |v| + 16 u (|ux vy| + |uy vx|)
 *       (the dropped remainder-by-remainder products are at most
 *       u^2 (|ux vy| + |uy vx|), the four remainder products are summed with
 *       at most 4 roundings of a sum bounded by 2u (|ux vy| + |uy vx|), and
 *       the two final additions add u |v| plus u^2 terms)
 *   double-float product / sum                         C = 16 u m
 *       (TwoProduct and TwoSum are exact; the low parts, of size at most a
 *       few u m with m the magnitude accumulated within the double-float
 *       chain, are added with one or two roundings)
 *   rounding a double-float to FP32                    C = |v|
 *   determinant a d - b c of double-float operands (low part at most 3u
 *   times the operand's magnitude M), rounded once
 *                                  C = 2 |v| + 48 u (M(a) M(d) + M(b) M(c))
 *   product of two such operands, before its rounding  C = 32 u M(a) M(b)
 * Each output gets a token event of 64 u |v|.  The products of two or more
 * events, which the first-order sum neglects, get an allowance of
 * n u / (1 - n u) times the same sum taken over the absolute values of the
 * partial derivatives along every path (n = the number of events on the
 * tape): a product of events is at most u times the absolute contribution
 * of one of them along its path, as in the gamma_n = n u / (1 - n u) of
 * Higham's Lemma 3.1.  Where a first-order term vanishes (the squared
 * residuals of the inlier test at a point mapped exactly), the squares of the
 * first-order bounds of the squared quantities are added explicitly.
 *
 * The evaluation orders (which quantities are rounded where) are those the
 * library states for its solvers: ACA in local frames anchored at M1 / M2
 * with exact edge differences, the eight cross products of Eq. 21, 25 and 27
 * (t1 as cross(N1P1, N1Q1)) each from exact differences, the core of
 * Eq. 28-29 and the local-frame product of Eq. 24 in double-float rounded
 * once per entry, the translation back in FP32; SKS (Eq. 4-14) with exact
 * differences, the similarity images P3, Q3, f_S and cross(ON, QP) as
 * double-float dot and cross products, n7, n8 of Eq. 10-11 formed from them
 * and rounded once, each side scaled by a power of two, the division-free
 * form of Eq. 11-13 over their common denominator, the composition of
 * Eq. 14 in the M frames in FP32 (the local map's zero entries not formed)
 * and the translation back in FP32; the inlier test in its threshold-folded
 * form.  A bound that fails
 * to cover the library's FP32 result therefore means that either the
 * library or its stated evaluation order is wrong.
 *
 * Pinned by tests/test_oracle_fp32_bounds.py: every rule against exact
 * rational arithmetic on random and cancellation-heavy FP32 operands, the
 * whole chains against an FP32 host evaluation of the same orders, and the
 * reverse sweep against the chains re-run at their worst rounding corner
 * (tape.pert); the inlier test also against every corner of its own
 * rounding events, enumerated.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* One tape per chain: node k holds its exact value v, its magnitude m, the
 * size C of its own rounding event (fl(q) = q + eps with |eps| <= u C, the
 * eps of different nodes independent) and the partial derivatives of v
 * with respect to up to four earlier nodes.  The ACA chain takes 118 nodes,
 * SKS 184 and the inlier test about 40; push() stops the process rather than
 * write past the end. */
#define TAPE_MAX 320
static const double U = 0x1p-24;
typedef struct {
    double v, m, C;
    int p[4];
    double w[4];
    int np;
} node;
typedef struct {
    node n[TAPE_MAX];
    int len;
    /* nullable: node k's value becomes v + pert[k] u C as it is pushed, so
     * a chain re-run with pert set evaluates exactly (in FP64) with every
     * rounding event placed at pert[k] times its bound (the pins of the
     * sweep below) */
    const double *pert;
} tape;
static void tape_init(tape *t, const double *pert)
{
    t->len = 0;
    t->pert = pert;
}


static int push(tape *t, double v, double m, double C)
{
    if (t->len >= TAPE_MAX) abort();
    node *q = &t->n[t->len];
    q->v = t->pert ? v + t->pert[t->len] * U * C : v;
    q->m = m;
    q->C = C;
    q->np = 0;
    return t->len++;
}
static void dep(tape *t, int k, int p, double w)
{
    node *q = &t->n[k];
    q->p[q->np] = p;
    q->w[q->np] = w;
    q->np++;
}
#define V(i) (t->n[i].v)
#define M(i) (t->n[i].m)

static int in(tape *t, double x) { return push(t, x, fabs(x), 0.0); }
static int neg(tape *t, int a)
{
    const int k = push(t, -V(a), M(a), 0.0);
    dep(t, k, a, -1.0);
    return k;
}
/* exact sum / difference (an exact TwoSum pair) */
static int xadd(tape *t, int a, int b, double sb)
{
    const double v = V(a) + sb * V(b);
    const int k = push(t, v, fabs(v), 0.0);
    dep(t, k, a, 1.0);
    dep(t, k, b, sb);
    return k;
}
static int xsub(tape *t, int a, int b) { return xadd(t, a, b, -1.0); }
/* exact product by a constant that is a power of two */
static int xscale(tape *t, int a, double c)
{
    const int k = push(t, c * V(a), fabs(c * V(a)), 0.0);
    dep(t, k, a, c);
    return k;
}
/* 2^-e with 2^e <= |x| < 2^(e+1) (1 for 0 or non-finite x) */
static double pow2_inv(float x)
{
    if (!(x != 0) || !isfinite(x)) return 1.0;
    int e;
    frexpf(x, &e);
    return ldexp(1.0, 1 - e);
}
/* the value of a, rounded once to FP32 */
static int rn(tape *t, int a)
{
    const int k = push(t, V(a), fabs(V(a)), fabs(V(a)));
    dep(t, k, a, 1.0);
    return k;
}
/* rounded FP32 operations */
static int add(tape *t, int a, int b)
{
    const double v = V(a) + V(b);
    const int k = push(t, v, fabs(v), fabs(v));
    dep(t, k, a, 1.0);
    dep(t, k, b, 1.0);
    return k;
}
static int sub(tape *t, int a, int b)
{
    const double v = V(a) - V(b);
    const int k = push(t, v, fabs(v), fabs(v));
    dep(t, k, a, 1.0);
    dep(t, k, b, -1.0);
    return k;
}
static int mul(tape *t, int a, int b)
{
    const double v = V(a) * V(b);
    const int k = push(t, v, fabs(v), fabs(v));
    dep(t, k, a, V(b));
    dep(t, k, b, V(a));
    return k;
}
static int fma3(tape *t, int a, int b, int c)
{
    const double v = V(a) * V(b) + V(c);
    const int k = push(t, v, fabs(v), fabs(v));
    dep(t, k, a, V(b));
    dep(t, k, b, V(a));
    dep(t, k, c, 1.0);
    return k;
}
static int dv(tape *t, int a, int b)
{
    const double v = V(a) / V(b);
    const int k = push(t, v, fabs(v), fabs(v));
    dep(t, k, a, 1.0 / V(b));
    dep(t, k, b, -v / V(b));
    return k;
}
/* Kahan's determinant a d - b c */
static int det2(tape *t, int a, int b, int c, int d)
{
    const double v = V(a) * V(d) - V(b) * V(c);
    const int k = push(t, v, fabs(v), 2.0 * fabs(v));
    dep(t, k, a, V(d));
    dep(t, k, d, V(a));
    dep(t, k, b, -V(c));
    dep(t, k, c, -V(b));
    return k;
}
/* ux vy - uy vx of exact differences (value + remainder) */
static int cross_x(tape *t, int ux, int uy, int vx, int vy)
{
    const double A = fabs(V(ux) * V(vy)) + fabs(V(uy) * V(vx));
    const double v = V(ux) * V(vy) - V(uy) * V(vx);
    const int k = push(t, v, fabs(v), 2.0 * fabs(v) + 16.0 * U * A);
    dep(t, k, ux, V(vy));
    dep(t, k, vy, V(ux));
    dep(t, k, uy, -V(vx));
    dep(t, k, vx, -V(uy));
    return k;
}
/* ux vy - uy vx of exact differences (value + remainder) as a double-float:
 * the exact products of the values, their difference by TwoSum, plus the
 * remainder products; only the low part is rounded, at the level of u^2
 * times the products' magnitude */
static int cross_df(tape *t, int ux, int uy, int vx, int vy)
{
    const double A = fabs(V(ux) * V(vy)) + fabs(V(uy) * V(vx));
    const double v = V(ux) * V(vy) - V(uy) * V(vx);
    const int k = push(t, v, A, 16.0 * U * A);
    dep(t, k, ux, V(vy));
    dep(t, k, vy, V(ux));
    dep(t, k, uy, -V(vx));
    dep(t, k, vx, -V(uy));
    return k;
}
/* a d - b c of four double-float operands (value + low part, the low part
 * at most 3u times the operand's magnitude M, as the dot and cross products
 * above and their sums leave it), as Kahan's determinant of the values plus
 * the low parts' first-order terms, rounded once: C = 2 |v| + 48 u S with
 * S = M(a) M(d) + M(b) M(c) (the dropped low-by-low products are at most
 * 9 u^2 S, the four low-part products sum to at most 6 u S and take four
 * roundings, the two final additions add u |v| plus u^2 terms) */
static int det2_dfin(tape *t, int a, int b, int c, int d)
{
    const double S = M(a) * M(d) + M(b) * M(c);
    const double v = V(a) * V(d) - V(b) * V(c);
    const int k = push(t, v, fabs(v), 2.0 * fabs(v) + 48.0 * U * S);
    dep(t, k, a, V(d));
    dep(t, k, d, V(a));
    dep(t, k, b, -V(c));
    dep(t, k, c, -V(b));
    return k;
}
/* the product of two such double-float operands before its rounding:
 * TwoProduct of the values plus the two first-order low-part products,
 * C = 32 u m with m = M(a) M(b) (the dropped low-by-low product is at most
 * 9 u^2 m, the three roundings of the low part at most 18 u^2 m) */
static int dfmul2(tape *t, int a, int b)
{
    const double m = M(a) * M(b);
    const int k = push(t, V(a) * V(b), m, 32.0 * U * m);
    dep(t, k, a, V(b));
    dep(t, k, b, V(a));
    return k;
}
/* double-float steps: exact value, event of size 16 u m with m the
 * magnitude accumulated within the double-float chain (an FP32 operand
 * enters it with m = |value|) */
static int dfmul(tape *t, int a, int b)
{
    const double m = M(a) * M(b);
    const int k = push(t, V(a) * V(b), m, 16.0 * U * m);
    dep(t, k, a, V(b));
    dep(t, k, b, V(a));
    return k;
}
static int dfadd(tape *t, int a, int b)
{
    const double m = M(a) + M(b);
    const int k = push(t, V(a) + V(b), m, 16.0 * U * m);
    dep(t, k, a, 1.0);
    dep(t, k, b, 1.0);
    return k;
}
static int dfsub(tape *t, int a, int b)
{
    const double m = M(a) + M(b);
    const int k = push(t, V(a) - V(b), m, 16.0 * U * m);
    dep(t, k, a, 1.0);
    dep(t, k, b, -1.0);
    return k;
}
/* u . v of exact differences as a double-float */
static int dot_x(tape *t, int ux, int uy, int vx, int vy)
{
    const double v = V(ux) * V(vx) + V(uy) * V(vy);
    const double m = fabs(V(ux) * V(vx)) + fabs(V(uy) * V(vy));
    const int k = push(t, v, m, 16.0 * U * m);
    dep(t, k, ux, V(vx));
    dep(t, k, vx, V(ux));
    dep(t, k, uy, V(vy));
    dep(t, k, vy, V(uy));
    return k;
}
/* token allowance for the neglected second-order terms of an output */
static int final_(tape *t, int a)
{
    const int k = push(t, V(a), fabs(V(a)), 64.0 * U * fabs(V(a)));
    dep(t, k, a, 1.0);
    return k;
}

/* Reverse sweep: adj[k] = dF/d(node k) for F = sum_j g[j] * node out[j]. */
static void sweep(const tape *t, const int *out, const double *g, int nout, double *adj)
{
    memset(adj, 0, sizeof(double) * (size_t)t->len);
    for (int j = 0; j < nout; ++j) adj[out[j]] += g[j];
    for (int k = t->len - 1; k >= 0; --k) {
        const double a = adj[k];
        if (a == 0.0) continue;
        const node *q = &t->n[k];
        for (int i = 0; i < q->np; ++i) adj[q->p[i]] += a * q->w[i];
    }
}

/* The same sweep over absolute weights: adj[k] = the sum over the paths
 * from node k to the outputs of |g| times the absolute product of the
 * partial derivatives along the path. */
static void sweep_abs(const tape *t, const int *out, const double *g, int nout, double *adj)
{
    memset(adj, 0, sizeof(double) * (size_t)t->len);
    for (int j = 0; j < nout; ++j) adj[out[j]] += fabs(g[j]);
    for (int k = t->len - 1; k >= 0; --k) {
        const double a = adj[k];
        if (a == 0.0) continue;
        const node *q = &t->n[k];
        for (int i = 0; i < q->np; ++i) adj[q->p[i]] += a * fabs(q->w[i]);
    }
}

static int n_events(const tape *t)
{
    int n = 0;
    for (int k = 0; k < t->len; ++k) n += t->n[k].C > 0;
    return n;
}

/* allowance for the products of events among n events, given R = the
 * first-order sum over absolute paths */
static double second_order(int n, double R)
{
    const double nu = n * U;
    return nu / (1.0 - nu) * R;
}

/* u * sum_k |adj[k]| C_k: the first-order bound on |fl(F) - F| */
static double event_sum(const tape *t, const double *adj)
{
    double s = 0;
    for (int k = 0; k < t->len; ++k) s += fabs(adj[k]) * t->n[k].C;
    return U * s;
}

/* ------------------------------------------------------------------ */
/* ACA (Eq. 20-29) in the library's evaluation order; H[9] receives the */
/* tape indices of the nine output entries.                             */
/* ------------------------------------------------------------------ */
static void aca_chain(tape *t, const double *s, int H[9])
{
    int x[16];
    for (int k = 0; k < 16; ++k) x[k] = in(t, s[k]);
    const int M1x = x[0], M1y = x[1], N1x = x[2], N1y = x[3], P1x = x[4], P1y = x[5], Q1x = x[6], Q1y = x[7];
    const int M2x = x[8], M2y = x[9], N2x = x[10], N2y = x[11], P2x = x[12], P2y = x[13], Q2x = x[14], Q2y = x[15];
    /* exact edge differences */
    const int mn1x = xsub(t, N1x, M1x), mn1y = xsub(t, N1y, M1y), mp1x = xsub(t, P1x, M1x), mp1y = xsub(t, P1y, M1y);
    const int mq1x = xsub(t, Q1x, M1x), mq1y = xsub(t, Q1y, M1y), np1x = xsub(t, P1x, N1x), np1y = xsub(t, P1y, N1y);
    const int nq1x = xsub(t, Q1x, N1x), nq1y = xsub(t, Q1y, N1y);
    const int mn2x = xsub(t, N2x, M2x), mn2y = xsub(t, N2y, M2y), mp2x = xsub(t, P2x, M2x), mp2y = xsub(t, P2y, M2y);
    const int mq2x = xsub(t, Q2x, M2x), mq2y = xsub(t, Q2y, M2y), np2x = xsub(t, P2x, N2x), np2y = xsub(t, P2y, N2y);
    const int nq2x = xsub(t, Q2x, N2x), nq2y = xsub(t, Q2y, N2y);
    /* Eq. 21, 25, 27 from the exact differences */
    const int fA1 = cross_x(t, mn1x, mn1y, mp1x, mp1y);
    const int Q3x = cross_x(t, mq1x, mq1y, mp1x, mp1y), Q3y = cross_x(t, mn1x, mn1y, mq1x, mq1y);
    const int Q4x = cross_x(t, mq2x, mq2y, mp2x, mp2y), Q4y = cross_x(t, mn2x, mn2y, mq2x, mq2y);
    const int t1 = cross_x(t, np1x, np1y, nq1x, nq1y), t2 = cross_x(t, np2x, np2y, nq2x, nq2y);
    /* the composition uses the edge vectors rounded once */
    const int MN1x = rn(t, mn1x), MN1y = rn(t, mn1y), MP1x = rn(t, mp1x), MP1y = rn(t, mp1y);
    const int NP1x = rn(t, np1x), NP1y = rn(t, np1y);
    const int MN2x = rn(t, mn2x), MN2y = rn(t, mn2y), MP2x = rn(t, mp2x), MP2y = rn(t, mp2y);
    /* Eq. 29 and the local-frame product of Eq. 24, double-float */
    const int c11 = dfmul(t, dfmul(t, t1, Q3y), Q4x), c22 = dfmul(t, dfmul(t, t1, Q3x), Q4y);
    const int c33 = dfmul(t, dfmul(t, t2, Q3x), Q3y);
    const int k0x = dfmul(t, c11, MN2x), k0y = dfmul(t, c11, MN2y), k1x = dfmul(t, c22, MP2x), k1y = dfmul(t, c22, MP2y);
    const int L00 = rn(t, dfsub(t, dfmul(t, k0x, MP1y), dfmul(t, k1x, MN1y)));
    const int L01 = rn(t, dfsub(t, dfmul(t, k1x, MN1x), dfmul(t, k0x, MP1x)));
    const int L10 = rn(t, dfsub(t, dfmul(t, k0y, MP1y), dfmul(t, k1y, MN1y)));
    const int L11 = rn(t, dfsub(t, dfmul(t, k1y, MN1x), dfmul(t, k0y, MP1x)));
    const int L20 = rn(t, dfsub(t, dfsub(t, dfmul(t, c11, MP1y), dfmul(t, c22, MN1y)), dfmul(t, c33, NP1y)));
    const int L21 = rn(t, dfadd(t, dfsub(t, dfmul(t, c22, MN1x), dfmul(t, c11, MP1x)), dfmul(t, c33, NP1x)));
    const int L22 = rn(t, dfmul(t, c33, fA1));
    /* H = T(M2) L T(-M1) in FP32 */
    const int G02 = neg(t, fma3(t, M1x, L00, mul(t, M1y, L01)));
    const int G12 = neg(t, fma3(t, M1x, L10, mul(t, M1y, L11)));
    const int G22 = fma3(t, neg(t, M1x), L20, fma3(t, neg(t, M1y), L21, L22));
    H[0] = fma3(t, M2x, L20, L00);
    H[1] = fma3(t, M2x, L21, L01);
    H[2] = fma3(t, M2x, G22, G02);
    H[3] = fma3(t, M2y, L20, L10);
    H[4] = fma3(t, M2y, L21, L11);
    H[5] = fma3(t, M2y, G22, G12);
    H[6] = L20;
    H[7] = L21;
    H[8] = G22;
    for (int i = 0; i < 9; ++i) H[i] = final_(t, H[i]);
}

/* ------------------------------------------------------------------ */
/* SKS (Eq. 4-14) in the library's evaluation order.                    */
/* ------------------------------------------------------------------ */
typedef struct {
    int onx, ony;        /* ON = MN / 2, exact (value + remainder) */
    int fS_df, fS;       /* |ON|^2: double-float, and rounded */
    int P3x_df, P3y_df, Q3x_df, Q3y_df, cQP_df;   /* double-float */
    int P3x, P3y, Q3y;   /* rounded once */
} sks_side_t;

static void sks_side(tape *t, int Mx, int My, int Nx, int Ny, int Px, int Py, int Qx, int Qy, sks_side_t *o)
{
    o->onx = xscale(t, xsub(t, Nx, Mx), 0.5);
    o->ony = xscale(t, xsub(t, Ny, My), 0.5);
    const int mpx = xsub(t, Px, Mx), mpy = xsub(t, Py, My), mqx = xsub(t, Qx, Mx), mqy = xsub(t, Qy, My);
    const int qpx = xsub(t, Px, Qx), qpy = xsub(t, Py, Qy);
    o->fS_df = dot_x(t, o->onx, o->ony, o->onx, o->ony);
    o->P3y_df = cross_df(t, o->onx, o->ony, mpx, mpy);
    o->Q3y_df = cross_df(t, o->onx, o->ony, mqx, mqy);
    o->P3x_df = dfsub(t, dot_x(t, o->onx, o->ony, mpx, mpy), o->fS_df);
    o->Q3x_df = dfsub(t, dot_x(t, o->onx, o->ony, mqx, mqy), o->fS_df);
    o->cQP_df = cross_df(t, o->onx, o->ony, qpx, qpy);
    o->fS = rn(t, o->fS_df);
    o->P3x = rn(t, o->P3x_df);
    o->P3y = rn(t, o->P3y_df);
    o->Q3y = rn(t, o->Q3y_df);
}

static void sks_chain(tape *t, const double *s, int H[9])
{
    int x[16];
    for (int k = 0; k < 16; ++k) x[k] = in(t, s[k]);
    sks_side_t a, b;
    sks_side(t, x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7], &a);
    sks_side(t, x[8], x[9], x[10], x[11], x[12], x[13], x[14], x[15], &b);
    /* each side's rounded P3, Q3, f_S scaled by the power of two k that
     * brings f_S (as rounded to FP32) into [1, 2) (exact) */
    const double ka = pow2_inv((float)V(a.fS)), kb = pow2_inv((float)V(b.fS));
    const int aP3x = xscale(t, a.P3x, ka), aP3y = xscale(t, a.P3y, ka);
    const int aQ3y = xscale(t, a.Q3y, ka), afS = xscale(t, a.fS, ka);
    const int bP3x = xscale(t, b.P3x, kb), bP3y = xscale(t, b.P3y, kb);
    const int bQ3y = xscale(t, b.Q3y, kb), bfS = xscale(t, b.fS, kb);
    /* Q7 = (n7x, n7y) / d7, Q8 = (n8x, n8y) / d8 (Eq. 10-11) from the
     * double-float sides: a determinant of double-floats and a product of
     * double-floats, each rounded once; then scaled by k^2 (exact) */
    const int n7x = xscale(t, det2_dfin(t, a.Q3x_df, a.P3x_df, a.Q3y_df, a.P3y_df), ka * ka);
    const int n8x = xscale(t, det2_dfin(t, b.Q3x_df, b.P3x_df, b.Q3y_df, b.P3y_df), kb * kb);
    const int n7y = xscale(t, rn(t, dfmul2(t, a.fS_df, a.cQP_df)), ka * ka);
    const int n8y = xscale(t, rn(t, dfmul2(t, b.fS_df, b.cQP_df)), kb * kb);
    /* Eq. 11 and Eq. 13 over the common denominator Q4.y P4.y m */
    const int A = det2(t, n8x, n8y, n7y, n7x), B = det2(t, n8y, n8x, n7y, n7x);
    const int m = mul(t, sub(t, n7x, n7y), add(t, n7x, n7y));
    const int q = mul(t, aQ3y, aP3y), bm = mul(t, bQ3y, m);
    const int aK = mul(t, q, A), bK = mul(t, q, B), dK = mul(t, bP3y, bm);
    const int uK = fma3(t, bP3x, bm, neg(t, mul(t, aQ3y, fma3(t, A, aP3x, mul(t, B, afS)))));
    const int vK = fma3(t, bfS, bm, neg(t, mul(t, aQ3y, fma3(t, B, aP3x, mul(t, A, afS)))));
    /* Eq. 14 in the M frames, FP32; ON rounded once where used.  J maps M1
     * to M2 (the frames' origins): its column 3 is (0, 0, J22), and the first
     * two entries are not formed */
    const int o1x = rn(t, a.onx), o1y = rn(t, a.ony), o2x = rn(t, b.onx), o2y = rn(t, b.ony);
    const int A00 = fma3(t, aK, o1x, neg(t, mul(t, uK, o1y)));
    const int A01 = fma3(t, aK, o1y, mul(t, uK, o1x));
    const int A20 = fma3(t, bK, o1x, neg(t, mul(t, vK, o1y)));
    const int A21 = fma3(t, bK, o1y, mul(t, vK, o1x));
    const int A22 = mul(t, aK, a.fS);
    const int D1x = mul(t, dK, o1x), D1y = mul(t, dK, o1y);
    const int L00 = fma3(t, A00, o2x, mul(t, D1y, o2y));
    const int L01 = fma3(t, A01, o2x, neg(t, mul(t, D1x, o2y)));
    const int L10 = fma3(t, A00, o2y, neg(t, mul(t, D1y, o2x)));
    const int L11 = fma3(t, A01, o2y, mul(t, D1x, o2x));
    const int j22 = fma3(t, neg(t, A20), o1x, fma3(t, neg(t, A21), o1y, A22));
    const int j00 = fma3(t, A20, o2x, L00), j01 = fma3(t, A21, o2x, L01);
    const int j10 = fma3(t, A20, o2y, L10), j11 = fma3(t, A21, o2y, L11);
    const int j20 = A20, j21 = A21;
    const int nM1x = neg(t, x[0]), nM1y = neg(t, x[1]);
    const int K02 = fma3(t, nM1x, j00, mul(t, nM1y, j01));
    const int K12 = fma3(t, nM1x, j10, mul(t, nM1y, j11));
    const int K22 = fma3(t, nM1x, j20, fma3(t, nM1y, j21, j22));
    H[0] = fma3(t, x[8], j20, j00);
    H[1] = fma3(t, x[8], j21, j01);
    H[2] = fma3(t, x[8], K22, K02);
    H[3] = fma3(t, x[9], j20, j10);
    H[4] = fma3(t, x[9], j21, j11);
    H[5] = fma3(t, x[9], K22, K12);
    H[6] = j20;
    H[7] = j21;
    H[8] = K22;
    for (int i = 0; i < 9; ++i) H[i] = final_(t, H[i]);
}

/* Per-entry bounds E_i on |H_fp32,i - H_i| and the bound on
 * max_i |H^_fp32,i - H^_i| at unit Frobenius norm (both normalised
 * exactly, signs aligned): to first order H^' - H^ = (D - H^ <H^, D>) / |H|
 * for the error D, a linear functional of the rounding events per i. */
static double chain_bounds(const tape *t, const int H[9], double *Hv, double *He)
{
    double adj[TAPE_MAX], h[9], n2 = 0;
    for (int i = 0; i < 9; ++i) {
        h[i] = t->n[H[i]].v;
        n2 += h[i] * h[i];
    }
    const double n = sqrt(n2);
    const int nev = n_events(t);
    double beta = 0;
    for (int i = 0; i < 9; ++i) {
        double g[9];
        const double one = 1.0;
        if (He) {
            sweep(t, &H[i], &one, 1, adj);
            He[i] = event_sum(t, adj);
            sweep_abs(t, &H[i], &one, 1, adj);
            He[i] += second_order(nev, event_sum(t, adj));
        }
        if (Hv) Hv[i] = h[i];
        for (int k = 0; k < 9; ++k) g[k] = ((k == i ? 1.0 : 0.0) - h[i] * h[k] / n2) / n;
        sweep(t, H, g, 9, adj);
        double b = event_sum(t, adj);
        sweep_abs(t, H, g, 9, adj);
        b += second_order(nev, event_sum(t, adj));
        beta = b > beta ? b : beta;
    }
    return beta;
}

/* Per set: the unit-Frobenius bound beta[i]; Hv / He (nullable): the exact H
 * of the evaluation order and per-entry absolute bounds, 9 values per set. */
void oracle_aca_fp32_bound(const double *pts, double *beta, double *Hv, double *He, int64_t n)
{
#pragma omp parallel
    {
        tape *t = (tape *)malloc(sizeof(tape));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            int H[9];
            tape_init(t, NULL);
            aca_chain(t, pts + 16 * i, H);
            beta[i] = chain_bounds(t, H, Hv ? Hv + 9 * i : NULL, He ? He + 9 * i : NULL);
        }
        free(t);
    }
}

void oracle_sks_fp32_bound(const double *pts, double *beta, double *Hv, double *He, int64_t n)
{
#pragma omp parallel
    {
        tape *t = (tape *)malloc(sizeof(tape));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            int H[9];
            tape_init(t, NULL);
            sks_chain(t, pts + 16 * i, H);
            beta[i] = chain_bounds(t, H, Hv ? Hv + 9 * i : NULL, He ? He + 9 * i : NULL);
        }
        free(t);
    }
}

/* ------------------------------------------------------------------ */
/* The RANSAC inlier test (forward transfer error, Sec. 6.2) in its     */
/* threshold-folded FP32 form:                                          */
/*   G = (-h11, -h12, -h13, -h21, -h22, -h23, RN(t h31), RN(t h32),     */
/*        RN(t h33)),  (Xs, Ys) = (RN(X RN(1/t)), RN(Y RN(1/t))),       */
/*   w' = fma(G6, x, fma(G7, y, G8)), -u = fma(G0, x, fma(G1, y, G2)),  */
/*   -v likewise, du = fma(Xs, w', -u), dv = fma(Ys, w', -v),           */
/*   e = fma(du, du, fma(dv, dv, RN(w' (-w')))),                        */
/* whose exact value is E = (X w - u)^2 + (Y w - v)^2 - t^2 w^2         */
/* = w^2 (r^2 - t^2), r the forward transfer error of the exact H.  The  */
/* hypothesis H is itself the FP32 ACA result, so the bound counts the   */
/* rounding events of its solve as well (exact power-of-two scalings of  */
/* H change neither the sign of E nor the ratio of E to its bound).  A   */
/* point is decided alike by the FP32 test and the exact one whenever    */
/* |E| exceeds the bound.                                               */
/* ------------------------------------------------------------------ */
typedef struct {
    tape *t;
    int H[9];
    int nev;          /* rounding events of the solve */
    int *ev;          /* their tape indices */
    double *J;        /* [9][nev]: dH_k / d(event node) */
    double Rabs[9];   /* per entry, the solve's first-order sum over absolute paths */
} hyp_model;

static void hyp_model_init(hyp_model *h, const double *s16)
{
    h->t = (tape *)malloc(sizeof(tape));
    tape_init(h->t, NULL);
    aca_chain(h->t, s16, h->H);
    tape *t = h->t;
    h->ev = (int *)malloc(sizeof(int) * (size_t)t->len);
    h->nev = 0;
    for (int k = 0; k < t->len; ++k)
        if (t->n[k].C > 0) h->ev[h->nev++] = k;
    h->J = (double *)malloc(sizeof(double) * 9 * (size_t)(h->nev > 0 ? h->nev : 1));
    double adj[TAPE_MAX];
    for (int i = 0; i < 9; ++i) {
        const double one = 1.0;
        sweep(t, &h->H[i], &one, 1, adj);
        for (int j = 0; j < h->nev; ++j) h->J[i * h->nev + j] = adj[h->ev[j]];
        sweep_abs(t, &h->H[i], &one, 1, adj);
        h->Rabs[i] = event_sum(t, adj);
    }
}

static void hyp_model_free(hyp_model *h)
{
    free(h->J);
    free(h->ev);
    free(h->t);
}

/* The test's quantities at point c under hypothesis h, on a small tape whose
 * inputs are the nine entries of H.  e = du^2 + dv^2 - w'^2 is quadratic in
 * du, dv, w', whose exact values vanish together at points that H maps
 * exactly (du = dv = 0) near its vanishing line (w' -> 0): there E itself
 * is of second order, and so are the squares of the errors of du, dv, w'.
 * The bound therefore is
 *   B = B1(e) + B(du)^2 + B(dv)^2 + B(w')^2,
 * B1(e) the first-order bound of e and B(q) those of du, dv, w' (the
 * remaining second-order products are of relative size u against B1). */
typedef struct {
    double E;
    double crude;     /* upper bound of the exact B (per-entry bounds of H) */
    double own[4];    /* u sum |adj| C over the test's own events: e, du, dv, w' */
    double g[4][9];   /* d(e, du, dv, w') / dH_k */
    double s2[4];     /* allowance for the products of events, solve included */
} test_parts;

/* The test's tape: inputs the nine entries Hval of H (nodes Hn) and the
 * point; tgt = (e, du, dv, w') */
static void test_chain(tape *t, const double *Hval, double thr, const float *c, int Hn[9], int tgt[4])
{
    for (int k = 0; k < 9; ++k) Hn[k] = in(t, Hval[k]);
    const int x = in(t, c[0]), y = in(t, c[1]), X = in(t, c[2]), Y = in(t, c[3]), T = in(t, thr);
    const int rt = dv(t, in(t, 1.0), T);
    const int Xs = mul(t, X, rt), Ys = mul(t, Y, rt);
    const int w = fma3(t, mul(t, T, Hn[6]), x, fma3(t, mul(t, T, Hn[7]), y, mul(t, T, Hn[8])));
    const int nu = fma3(t, neg(t, Hn[0]), x, fma3(t, neg(t, Hn[1]), y, neg(t, Hn[2])));
    const int nv = fma3(t, neg(t, Hn[3]), x, fma3(t, neg(t, Hn[4]), y, neg(t, Hn[5])));
    const int du = fma3(t, Xs, w, nu), dvv = fma3(t, Ys, w, nv);
    const int e = final_(t, fma3(t, du, du, fma3(t, dvv, dvv, mul(t, w, neg(t, w)))));
    tgt[0] = e;
    tgt[1] = du;
    tgt[2] = dvv;
    tgt[3] = w;
}

static void test_parts_of(const hyp_model *h, const double *Eh, double thr, const float *c, test_parts *o)
{
    tape tt;
    tape *t = &tt;
    tape_init(t, NULL);
    int Hn[9], tgt[4];
    double Hval[9];
    for (int k = 0; k < 9; ++k) Hval[k] = h->t->n[h->H[k]].v;
    test_chain(t, Hval, thr, c, Hn, tgt);
    o->E = V(tgt[0]);
    double adj[TAPE_MAX], cr[4];
    const int nev = h->nev + n_events(t);
    for (int q = 0; q < 4; ++q) {
        const double one = 1.0;
        sweep(t, &tgt[q], &one, 1, adj);
        o->own[q] = event_sum(t, adj);
        cr[q] = o->own[q];
        for (int k = 0; k < 9; ++k) {
            o->g[q][k] = adj[Hn[k]];
            cr[q] += fabs(adj[Hn[k]]) * Eh[k];
        }
        sweep_abs(t, &tgt[q], &one, 1, adj);
        double R = event_sum(t, adj);
        for (int k = 0; k < 9; ++k) R += adj[Hn[k]] * h->Rabs[k];
        o->s2[q] = second_order(nev, R);
        cr[q] += o->s2[q];
    }
    o->crude = cr[0] + cr[1] * cr[1] + cr[2] * cr[2] + cr[3] * cr[3];
}

/* the exact first-order sums with the solve's events, completed as above */
static double test_exact_bound(const hyp_model *h, const test_parts *o)
{
    double b[4];
    for (int q = 0; q < 4; ++q) {
        double s = 0;
        for (int j = 0; j < h->nev; ++j) {
            double d = 0;
            for (int k = 0; k < 9; ++k) d += o->g[q][k] * h->J[k * h->nev + j];
            s += fabs(d) * h->t->n[h->ev[j]].C;
        }
        b[q] = o->own[q] + U * s + o->s2[q];
    }
    return b[0] + b[1] * b[1] + b[2] * b[2] + b[3] * b[3];
}

/* per-entry bounds of H (the crude filter's input) */
static void entry_bounds(const hyp_model *h, double *Eh)
{
    for (int k = 0; k < 9; ++k) {
        double e = 0;
        for (int j = 0; j < h->nev; ++j) e += fabs(h->J[k * h->nev + j]) * h->t->n[h->ev[j]].C;
        Eh[k] = U * e;
    }
}

/* bound on |fl(e) - E| for point c under hypothesis h; *E = exact value */
static double test_bound(const hyp_model *h, double thr, const float *c, double *E)
{
    double Eh[9];
    entry_bounds(h, Eh);
    test_parts o;
    test_parts_of(h, Eh, thr, c, &o);
    *E = o.E;
    return test_exact_bound(h, &o);
}

/* Ambiguity of one point under one hypothesis model: 1 if the FP32 test may
 * decide it otherwise than the exact test.  The bound is first computed
 * with the per-entry bounds of H (an upper bound of the exact sum); only
 * points that this cheaper bound cannot decide get the exact sum. */
static int point_ambiguous(const hyp_model *h, const double *Eh, double thr, const float *c)
{
    test_parts o;
    test_parts_of(h, Eh, thr, c, &o);
    if (!isfinite(o.E)) return 1;
    if (fabs(o.E) > o.crude) return 0;
    return !(fabs(o.E) > test_exact_bound(h, &o));
}
#undef V
#undef M

/* Opaque per-hypothesis model for the brute-force scorer in oracle.c. */
typedef struct {
    hyp_model h;
    double Eh[9];
} test_model;

void *oracle_fp32_test_model_new(const double *s16)
{
    test_model *m = (test_model *)malloc(sizeof(test_model));
    hyp_model_init(&m->h, s16);
    entry_bounds(&m->h, m->Eh);
    return m;
}

int oracle_fp32_test_ambiguous(const void *model, double thr, const float *c)
{
    const test_model *m = (const test_model *)model;
    return point_ambiguous(&m->h, m->Eh, thr, c);
}

void oracle_fp32_test_model_free(void *model)
{
    test_model *m = (test_model *)model;
    hyp_model_free(&m->h);
    free(m);
}

/* Scoring band of one hypothesis over N points: amb[i] = 1 if the FP32 test
 * may decide point i otherwise than the exact test (|E| <= its bound, or E
 * not finite) or if its exact residual lies within band_px of the threshold
 * (|r - t| < band_px, the stated count tolerance), else 0.  s16 is the hypothesis's
 * minimal set (16 FP32 coordinates as doubles).  Returns the number of
 * ambiguous points. */
int64_t oracle_score_band(const double *s16, const float *corr, int64_t N, double thr, double band_px,
                          uint8_t *amb)
{
    hyp_model h;
    hyp_model_init(&h, s16);
    const tape *t = h.t;
    double Hv[9];
    for (int k = 0; k < 9; ++k) Hv[k] = t->n[h.H[k]].v;
    int64_t nb = 0;
    for (int64_t i = 0; i < N; ++i) {
        const float *c = corr + 4 * i;
        double E;
        const double B = test_bound(&h, thr, c, &E);
        int a = !(fabs(E) > B);
        if (!a && band_px > 0) {
            const double x = c[0], y = c[1];
            const double u = Hv[0] * x + Hv[1] * y + Hv[2];
            const double v = Hv[3] * x + Hv[4] * y + Hv[5];
            const double w = Hv[6] * x + Hv[7] * y + Hv[8];
            const double r = hypot(c[2] - u / w, c[3] - v / w);
            a = !(fabs(r - thr) >= band_px);
        }
        amb[i] = (uint8_t)a;
        nb += a;
    }
    hyp_model_free(&h);
    return nb;
}

/* The FP32 test's bound alone at each point, in pixels of |r - t|:
 * B / (w^2 (r + t)), with w, r from the exact H. */
void oracle_score_band_px(const double *s16, const float *corr, int64_t N, double thr, double *px)
{
    hyp_model h;
    hyp_model_init(&h, s16);
    double Hv[9];
    for (int k = 0; k < 9; ++k) Hv[k] = h.t->n[h.H[k]].v;
    for (int64_t i = 0; i < N; ++i) {
        const float *c = corr + 4 * i;
        double E;
        const double B = test_bound(&h, thr, c, &E);
        const double x = c[0], y = c[1];
        const double u = Hv[0] * x + Hv[1] * y + Hv[2];
        const double v = Hv[3] * x + Hv[4] * y + Hv[5];
        const double w = Hv[6] * x + Hv[7] * y + Hv[8];
        const double r = hypot(c[2] - u / w, c[3] - v / w);
        px[i] = B / (w * w * (r + thr));
    }
    hyp_model_free(&h);
}

/* ------------------------------------------------------------------ */
/* Hooks for the pins of the rules above (tests only).                  */
/* ------------------------------------------------------------------ */
/* Bound of one rule on FP32 operands a[0..3]: op 0 = a0 + a1, 1 = a0 * a1,
 * 2 = fma(a0, a1, a2), 3 = a0 / a1, 4 = Kahan's a0 a3 - a1 a2, 5 = the
 * cross product of the exact differences (a0 - a1, a2 - a3) and
 * (a4 - a5, a6 - a7) (8 operands), 6 = the double-float product
 * (a0 a1) a2 (TwoProduct, then a double-float times FP32 product) rounded
 * once, 7 and 8 = n7x and n7y of SKS (Eq. 10-11) for one side whose
 * points M, N, P, Q are (a0, a1) ... (a6, a7): the determinant and the
 * product of the side's double-floats, rounded once, 9 = the cross product of
 * op 5 kept as a double-float (its high plus low part against the exact
 * value).  *v = exact value, returns the bound on |fl - v|. */
double oracle_fp32_rule_bound(int op, const double *a, double *v)
{
    tape tt;
    tape *t = &tt;
    tape_init(t, NULL);
    int x[8];
    for (int k = 0; k < 8; ++k) x[k] = in(t, a[k]);
    int r;
    switch (op) {
    case 0: r = add(t, x[0], x[1]); break;
    case 1: r = mul(t, x[0], x[1]); break;
    case 2: r = fma3(t, x[0], x[1], x[2]); break;
    case 3: r = dv(t, x[0], x[1]); break;
    case 4: r = det2(t, x[0], x[1], x[2], x[3]); break;
    case 5: r = cross_x(t, xsub(t, x[0], x[1]), xsub(t, x[2], x[3]), xsub(t, x[4], x[5]), xsub(t, x[6], x[7])); break;
    case 7:
    case 8: {
        sks_side_t o;
        sks_side(t, x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7], &o);
        r = op == 7 ? det2_dfin(t, o.Q3x_df, o.P3x_df, o.Q3y_df, o.P3y_df) : rn(t, dfmul2(t, o.fS_df, o.cQP_df));
        break;
    }
    case 9: r = cross_df(t, xsub(t, x[0], x[1]), xsub(t, x[2], x[3]), xsub(t, x[4], x[5]), xsub(t, x[6], x[7])); break;
    default: r = rn(t, dfmul(t, dfmul(t, x[0], x[1]), x[2])); break;
    }
    *v = t->n[r].v;
    double adj[TAPE_MAX];
    const double one = 1.0;
    sweep(t, &r, &one, 1, adj);
    return event_sum(t, adj);
}

/* Per point of one hypothesis: the exact E of the inlier test and the
 * bound on |fl(e) - E| (the FP32 evaluation, solve included). */
void oracle_score_bound_E(const double *s16, const float *corr, int64_t N, double thr, double *E, double *B)
{
    hyp_model h;
    hyp_model_init(&h, s16);
    for (int64_t i = 0; i < N; ++i) B[i] = test_bound(&h, thr, corr + 4 * i, &E[i]);
    hyp_model_free(&h);
}

/* ------------------------------------------------------------------ */
/* Hooks for the pins of the sweep: each chain re-run with its rounding */
/* events placed at the corner the bound says is the worst (tests only).*/
/* ------------------------------------------------------------------ */
static double sgn(double a) { return a > 0 ? 1.0 : a < 0 ? -1.0 : 0.0; }

/* F = sum_i g_i H_i for the ACA (solver 0) or SKS (solver 1) chain at the
 * set s16.  *b1 = the first-order bound u sum |dF/d(event)| C; *dev = F
 * re-evaluated with every event at sign(dF/d(event)) times its bound,
 * minus F of the exact chain (to first order *dev equals *b1).  Returns
 * the whole bound: *b1 plus the allowance for products of events. */
double oracle_fp32_chain_corner(int solver, const double *s16, const double *g9, double *dev, double *b1)
{
    tape *t = (tape *)malloc(sizeof(tape)), *tp = (tape *)malloc(sizeof(tape));
    double *adj = (double *)malloc(sizeof(double) * TAPE_MAX);
    double *pert = (double *)calloc(TAPE_MAX, sizeof(double));
    int H[9], Hp[9];
    tape_init(t, NULL);
    if (solver) sks_chain(t, s16, H); else aca_chain(t, s16, H);
    sweep(t, H, g9, 9, adj);
    *b1 = event_sum(t, adj);
    for (int k = 0; k < t->len; ++k) pert[k] = sgn(adj[k]);
    sweep_abs(t, H, g9, 9, adj);
    const double b = *b1 + second_order(n_events(t), event_sum(t, adj));
    tape_init(tp, pert);
    if (solver) sks_chain(tp, s16, Hp); else aca_chain(tp, s16, Hp);
    double F = 0, Fp = 0;
    for (int i = 0; i < 9; ++i) {
        F += g9[i] * t->n[H[i]].v;
        Fp += g9[i] * tp->n[Hp[i]].v;
    }
    *dev = Fp - F;
    free(pert);
    free(adj);
    free(tp);
    free(t);
    return b;
}

/* The inlier test at an exact FP32 H (the nine values H9, no solve
 * events): per point the exact E and the bound of the test's own events,
 * completed with the squares of the bounds of du, dv, w' as in the scorer. */
void oracle_score_bound_E_fixed(const double *H9, const float *corr, int64_t N, double thr, double *E, double *B)
{
    tape *t = (tape *)malloc(sizeof(tape));
    double adj[TAPE_MAX];
    for (int64_t i = 0; i < N; ++i) {
        int Hn[9], tgt[4];
        tape_init(t, NULL);
        test_chain(t, H9, thr, corr + 4 * i, Hn, tgt);
        E[i] = t->n[tgt[0]].v;
        double b[4];
        const int nev = n_events(t);
        for (int q = 0; q < 4; ++q) {
            const double one = 1.0;
            sweep(t, &tgt[q], &one, 1, adj);
            b[q] = event_sum(t, adj);
            sweep_abs(t, &tgt[q], &one, 1, adj);
            b[q] += second_order(nev, event_sum(t, adj));
        }
        B[i] = b[0] + b[1] * b[1] + b[2] * b[2] + b[3] * b[3];
    }
    free(t);
}

/* The inlier test at point c under the hypothesis of the minimal set s16,
 * solve included.  *B1 = the first-order bound of e (the test's own events
 * plus the solve's, through dH/d(event)); *dev = e re-evaluated with the
 * solve's events and then the test's at the signs of their first-order
 * weights, minus the exact E (*E). */
void oracle_score_corner(const double *s16, const float *c, double thr, double *B1, double *dev, double *E)
{
    hyp_model h;
    hyp_model_init(&h, s16);
    tape *tt = (tape *)malloc(sizeof(tape)), *tp = (tape *)malloc(sizeof(tape));
    double *adj_t = (double *)malloc(sizeof(double) * TAPE_MAX), *adj_s = (double *)malloc(sizeof(double) * TAPE_MAX);
    double *pert_t = (double *)calloc(TAPE_MAX, sizeof(double)), *pert_s = (double *)calloc(TAPE_MAX, sizeof(double));
    int Hn[9], tgt[4], Hp[9];
    double Hval[9], g[9];
    for (int k = 0; k < 9; ++k) Hval[k] = h.t->n[h.H[k]].v;
    tape_init(tt, NULL);
    test_chain(tt, Hval, thr, c, Hn, tgt);
    *E = tt->n[tgt[0]].v;
    const double one = 1.0;
    sweep(tt, &tgt[0], &one, 1, adj_t);
    for (int k = 0; k < 9; ++k) g[k] = adj_t[Hn[k]];
    sweep(h.t, h.H, g, 9, adj_s);
    *B1 = event_sum(tt, adj_t) + event_sum(h.t, adj_s);
    for (int k = 0; k < h.t->len; ++k) pert_s[k] = sgn(adj_s[k]);
    for (int k = 0; k < tt->len; ++k) pert_t[k] = sgn(adj_t[k]);
    tape_init(tp, pert_s);
    aca_chain(tp, s16, Hp);
    for (int k = 0; k < 9; ++k) Hval[k] = tp->n[Hp[k]].v;
    tape_init(tp, pert_t);
    test_chain(tp, Hval, thr, c, Hn, tgt);
    *dev = tp->n[tgt[0]].v - *E;
    free(pert_s);
    free(pert_t);
    free(adj_s);
    free(adj_t);
    free(tp);
    free(tt);
    hyp_model_free(&h);
}
