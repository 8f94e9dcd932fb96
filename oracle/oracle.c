/*
 * FP64 CPU oracle for the ACA / SKS minimal homography solvers, the RANSAC
 * scoring they feed and the ACA derivative.  TEST INFRASTRUCTURE ONLY: the
 * tests, the smoke check and the benchmark's CPU-baseline leg call this; the
 * library never does.  It shares no code with the CUDA path.
 *
 * Every function follows the paper (arXiv 2402.18008) step by step in its
 * notation; no blocking, fusion or reordering beyond what the equations state.
 *
 * Layouts: a minimal set is 16 doubles, M1 N1 P1 Q1 M2 N2 P2 Q2 as (x, y)
 * pairs (side 1 = source, side 2 = target); a homography is 9 doubles,
 * row-major h11..h33.  Correspondences for RANSAC are float32 (x1, y1, x2, y2).
 *
 * Parity status of each function is stated in its comment; all are pinned by
 * the CPU tests (exact rational DLT, invariants, special cases, cuRAND's
 * Philox, brute force) except where it says "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel loops (timing on one core or all). */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* 3x3 helpers                                                          */
/* ------------------------------------------------------------------ */
static void mat3_mul(const double *A, const double *B, double *C)
{
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = A[3 * i + 0] * B[0 + j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
    memcpy(C, T, sizeof T);
}

static void mat3_vec(const double *A, const double *x, double *y)
{
    double t[3];
    for (int i = 0; i < 3; ++i)
        t[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
    memcpy(y, t, sizeof t);
}

/* ------------------------------------------------------------------ */
/* ACA: Sec. 4.2-4.3, Eq. 20-29                                         */
/* ------------------------------------------------------------------ */
/* Steps, in the paper's order:
 *  (Eq. 20, Table 4) vectors M1N1, M1P1 and f_A1 (Eq. 21); same on target;
 *  (Eq. 25) Q3 = H_A1 Q1 = (cross(M1Q1, M1P1), cross(M1N1, M1Q1), f_A1), Q4 alike;
 *  (Eq. 27) t1 = f_A1 - Q3.x - Q3.y, t2 = f_A2 - Q4.x - Q4.y;
 *  (Eq. 29) c11 = t1 Q3.y Q4.x, c22 = t1 Q3.x Q4.y, c33 = t2 Q3.x Q3.y;
 *  (Eq. 28) H_C = [[c11,0,0],[0,c22,0],[c11-c33, c22-c33, c33]];
 *  (Eq. 20) H_A1 = [[M1P1.y, -M1P1.x, 0],[-M1N1.y, M1N1.x, 0],[0,0,f_A1]] T(-M1);
 *  (Eq. 22) H_A2^-1 = [[M2N2.x, M2P2.x, M2.x],[M2N2.y, M2P2.y, M2.y],[0,0,1]];
 *  (Eq. 24) H = H_A2^-1 H_C H_A1.
 * Returns the unnormalised, division-free H. */
static void aca_one(const double *s, double *H)
{
    const double M1x = s[0], M1y = s[1], N1x = s[2], N1y = s[3];
    const double P1x = s[4], P1y = s[5], Q1x = s[6], Q1y = s[7];
    const double M2x = s[8], M2y = s[9], N2x = s[10], N2y = s[11];
    const double P2x = s[12], P2y = s[13], Q2x = s[14], Q2y = s[15];

    const double MN1x = N1x - M1x, MN1y = N1y - M1y;
    const double MP1x = P1x - M1x, MP1y = P1y - M1y;
    const double fA1 = MN1x * MP1y - MN1y * MP1x;
    const double MN2x = N2x - M2x, MN2y = N2y - M2y;
    const double MP2x = P2x - M2x, MP2y = P2y - M2y;
    const double fA2 = MN2x * MP2y - MN2y * MP2x;

    const double MQ1x = Q1x - M1x, MQ1y = Q1y - M1y;
    const double MQ2x = Q2x - M2x, MQ2y = Q2y - M2y;
    const double Q3x = MQ1x * MP1y - MQ1y * MP1x;
    const double Q3y = MN1x * MQ1y - MN1y * MQ1x;
    const double Q4x = MQ2x * MP2y - MQ2y * MP2x;
    const double Q4y = MN2x * MQ2y - MN2y * MQ2x;

    const double t1 = fA1 - Q3x - Q3y;
    const double t2 = fA2 - Q4x - Q4y;

    const double c11 = t1 * Q3y * Q4x;
    const double c22 = t1 * Q3x * Q4y;
    const double c33 = t2 * Q3x * Q3y;

    const double HC[9] = {c11, 0, 0, 0, c22, 0, c11 - c33, c22 - c33, c33};
    const double L1[9] = {MP1y, -MP1x, 0, -MN1y, MN1x, 0, 0, 0, fA1};
    const double T1[9] = {1, 0, -M1x, 0, 1, -M1y, 0, 0, 1};
    double HA1[9];
    mat3_mul(L1, T1, HA1);
    const double HA2inv[9] = {MN2x, MP2x, M2x, MN2y, MP2y, M2y, 0, 0, 1};
    double T[9];
    mat3_mul(HA2inv, HC, T);
    mat3_mul(T, HA1, H);
}

void oracle_aca(const double *pts, double *H, int64_t n)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        aca_one(pts + 16 * i, H + 9 * i);
}

/* Same chain with the core of Eq. 23 / Eq. 26 (division form):
 * a_C = t1 Q4.x / (t2 Q3.x), b_C = t1 Q4.y / (t2 Q3.y),
 * H_C = [[a_C,0,0],[0,b_C,0],[a_C-1, b_C-1, 1]].  Cross-check of Eq. 28. */
static void aca_divform_one(const double *s, double *H)
{
    const double M1x = s[0], M1y = s[1], N1x = s[2], N1y = s[3];
    const double P1x = s[4], P1y = s[5], Q1x = s[6], Q1y = s[7];
    const double M2x = s[8], M2y = s[9], N2x = s[10], N2y = s[11];
    const double P2x = s[12], P2y = s[13], Q2x = s[14], Q2y = s[15];
    const double MN1x = N1x - M1x, MN1y = N1y - M1y, MP1x = P1x - M1x, MP1y = P1y - M1y;
    const double MN2x = N2x - M2x, MN2y = N2y - M2y, MP2x = P2x - M2x, MP2y = P2y - M2y;
    const double fA1 = MN1x * MP1y - MN1y * MP1x;
    const double fA2 = MN2x * MP2y - MN2y * MP2x;
    const double MQ1x = Q1x - M1x, MQ1y = Q1y - M1y, MQ2x = Q2x - M2x, MQ2y = Q2y - M2y;
    const double Q3x = MQ1x * MP1y - MQ1y * MP1x, Q3y = MN1x * MQ1y - MN1y * MQ1x;
    const double Q4x = MQ2x * MP2y - MQ2y * MP2x, Q4y = MN2x * MQ2y - MN2y * MQ2x;
    const double t1 = fA1 - Q3x - Q3y, t2 = fA2 - Q4x - Q4y;
    const double aC = t1 * Q4x / (t2 * Q3x);
    const double bC = t1 * Q4y / (t2 * Q3y);
    const double HC[9] = {aC, 0, 0, 0, bC, 0, aC - 1, bC - 1, 1};
    const double L1[9] = {MP1y, -MP1x, 0, -MN1y, MN1x, 0, 0, 0, fA1};
    const double T1[9] = {1, 0, -M1x, 0, 1, -M1y, 0, 0, 1};
    double HA1[9], T[9];
    mat3_mul(L1, T1, HA1);
    const double HA2inv[9] = {MN2x, MP2x, M2x, MN2y, MP2y, M2y, 0, 0, 1};
    mat3_mul(HA2inv, HC, T);
    mat3_mul(T, HA1, H);
}

void oracle_aca_divform(const double *pts, double *H, int64_t n)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        aca_divform_one(pts + 16 * i, H + 9 * i);
}

/* ------------------------------------------------------------------ */
/* Affine transformation from three correspondences: Sec. 5.2, Eq. 38   */
/* ------------------------------------------------------------------ */
/* H_A = H_A2^-1 H_A1 with H_A1 of Eq. 20 (anchor points M1, N1, P1) and
 * H_A2^-1 of Eq. 22 (M2, N2, P2): the core is the identity when the map is
 * affine.  s: 12 doubles M1 N1 P1 M2 N2 P2 (x, y); H: 9 doubles, third row
 * (0, 0, f_A1) (division-free, like ACA). */
static void affine_one(const double *s, double *H)
{
    const double M1x = s[0], M1y = s[1], N1x = s[2], N1y = s[3], P1x = s[4], P1y = s[5];
    const double M2x = s[6], M2y = s[7], N2x = s[8], N2y = s[9], P2x = s[10], P2y = s[11];
    const double MN1x = N1x - M1x, MN1y = N1y - M1y, MP1x = P1x - M1x, MP1y = P1y - M1y;
    const double MN2x = N2x - M2x, MN2y = N2y - M2y, MP2x = P2x - M2x, MP2y = P2y - M2y;
    const double fA1 = MN1x * MP1y - MN1y * MP1x;
    const double L1[9] = {MP1y, -MP1x, 0, -MN1y, MN1x, 0, 0, 0, fA1};
    const double T1[9] = {1, 0, -M1x, 0, 1, -M1y, 0, 0, 1};
    double HA1[9];
    mat3_mul(L1, T1, HA1);
    const double HA2inv[9] = {MN2x, MP2x, M2x, MN2y, MP2y, M2y, 0, 0, 1};
    mat3_mul(HA2inv, HA1, H);
}

void oracle_aca_affine(const double *pts, double *H, int64_t n)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        affine_one(pts + 12 * i, H + 9 * i);
}

/* ------------------------------------------------------------------ */
/* DLT: Sec. 2.1, Eq. 1-3, inhomogeneous 8x8 form (h33 = 1) solved by   */
/* Gaussian elimination with partial pivoting (the GPT-LU solver the    */
/* paper compares against).  Independent of the ACA code above.         */
/* ------------------------------------------------------------------ */
/* Each correspondence x1 -> x2 gives the two rows of Eq. 2:
 *   [x1^T, 0^T, -x2 x1^T] h = 0 ;  [0^T, -x1^T, y2 x1^T] h = 0,
 * h = (h11 h12 h13 h21 h22 h23 h31 h32 h33); with h33 = 1 the last column
 * moves to the right-hand side.  Returns 0 on success, 1 if a zero pivot
 * was met (degenerate set: H filled with NaN). */
static int dlt_one(const double *s, double *H)
{
    double A[8][9];
    for (int k = 0; k < 4; ++k) {
        const double x = s[2 * k], y = s[2 * k + 1];
        const double X = s[8 + 2 * k], Y = s[8 + 2 * k + 1];
        double *r0 = A[2 * k], *r1 = A[2 * k + 1];
        r0[0] = x; r0[1] = y; r0[2] = 1; r0[3] = 0; r0[4] = 0; r0[5] = 0;
        r0[6] = -X * x; r0[7] = -X * y; r0[8] = X;      /* rhs = -(-X * 1) */
        r1[0] = 0; r1[1] = 0; r1[2] = 0; r1[3] = -x; r1[4] = -y; r1[5] = -1;
        r1[6] = Y * x; r1[7] = Y * y; r1[8] = -Y;       /* rhs = -(Y * 1) */
    }
    for (int c = 0; c < 8; ++c) {
        int piv = c;
        for (int r = c + 1; r < 8; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c]))
                piv = r;
        if (A[piv][c] == 0.0) {
            for (int i = 0; i < 9; ++i)
                H[i] = NAN;
            return 1;
        }
        if (piv != c)
            for (int j = 0; j < 9; ++j) {
                double t = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = t;
            }
        for (int r = c + 1; r < 8; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int j = c; j < 9; ++j)
                A[r][j] -= f * A[c][j];
        }
    }
    double h[8];
    for (int r = 7; r >= 0; --r) {
        double acc = A[r][8];
        for (int j = r + 1; j < 8; ++j)
            acc -= A[r][j] * h[j];
        h[r] = acc / A[r][r];
    }
    for (int i = 0; i < 8; ++i)
        H[i] = h[i];
    H[8] = 1.0;
    return 0;
}

int64_t oracle_dlt(const double *pts, double *H, int64_t n)
{
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = 0; i < n; ++i)
        bad += dlt_one(pts + 16 * i, H + 9 * i);
    return bad;
}

/* ------------------------------------------------------------------ */
/* SKS: Sec. 3, Eq. 4-14                                                */
/* ------------------------------------------------------------------ */
/* (Eq. 4-6) O = midpoint of MN, ON = N - O, f_S = |ON|^2,
 *           H_S = [[ON.x, ON.y, 0],[-ON.y, ON.x, 0],[0,0,f_S]] T(-O);
 * (Eq. 8)   H_S^-1 = [[ON.x, -ON.y, O.x],[ON.y, ON.x, O.y],[0,0,1]];
 * P3 = H_S1 P1, Q3 = H_S1 Q1, P4 = H_S2 P2, Q4 = H_S2 Q2 (homogeneous);
 * (Eq. 10)  H_E swaps the 2nd and 3rd homogeneous coordinates; P5, P6 are
 *           the dehomogenised H_E P3, H_E P4;
 * (Eq. 11)  Q7 = dehom(H_E Q3) - P5, Q8 = dehom(H_E Q4) - P6 (H_T1 H_E and
 *           H_T2 H_E), then a_G, b_G from the 2x2 system of Eq. 11;
 * (Eq. 13)  a_K = a_G, b_K = b_G, u_K = P6.x - a_K P5.x - b_K P5.y,
 *           v_K = P6.y - b_K P5.x - a_K P5.y;
 * (Eq. 9, 14) H = H_S2^-1 [[a_K,u_K,b_K],[0,1,0],[b_K,v_K,a_K]] H_S1. */
static void sks_one(const double *s, double *H)
{
    const double M1x = s[0], M1y = s[1], N1x = s[2], N1y = s[3];
    const double M2x = s[8], M2y = s[9], N2x = s[10], N2y = s[11];
    const double O1x = 0.5 * (M1x + N1x), O1y = 0.5 * (M1y + N1y);
    const double ON1x = N1x - O1x, ON1y = N1y - O1y;
    const double fS1 = ON1x * ON1x + ON1y * ON1y;
    const double O2x = 0.5 * (M2x + N2x), O2y = 0.5 * (M2y + N2y);
    const double ON2x = N2x - O2x, ON2y = N2y - O2y;
    const double fS2 = ON2x * ON2x + ON2y * ON2y;

    const double R1[9] = {ON1x, ON1y, 0, -ON1y, ON1x, 0, 0, 0, fS1};
    const double T1[9] = {1, 0, -O1x, 0, 1, -O1y, 0, 0, 1};
    const double R2[9] = {ON2x, ON2y, 0, -ON2y, ON2x, 0, 0, 0, fS2};
    const double T2[9] = {1, 0, -O2x, 0, 1, -O2y, 0, 0, 1};
    double HS1[9], HS2[9];
    mat3_mul(R1, T1, HS1);
    mat3_mul(R2, T2, HS2);
    const double HS2inv[9] = {ON2x, -ON2y, O2x, ON2y, ON2x, O2y, 0, 0, 1};

    const double P1h[3] = {s[4], s[5], 1}, Q1h[3] = {s[6], s[7], 1};
    const double P2h[3] = {s[12], s[13], 1}, Q2h[3] = {s[14], s[15], 1};
    double P3[3], Q3[3], P4[3], Q4[3];
    mat3_vec(HS1, P1h, P3);
    mat3_vec(HS1, Q1h, Q3);
    mat3_vec(HS2, P2h, P4);
    mat3_vec(HS2, Q2h, Q4);

    /* H_E [x, y, w] = [x, w, y]; dehomogenise by the new 3rd coordinate. */
    const double P5x = P3[0] / P3[1], P5y = P3[2] / P3[1];
    const double P6x = P4[0] / P4[1], P6y = P4[2] / P4[1];
    const double Q7x = Q3[0] / Q3[1] - P5x, Q7y = Q3[2] / Q3[1] - P5y;
    const double Q8x = Q4[0] / Q4[1] - P6x, Q8y = Q4[2] / Q4[1] - P6y;

    const double det = Q7x * Q7x - Q7y * Q7y;
    const double aG = (Q8x * Q7x - Q8y * Q7y) / det;
    const double bG = (Q8y * Q7x - Q8x * Q7y) / det;

    const double aK = aG, bK = bG;
    const double uK = P6x - aK * P5x - bK * P5y;
    const double vK = P6y - bK * P5x - aK * P5y;
    const double HK[9] = {aK, uK, bK, 0, 1, 0, bK, vK, aK};
    double T[9];
    mat3_mul(HS2inv, HK, T);
    mat3_mul(T, HS1, H);
}

void oracle_sks(const double *pts, double *H, int64_t n)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        sks_one(pts + 16 * i, H + 9 * i);
}

/* ------------------------------------------------------------------ */
/* Rectangle source: Sec. 5.3, Eq. 39-42 and Algorithm 1               */
/* ------------------------------------------------------------------ */
/* tgt: 8 doubles M2 N2 P2 Q2; rectangle (x0, y0) upper-left, width w,
 * aspect ratio r = w / h.  Q4 and t2 as in Eq. 25 and Eq. 27 on the target;
 * Eq. 42: H = [[N2.x,P2.x,M2.x],[N2.y,P2.y,M2.y],[1,1,1]] *
 *   [[Q4.x, 0, -Q4.x x0],[0, r Q4.y, -r Q4.y y0],[t2, r t2, -t2 (x0 + r y0 + w)]]. */
static void rect_eq42_one(const double *t, double x0, double y0, double w, double r, double *H)
{
    const double M2x = t[0], M2y = t[1], N2x = t[2], N2y = t[3];
    const double P2x = t[4], P2y = t[5], Q2x = t[6], Q2y = t[7];
    const double MN2x = N2x - M2x, MN2y = N2y - M2y, MP2x = P2x - M2x, MP2y = P2y - M2y;
    const double MQ2x = Q2x - M2x, MQ2y = Q2y - M2y;
    const double fA2 = MN2x * MP2y - MN2y * MP2x;
    const double Q4x = MQ2x * MP2y - MQ2y * MP2x;
    const double Q4y = MN2x * MQ2y - MN2y * MQ2x;
    const double t2 = fA2 - Q4x - Q4y;
    const double A[9] = {N2x, P2x, M2x, N2y, P2y, M2y, 1, 1, 1};
    const double B[9] = {Q4x, 0, -Q4x * x0, 0, r * Q4y, -r * Q4y * y0, t2, r * t2, -t2 * (x0 + r * y0 + w)};
    mat3_mul(A, B, H);
}

void oracle_aca_rect(const double *tgt, double x0, double y0, double w, double r, double *H, int64_t n)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        rect_eq42_one(tgt + 8 * i, x0, y0, w, r, H + 9 * i);
}

/* Algorithm 1's vector operations, as operations (its comments' signs are
 * not used): d1, d2 difference vectors; c = d1 x d2; b = sum(c) m2;
 * h1 = c1 n2 - b; h2 = r (c2 p2 - b); h3 = w b - x0 h1 - y0 h2 (columns). */
static void rect_alg1_one(const double *t, double x0, double y0, double w, double r, double *H)
{
    const double m2[3] = {t[0], t[1], 1}, n2[3] = {t[2], t[3], 1};
    const double p2[3] = {t[4], t[5], 1}, q2[3] = {t[6], t[7], 1};
    const double d1[3] = {n2[0] - m2[0], p2[0] - m2[0], q2[0] - m2[0]};
    const double d2[3] = {n2[1] - m2[1], p2[1] - m2[1], q2[1] - m2[1]};
    const double c[3] = {d1[1] * d2[2] - d1[2] * d2[1], d1[2] * d2[0] - d1[0] * d2[2],
                         d1[0] * d2[1] - d1[1] * d2[0]};
    const double sc = c[0] + c[1] + c[2];
    double b[3], h1[3], h2[3], h3[3];
    for (int k = 0; k < 3; ++k) b[k] = sc * m2[k];
    for (int k = 0; k < 3; ++k) h1[k] = c[0] * n2[k] - b[k];
    for (int k = 0; k < 3; ++k) h2[k] = r * (c[1] * p2[k] - b[k]);
    for (int k = 0; k < 3; ++k) h3[k] = w * b[k] - x0 * h1[k] - y0 * h2[k];
    for (int k = 0; k < 3; ++k) {
        H[3 * k + 0] = h1[k];
        H[3 * k + 1] = h2[k];
        H[3 * k + 2] = h3[k];
    }
}

void oracle_aca_rect_alg1(const double *tgt, double x0, double y0, double w, double r, double *H, int64_t n)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        rect_alg1_one(tgt + 8 * i, x0, y0, w, r, H + 9 * i);
}

/* ------------------------------------------------------------------ */
/* Analytic Jacobian dH/d(target coordinates), source fixed.           */
/* Forward-mode chain rule through the same steps as aca_one and        */
/* rect_eq42_one: every intermediate carries its 8 partial derivatives  */
/* w.r.t. (M2.x, M2.y, N2.x, N2.y, P2.x, P2.y, Q2.x, Q2.y).  H is a     */
/* polynomial (Sec. 4.5), so these derivatives are exact up to rounding. */
/* ------------------------------------------------------------------ */
typedef struct {
    double v;
    double d[8];
} dual;

static dual dconst(double v)
{
    dual r;
    r.v = v;
    memset(r.d, 0, sizeof r.d);
    return r;
}
static dual dvar(double v, int k)
{
    dual r = dconst(v);
    r.d[k] = 1.0;
    return r;
}
static dual dadd(dual a, dual b)
{
    dual r;
    r.v = a.v + b.v;
    for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] + b.d[k];
    return r;
}
static dual dsub(dual a, dual b)
{
    dual r;
    r.v = a.v - b.v;
    for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] - b.d[k];
    return r;
}
static dual dmul(dual a, dual b)
{
    dual r;
    r.v = a.v * b.v;
    for (int k = 0; k < 8; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
static dual dneg(dual a)
{
    return dsub(dconst(0.0), a);
}
static void dmat3_mul(const dual *A, const dual *B, dual *C)
{
    dual T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            T[3 * i + j] = dadd(dadd(dmul(A[3 * i], B[j]), dmul(A[3 * i + 1], B[3 + j])), dmul(A[3 * i + 2], B[6 + j]));
    memcpy(C, T, sizeof T);
}

/* Derivatives w.r.t. the 8 coordinates of one side (side 0 = source,
 * side 1 = target); the other side is held constant. */
static void aca_jac_side(const double *s, int side, double *J)
{
    dual v[16];
    for (int k = 0; k < 16; ++k)
        v[k] = (k / 8 == side) ? dvar(s[k], k % 8) : dconst(s[k]);
    const dual M1x = v[0], M1y = v[1], N1x = v[2], N1y = v[3], P1x = v[4], P1y = v[5], Q1x = v[6], Q1y = v[7];
    const dual M2x = v[8], M2y = v[9], N2x = v[10], N2y = v[11], P2x = v[12], P2y = v[13], Q2x = v[14], Q2y = v[15];

    const dual MN1x = dsub(N1x, M1x), MN1y = dsub(N1y, M1y), MP1x = dsub(P1x, M1x), MP1y = dsub(P1y, M1y);
    const dual fA1 = dsub(dmul(MN1x, MP1y), dmul(MN1y, MP1x));
    const dual MN2x = dsub(N2x, M2x), MN2y = dsub(N2y, M2y), MP2x = dsub(P2x, M2x), MP2y = dsub(P2y, M2y);
    const dual fA2 = dsub(dmul(MN2x, MP2y), dmul(MN2y, MP2x));
    const dual MQ1x = dsub(Q1x, M1x), MQ1y = dsub(Q1y, M1y), MQ2x = dsub(Q2x, M2x), MQ2y = dsub(Q2y, M2y);
    const dual Q3x = dsub(dmul(MQ1x, MP1y), dmul(MQ1y, MP1x));
    const dual Q3y = dsub(dmul(MN1x, MQ1y), dmul(MN1y, MQ1x));
    const dual Q4x = dsub(dmul(MQ2x, MP2y), dmul(MQ2y, MP2x));
    const dual Q4y = dsub(dmul(MN2x, MQ2y), dmul(MN2y, MQ2x));
    const dual t1 = dsub(dsub(fA1, Q3x), Q3y);
    const dual t2 = dsub(dsub(fA2, Q4x), Q4y);
    const dual c11 = dmul(dmul(t1, Q3y), Q4x);
    const dual c22 = dmul(dmul(t1, Q3x), Q4y);
    const dual c33 = dmul(dmul(t2, Q3x), Q3y);
    const dual z = dconst(0), one = dconst(1);
    const dual HC[9] = {c11, z, z, z, c22, z, dsub(c11, c33), dsub(c22, c33), c33};
    const dual L1[9] = {MP1y, dneg(MP1x), z, dneg(MN1y), MN1x, z, z, z, fA1};
    const dual T1[9] = {one, z, dneg(M1x), z, one, dneg(M1y), z, z, one};
    const dual HA2inv[9] = {MN2x, MP2x, M2x, MN2y, MP2y, M2y, z, z, one};
    dual HA1[9], T[9], H[9];
    dmat3_mul(L1, T1, HA1);
    dmat3_mul(HA2inv, HC, T);
    dmat3_mul(T, HA1, H);
    for (int i = 0; i < 9; ++i)
        for (int k = 0; k < 8; ++k)
            J[8 * i + k] = H[i].d[k];
}

static void aca_jac_one(const double *s, double *J)
{
    aca_jac_side(s, 1, J);
}

/* J: n x 9 x 8, J[i][r][k] = dH_r / d tgt_k. */
void oracle_aca_jacobian(const double *pts, double *J, int64_t n)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        aca_jac_one(pts + 16 * i, J + 72 * i);
}

/* J: n x 9 x 8, derivatives w.r.t. the source coordinates (target fixed). */
void oracle_aca_jacobian_src(const double *pts, double *J, int64_t n)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        aca_jac_side(pts + 16 * i, 0, J + 72 * i);
}

/* Componentwise condition number of the unit-Frobenius ACA homography
 * H^ = H / |H| with respect to relative perturbations of all 16 input
 * coordinates: kappa = max_i sum_k |dH^_i / dx_k| |x_k|, with
 * dH^/dx_k = (dH/dx_k - H^ <H^, dH/dx_k>) / |H|.  kappa * u bounds, to first
 * order, how far H^ moves when every coordinate is perturbed by a relative
 * u (u = 2^-24 for the rounding of FP32 inputs).  Used to state which sets
 * are well-conditioned enough for an FP32 solver to meet a tolerance. */
static double aca_condition_one(const double *s);

void oracle_aca_condition(const double *pts, double *kappa, int64_t n)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        kappa[i] = aca_condition_one(pts + 16 * i);
}

static double aca_condition_one(const double *s)
{
    {
        double H[9], Js[72], Jt[72];
        aca_one(s, H);
        aca_jac_side(s, 0, Js);
        aca_jac_side(s, 1, Jt);
        double nrm = 0;
        for (int r = 0; r < 9; ++r) nrm += H[r] * H[r];
        nrm = sqrt(nrm);
        double Hh[9];
        for (int r = 0; r < 9; ++r) Hh[r] = H[r] / nrm;
        double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = 0; k < 16; ++k) {
            double d[9], proj = 0;
            for (int r = 0; r < 9; ++r) {
                d[r] = k < 8 ? Js[8 * r + k] : Jt[8 * r + (k - 8)];
                proj += Hh[r] * d[r];
            }
            for (int r = 0; r < 9; ++r)
                acc[r] += fabs((d[r] - Hh[r] * proj) / nrm) * fabs(s[k]);
        }
        double m = 0;
        for (int r = 0; r < 9; ++r) m = acc[r] > m ? acc[r] : m;
        return m;
    }
}

static void rect_jac_one(const double *t, double x0, double y0, double w, double r, double *J)
{
    const dual M2x = dvar(t[0], 0), M2y = dvar(t[1], 1), N2x = dvar(t[2], 2), N2y = dvar(t[3], 3);
    const dual P2x = dvar(t[4], 4), P2y = dvar(t[5], 5), Q2x = dvar(t[6], 6), Q2y = dvar(t[7], 7);
    const dual MN2x = dsub(N2x, M2x), MN2y = dsub(N2y, M2y), MP2x = dsub(P2x, M2x), MP2y = dsub(P2y, M2y);
    const dual MQ2x = dsub(Q2x, M2x), MQ2y = dsub(Q2y, M2y);
    const dual fA2 = dsub(dmul(MN2x, MP2y), dmul(MN2y, MP2x));
    const dual Q4x = dsub(dmul(MQ2x, MP2y), dmul(MQ2y, MP2x));
    const dual Q4y = dsub(dmul(MN2x, MQ2y), dmul(MN2y, MQ2x));
    const dual t2 = dsub(dsub(fA2, Q4x), Q4y);
    const dual X0 = dconst(x0), Y0 = dconst(y0), W = dconst(w), R = dconst(r), z = dconst(0), one = dconst(1);
    const dual A[9] = {N2x, P2x, M2x, N2y, P2y, M2y, one, one, one};
    const dual B[9] = {Q4x, z, dneg(dmul(Q4x, X0)),
                       z, dmul(R, Q4y), dneg(dmul(dmul(R, Q4y), Y0)),
                       t2, dmul(R, t2), dneg(dmul(t2, dadd(dadd(X0, dmul(R, Y0)), W)))};
    dual H[9];
    dmat3_mul(A, B, H);
    for (int i = 0; i < 9; ++i)
        for (int k = 0; k < 8; ++k)
            J[8 * i + k] = H[i].d[k];
}

void oracle_aca_rect_jacobian(const double *tgt, double x0, double y0, double w, double r, double *J, int64_t n)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        rect_jac_one(tgt + 8 * i, x0, y0, w, r, J + 72 * i);
}

/* ------------------------------------------------------------------ */
/* Counter-based sampling for RANSAC (the paper gives no sampler).      */
/* ------------------------------------------------------------------ */
/* Philox4x32-10 from its published definition (Salmon, Moraes, Dror and
 * Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds
 * of two 32x32->64 multiplications by 0xD2511F53 and 0xCD9E8D57 with the
 * Feistel-like permutation, the key bumped by the Weyl constants
 * 0x9E3779B9 / 0xBB67AE85 between rounds. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Four distinct indices in [0, N) for hypothesis `hyp` of problem `prob`:
 * counter (hyp, prob, 0, 0), key (seed low, seed high) -> u0..u3;
 * j_k = floor(u_k (N - k) / 2^32) is a rank among the N - k indices not
 * yet drawn; it is turned into an index by stepping over the earlier
 * draws in ascending order (j += 1 for each earlier index <= j).
 * Draw k = 0, 1, 2, 3 becomes M, N, P, Q.  Requires N >= 4. */
void oracle_sample4(uint64_t seed, uint32_t prob, uint32_t hyp, int64_t N, int64_t idx[4])
{
    const uint32_t ctr[4] = {hyp, prob, 0u, 0u};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t u[4];
    oracle_philox4x32_10(ctr, key, u);
    int64_t taken[4];
    int nt = 0;
    for (int k = 0; k < 4; ++k) {
        int64_t j = (int64_t)(((uint64_t)u[k] * (uint64_t)(N - k)) >> 32);
        /* earlier draws sorted ascending */
        int64_t sorted[4];
        for (int a = 0; a < nt; ++a) sorted[a] = taken[a];
        for (int a = 1; a < nt; ++a)
            for (int b = a; b > 0 && sorted[b - 1] > sorted[b]; --b) {
                int64_t t = sorted[b];
                sorted[b] = sorted[b - 1];
                sorted[b - 1] = t;
            }
        for (int a = 0; a < nt; ++a)
            if (j >= sorted[a])
                ++j;
        taken[nt++] = j;
        idx[k] = j;
    }
}

/* ------------------------------------------------------------------ */
/* RANSAC hypothesis scoring (Sec. 2.2, Sec. 6.2): brute force.         */
/* ------------------------------------------------------------------ */
/* A sample is degenerate (scores -1, can never win) if on either side one of
 * its four triples (M,N,P), (M,Q,P), (M,N,Q), (N,P,Q) has
 * |cross|^2 <= tau^2 |a|^2 |b|^2 for its two edge vectors a, b, i.e. the
 * sine of the angle between them is at most tau (the paper is silent on
 * degenerate samples). */
#define ORACLE_DEGEN_TAU 1e-3

static int triple_degenerate(double ax, double ay, double bx, double by)
{
    const double c = ax * by - ay * bx;
    const double la = ax * ax + ay * ay, lb = bx * bx + by * by;
    return c * c <= ORACLE_DEGEN_TAU * ORACLE_DEGEN_TAU * la * lb;
}

static int side_degenerate(const double *p)
{
    const double MNx = p[2] - p[0], MNy = p[3] - p[1];
    const double MPx = p[4] - p[0], MPy = p[5] - p[1];
    const double MQx = p[6] - p[0], MQy = p[7] - p[1];
    const double NPx = p[4] - p[2], NPy = p[5] - p[3];
    const double NQx = p[6] - p[2], NQy = p[7] - p[3];
    return triple_degenerate(MNx, MNy, MPx, MPy) || triple_degenerate(MQx, MQy, MPx, MPy) ||
           triple_degenerate(MNx, MNy, MQx, MQy) || triple_degenerate(NPx, NPy, NQx, NQy);
}

int oracle_sample_degenerate(const double *s16)
{
    /* a sample with a non-finite coordinate is degenerate (it defines no map) */
    for (int k = 0; k < 16; ++k)
        if (!isfinite(s16[k])) return 1;
    return side_degenerate(s16) || side_degenerate(s16 + 8);
}

/* Unit Frobenius norm; sign so that h33 > 0, or, when |h33| < 1e-6 |H|,
 * so that the entry of largest magnitude is positive. */
void oracle_normalize_frob(double *H)
{
    double s = 0;
    for (int i = 0; i < 9; ++i) s += H[i] * H[i];
    s = sqrt(s);
    if (s == 0) return;
    int big = 0;
    for (int i = 1; i < 9; ++i)
        if (fabs(H[i]) > fabs(H[big])) big = i;
    double sign = (fabs(H[8]) >= 1e-6 * s) ? (H[8] > 0 ? 1.0 : -1.0) : (H[big] > 0 ? 1.0 : -1.0);
    for (int i = 0; i < 9; ++i) H[i] = sign * H[i] / s;
}

/* Inlier test (forward transfer error, inclusive):
 * || (x2, y2) - (u / w, v / w) || <= thr with (u, v, w) = H (x1, y1, 1);
 * a point mapped to infinity (w = 0) is an outlier.  The test does not
 * depend on the arbitrary sign of the division-free H.  Returns 1 / 0 and
 * the margin ||r|| - thr (NaN margin when w = 0). */
static int score_point(const double *H, const float *c, double thr, double *margin)
{
    const double x = c[0], y = c[1], X = c[2], Y = c[3];
    const double u = H[0] * x + H[1] * y + H[2];
    const double v = H[3] * x + H[4] * y + H[5];
    const double w = H[6] * x + H[7] * y + H[8];
    if (w == 0) {
        *margin = NAN;
        return 0;
    }
    const double dx = X - u / w, dy = Y - v / w;
    const double r = sqrt(dx * dx + dy * dy);
    *margin = r - thr;
    return r <= thr;
}

/* Ambiguity band of the RANSAC count parity.  The stated tolerance is that
 * counts are exact except for points within band_px of the threshold.  An
 * FP32 implementation also meets points whose decision its own rounding can
 * flip: fp32_bounds.c bounds, to first order, the rounding error of the
 * library's FP32 evaluation of the test (its hypothesis solve included) at
 * each point, and a point whose exact E = w^2 (r^2 - thr^2) lies within
 * that bound is ambiguous too.  amb_in / amb_out count the ambiguous points
 * that the exact test takes as inliers / outliers, so an FP32 count c must
 * satisfy counts[h] - amb_in[h] <= c <= counts[h] + amb_out[h]. */
void *oracle_fp32_test_model_new(const double *s16);
int oracle_fp32_test_ambiguous(const void *model, double thr, const float *c);
void oracle_fp32_test_model_free(void *model);

/* Per-hypothesis inlier counts for one problem (N correspondences).
 * counts[h] = -1 for degenerate samples; amb_in / amb_out (nullable, both or
 * neither) as described above. */
void oracle_score_problem(const float *corr, int64_t N, int32_t n_hyp, double thr, uint64_t seed,
                          uint32_t prob, int32_t *counts, int32_t *amb_in, int32_t *amb_out, double band_px)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int32_t h = 0; h < n_hyp; ++h) {
        if (N < 4) {
            counts[h] = -1;
            if (amb_in) amb_in[h] = amb_out[h] = 0;
            continue;
        }
        int64_t idx[4];
        oracle_sample4(seed, prob, (uint32_t)h, N, idx);
        double s[16];
        for (int k = 0; k < 4; ++k) {
            const float *c = corr + 4 * idx[k];
            s[2 * k] = c[0];
            s[2 * k + 1] = c[1];
            s[8 + 2 * k] = c[2];
            s[8 + 2 * k + 1] = c[3];
        }
        if (oracle_sample_degenerate(s)) {
            counts[h] = -1;
            if (amb_in) amb_in[h] = amb_out[h] = 0;
            continue;
        }
        double H[9];
        aca_one(s, H);
        void *model = amb_in ? oracle_fp32_test_model_new(s) : NULL;
        int32_t cnt = 0, ni = 0, no = 0;
        for (int64_t i = 0; i < N; ++i) {
            double m;
            const int inl = score_point(H, corr + 4 * i, thr, &m);
            cnt += inl;
            if (model) {
                /* NaN margin (w = 0 or a non-finite point) counts as ambiguous */
                const int amb = !(fabs(m) >= band_px) || oracle_fp32_test_ambiguous(model, thr, corr + 4 * i);
                if (amb) {
                    if (inl) ++ni;
                    else ++no;
                }
            }
        }
        counts[h] = cnt;
        if (model) {
            amb_in[h] = ni;
            amb_out[h] = no;
            oracle_fp32_test_model_free(model);
        }
    }
}

/* Full RANSAC over P problems (CSR offsets in points, n_hyp[p] hypotheses
 * each).  Best = highest count, ties to the lowest hypothesis index;
 * best_H unit-Frobenius sign-fixed; best_hyp = -1 and best_count = 0 when
 * every sample is degenerate.  hyp_counts (nullable) is laid
 * out problem after problem (prefix sums of n_hyp); so are amb_in / amb_out
 * (nullable, both or neither; see oracle_score_problem).  inlier_mask (nullable)
 * marks the best hypothesis's inliers. */
void oracle_ransac(const float *corr, const int64_t *offsets, const int32_t *n_hyp, int32_t P, double thr,
                   uint64_t seed, uint32_t problem_base, double *best_H, int32_t *best_count,
                   int32_t *best_hyp, int32_t *hyp_counts, int32_t *amb_in, int32_t *amb_out, double band_px,
                   uint8_t *inlier_mask)
{
    int64_t hoff = 0;
    for (int32_t p = 0; p < P; ++p) {
        const int64_t N = offsets[p + 1] - offsets[p];
        const float *c = corr + 4 * offsets[p];
        const int32_t k = n_hyp[p];
        int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * (k > 0 ? k : 1));
        oracle_score_problem(c, N, k, thr, seed, problem_base + (uint32_t)p, cnt, amb_in ? amb_in + hoff : NULL,
                             amb_in ? amb_out + hoff : NULL, band_px);
        int32_t bh = -1, bc = -1;
        for (int32_t h = 0; h < k; ++h)
            if (cnt[h] > bc) {
                bc = cnt[h];
                bh = h;
            }
        if (bc < 0) {
            bh = -1;
            bc = 0;
        }
        if (hyp_counts) memcpy(hyp_counts + hoff, cnt, sizeof(int32_t) * k);
        best_hyp[p] = bh;
        best_count[p] = bc;
        double H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (bh >= 0) {
            int64_t idx[4];
            oracle_sample4(seed, problem_base + (uint32_t)p, (uint32_t)bh, N, idx);
            double s[16];
            for (int q = 0; q < 4; ++q) {
                s[2 * q] = c[4 * idx[q]];
                s[2 * q + 1] = c[4 * idx[q] + 1];
                s[8 + 2 * q] = c[4 * idx[q] + 2];
                s[8 + 2 * q + 1] = c[4 * idx[q] + 3];
            }
            aca_one(s, H);
            if (inlier_mask)
                for (int64_t i = 0; i < N; ++i) {
                    double m;
                    inlier_mask[offsets[p] + i] = (uint8_t)score_point(H, c + 4 * i, thr, &m);
                }
            oracle_normalize_frob(H);
        } else if (inlier_mask) {
            memset(inlier_mask + offsets[p], 0, (size_t)N);
        }
        memcpy(best_H + 9 * p, H, sizeof H);
        free(cnt);
        hoff += k;
    }
}

/* ---------------------------------------------------------------------------
 * Online adaptive termination (Sec. 6.2: the number of loops follows from the
 * inlier ratio with 99% probability that one 4-point sample is all inliers,
 * with a cap).  With the best count c so far among N correspondences,
 * w = c / N and the required number of hypotheses is
 *     K(c) = ceil(log(1 - confidence) / log(1 - w^4)),
 * clamped to [1, cap]; c <= 0 gives cap.  log_fail = log(1 - confidence).
 * ------------------------------------------------------------------------- */
int32_t oracle_adaptive_k(int32_t c, int64_t N, int32_t cap, double log_fail)
{
    if (c <= 0 || N <= 0) return cap;
    const double w = (double)c / (double)N;
    const double w4 = (w * w) * (w * w);
    if (w4 >= 1.0) return 1;
    const double den = log1p(-w4);
    if (!(den < 0.0)) return cap;
    const double r = ceil(log_fail / den);
    if (!(r < (double)cap)) return cap;
    return r < 1.0 ? 1 : (int32_t)r;
}

/* The sequential loop: before hypothesis i, stop if i >= K(best of 0..i-1);
 * the best improves only on a strictly larger count.  Returns the number of
 * hypotheses evaluated (1..k; k if the cap is reached). */
int32_t oracle_adaptive_stop(const int32_t *cnt, int32_t k, int64_t N, double log_fail)
{
    int32_t best = -1, kreq = k;
    for (int32_t i = 0; i < k; ++i) {
        if (i >= kreq) return i;
        if (cnt[i] > best) {
            best = cnt[i];
            kreq = oracle_adaptive_k(best, N, k, log_fail);
        }
    }
    return k;
}

/* RANSAC with the online stop: every problem scores its cap max_hyp[p]
 * hypotheses (hyp_counts / amb_in / amb_out as in oracle_ransac, all of them),
 * n_eval[p] = the stop index, and the best is the argmax over the evaluated
 * hypotheses only (ties to the lowest index). */
void oracle_ransac_adaptive(const float *corr, const int64_t *offsets, const int32_t *max_hyp, int32_t P, double thr,
                            uint64_t seed, uint32_t problem_base, double confidence, double *best_H,
                            int32_t *best_count, int32_t *best_hyp, int32_t *n_eval, int32_t *hyp_counts,
                            int32_t *amb_in, int32_t *amb_out, double band_px, uint8_t *inlier_mask)
{
    const double log_fail = log(1.0 - confidence);
    int64_t hoff = 0;
    for (int32_t p = 0; p < P; ++p) {
        const int64_t N = offsets[p + 1] - offsets[p];
        const float *c = corr + 4 * offsets[p];
        const int32_t k = max_hyp[p];
        int32_t *cnt = (int32_t *)malloc(sizeof(int32_t) * (k > 0 ? k : 1));
        oracle_score_problem(c, N, k, thr, seed, problem_base + (uint32_t)p, cnt, amb_in ? amb_in + hoff : NULL,
                             amb_in ? amb_out + hoff : NULL, band_px);
        const int32_t ne = N >= 4 && k > 0 ? oracle_adaptive_stop(cnt, k, N, log_fail) : 0;
        int32_t bh = -1, bc = -1;
        for (int32_t h = 0; h < ne; ++h)
            if (cnt[h] > bc) {
                bc = cnt[h];
                bh = h;
            }
        if (bc < 0) {
            bh = -1;
            bc = 0;
        }
        if (hyp_counts) memcpy(hyp_counts + hoff, cnt, sizeof(int32_t) * (k > 0 ? k : 0));
        best_hyp[p] = bh;
        best_count[p] = bc;
        n_eval[p] = ne;
        double H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (bh >= 0) {
            int64_t idx[4];
            oracle_sample4(seed, problem_base + (uint32_t)p, (uint32_t)bh, N, idx);
            double s[16];
            for (int q = 0; q < 4; ++q) {
                s[2 * q] = c[4 * idx[q]];
                s[2 * q + 1] = c[4 * idx[q] + 1];
                s[8 + 2 * q] = c[4 * idx[q] + 2];
                s[8 + 2 * q + 1] = c[4 * idx[q] + 3];
            }
            aca_one(s, H);
            if (inlier_mask)
                for (int64_t i = 0; i < N; ++i) {
                    double m;
                    inlier_mask[offsets[p] + i] = (uint8_t)score_point(H, c + 4 * i, thr, &m);
                }
            oracle_normalize_frob(H);
        } else if (inlier_mask) {
            memset(inlier_mask + offsets[p], 0, (size_t)N);
        }
        memcpy(best_H + 9 * p, H, sizeof H);
        free(cnt);
        hoff += k > 0 ? k : 0;
    }
}
