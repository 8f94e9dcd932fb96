// Refit of one homography per problem on all of its masked correspondences:
// the global optimisation with all inliers that ends the RANSAC pipeline
// (Sec. 6.2, stage 5).  One block per problem:
//   1. Hartley normalisation of each side: centroid to the origin, mean
//      distance sqrt(2) (two passes over the points);
//   2. normalised DLT: the 9x9 normal matrix M of the two Eq. 2 rows of every
//      point (one pass), its eigenvector of the smallest eigenvalue by inverse
//      iteration on a Cholesky factor (FP64), started from e_k with k the
//      largest diagonal entry of M^-1 (sum_j v_j[k]^2 / lambda_j, dominated by
//      the smallest eigenvalue's vector, so e_k has a component of at least
//      1/3 along it);
//   3. Levenberg-Marquardt on the reprojection error in the normalised frames
//      (the eight entries of H with h33 = 1), with the damping schedule of
//      Madsen, Nielsen & Tingleff, "Methods for non-linear least squares
//      problems" (2004), Alg. 3.16; each trial step is one pass.
//
// Precision on GB300, where FP64 runs at 1/64 of the FP32 rate:
//   - per-point arithmetic is FP32 on O(1) normalised coordinates;
//   - sums whose cancellation matters (the DLT moments, the gradient J^T r
//     and the cost) are double-float: FP32 partials over chunks of 8 points,
//     accumulated by TwoSum, reduced by a fixed shuffle tree (deterministic);
//     J^T J, which only shapes the step, is summed in FP32;
//   - the 9x9 DLT solves run in FP64, the 8x8 LM steps in FP32 (an inexact
//     step only slows the iteration; its fixed point is set by the gradient),
//     both by one warp with lane i owning row i;
//   - the cost of a trial point carries FP32 rounding noise of about 2^-16
//     relative, so near the optimum, where the predicted decrease is below
//     that noise, a step is accepted unless the cost rises by more than the
//     noise: the gain ratio could not tell such steps apart.
#include <math.h>

#include "common.cuh"
#include "fp32.cuh"

namespace aca {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 8;
constexpr int kInvIters = 16;         // inverse-iteration cap
constexpr float kTau = 1e-3f;         // mu0 = tau * max diag(J^T J)
constexpr double kEpsStep = 5.9604644775390625e-8;   // 2^-24: parameters are used in FP32
constexpr double kCostNoise = 1.52587890625e-05;     // 2^-16: FP32 noise of the cost, relative

constexpr int kDF_DLT = 24;           // double-float sums of the DLT pass
constexpr int kDF_LM = 9;             // gradient (8) and cost (1)
constexpr int kF_LM = 19;             // J^T J moments

struct Shared {
    DF red[kWarps][kDF_DLT];          // per-warp double-float partials
    float redf[kWarps][kF_LM];
    double sum[kDF_DLT];              // block sums (double-float -> FP64)
    float sumf[kF_LM];
    double M[81], L9[81], r9[9];      // DLT normal matrix, Cholesky factor, 1 / diagonal
    double v[9];                      // DLT eigenvector
    float S8[64], L8[64], r8[8];      // LM matrix, factor, 1 / diagonal
    float par[8];                     // parameters broadcast to the pass
    float mu1x, mu1y, s1, mu2x, mu2y, s2;
    int go;                           // leader -> block decision
    // Levenberg-Marquardt state (leader warp)
    float A[64];                      // J^T J at pd
    double g[8], F;                   // J^T r and ||r||^2 / 2 at pd
    double pd[8], d[8], mu, nu;
};

// Double-float accumulator: FP32 partials per chunk of kChunk points, then
// TwoSum into (h, l).
template <int K>
struct DFAcc {
    float f[K];
    DF s[K];
    int c;
    __device__ void zero()
    {
#pragma unroll
        for (int k = 0; k < K; ++k) { f[k] = 0.0f; s[k] = DF{0.0f, 0.0f}; }
        c = 0;
    }
    __device__ void flush()
    {
#pragma unroll
        for (int k = 0; k < K; ++k) { s[k] = df_add(s[k], DF{f[k], 0.0f}); f[k] = 0.0f; }
        c = 0;
    }
    __device__ void tick()
    {
        if (++c == kChunk) flush();
    }
};

__device__ __forceinline__ DF df_renorm(DF x)
{
    const float s = F_ADD(x.h, x.l);
    return DF{s, F_SUB(x.l, F_SUB(s, x.h))};
}

__device__ __forceinline__ DF warp_sum_df(DF x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DF y{__shfl_xor_sync(0xffffffffu, x.h, o), __shfl_xor_sync(0xffffffffu, x.l, o)};
        x = df_renorm(df_add(x, y));
    }
    return x;
}

__device__ __forceinline__ float warp_sum_f(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ double warp_sum_d(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block sums: double-float values into sh.sum[0..K) (as FP64) and FP32 values
// into sh.sumf[0..KF); visible to all threads on return.
template <int K, int KF>
__device__ void block_reduce(DF (&s)[K], float (&f)[KF], Shared &sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const DF v = warp_sum_df(s[k]);
        if (lane == 0) sh.red[warp][k] = v;
    }
#pragma unroll
    for (int k = 0; k < KF; ++k) {
        const float v = warp_sum_f(f[k]);
        if (lane == 0) sh.redf[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        DF a = sh.red[0][threadIdx.x];
#pragma unroll
        for (int w = 1; w < kWarps; ++w) a = df_renorm(df_add(a, sh.red[w][threadIdx.x]));
        sh.sum[threadIdx.x] = (double)a.h + (double)a.l;
    } else if (threadIdx.x >= 32 && threadIdx.x < 32 + KF) {
        const int k = threadIdx.x - 32;
        float a = 0.0f;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) a += sh.redf[w][k];
        sh.sumf[k] = a;
    }
    __syncthreads();
}

// Cholesky factor of the n x n symmetric S (row-major, shared) by one warp:
// lane i builds row i of L in registers.  Pivots below `floor` are raised to
// it.  Writes L (row-major, lower) and rd[j] = 1 / L[j][j]; returns false on
// a non-positive or non-finite pivot (all lanes agree).
template <int n, typename T>
__device__ bool warp_cholesky(const T *S, T *L, T *rd, T floor)
{
    const int lane = threadIdx.x & 31;
    T row[n];
#pragma unroll
    for (int k = 0; k < n; ++k) row[k] = T(0);
    bool ok = true;
#pragma unroll
    for (int j = 0; j < n; ++j) {
        T s = lane < n ? S[lane * n + j] : T(0);
#pragma unroll
        for (int k = 0; k < j; ++k) s -= row[k] * __shfl_sync(0xffffffffu, row[k], j);
        T d = __shfl_sync(0xffffffffu, s, j);
        if (d < floor) d = floor;
        ok = ok && d > T(0) && isfinite(d);
        const T ljj = sqrt(d);
        const T r = T(1) / ljj;
        if (lane == j) row[j] = ljj;
        else if (lane > j && lane < n) row[j] = s * r;
        if (lane == 0) rd[j] = r;
    }
    if (lane < n) {
#pragma unroll
        for (int k = 0; k < n; ++k) L[lane * n + k] = k <= lane ? row[k] : T(0);
    }
    __syncwarp();
    return ok;
}

// x := (L L^T)^-1 x by one warp; lane i holds x_i (lanes >= n hold 0).
template <int n, typename T>
__device__ T warp_chol_solve(const T *L, const T *rd, T x)
{
    const int lane = threadIdx.x & 31;
    // L y = x (column-oriented: y_j final at step j, then eliminated below)
#pragma unroll
    for (int j = 0; j < n; ++j) {
        const T yj = __shfl_sync(0xffffffffu, x, j) * rd[j];
        if (lane == j) x = yj;
        else if (lane > j && lane < n) x -= L[lane * n + j] * yj;
    }
    // L^T z = y
#pragma unroll
    for (int j = n - 1; j >= 0; --j) {
        const T zj = __shfl_sync(0xffffffffu, x, j) * rd[j];
        if (lane == j) x = zj;
        else if (lane < j) x -= L[j * n + lane] * zj;
    }
    return x;
}

__device__ __forceinline__ bool take(const uint8_t *mask, int64_t i) { return mask == nullptr || mask[i] != 0; }

// Unit Frobenius norm in FP64, sign so that h33 > 0 (or, when |h33| < 1e-6
// |H|, so that the entry of largest magnitude is positive); written as FP32.
__device__ void store_frob(const double h[9], float *out)
{
    double ss = 0.0;
    int big = 0;
    for (int i = 0; i < 9; ++i) {
        ss += h[i] * h[i];
        if (fabs(h[i]) > fabs(h[big])) big = i;
    }
    const double nrm = sqrt(ss);
    if (!(nrm > 0.0) || !isfinite(nrm)) {
        for (int i = 0; i < 9; ++i) out[i] = 0.0f;
        return;
    }
    const double sgn = fabs(h[8]) >= 1e-6 * nrm ? (h[8] > 0 ? 1.0 : -1.0) : (h[big] > 0 ? 1.0 : -1.0);
    for (int i = 0; i < 9; ++i) out[i] = (float)(sgn * h[i] / nrm);
}

struct Frame {
    float m1x, m1y, s1, m2x, m2y, s2;
    __device__ explicit Frame(const Shared &sh)
        : m1x(sh.mu1x), m1y(sh.mu1y), s1(sh.s1), m2x(sh.mu2x), m2y(sh.mu2y), s2(sh.s2) {}
    __device__ void apply(float4 q, float &x, float &y, float &X, float &Y) const
    {
        x = s1 * (q.x - m1x);
        y = s1 * (q.y - m1y);
        X = s2 * (q.z - m2x);
        Y = s2 * (q.w - m2y);
    }
};

// One LM pass at the parameters in sh.par.  Sums, with xb = (x, y, 1),
// b = (x, y), q = 1/w^2:
//   double-float: g = J^T r (u rows: r_u xb / w; v rows: r_v xb / w;
//                 perspective: -(u r_u + v r_v) b / w) and ||r||^2;
//   FP32: sum q {xx, xy, yy, x, y, 1}, sum q u {xx, xy, yy, x, y},
//         sum q v {...}, sum q (u^2 + v^2) {xx, xy, yy}, the blocks of J^T J.
__device__ void lm_pass(const float4 *c, const uint8_t *m, int64_t n, Shared &sh)
{
    DFAcc<kDF_LM> a;
    a.zero();
    float f[kF_LM];
#pragma unroll
    for (int k = 0; k < kF_LM; ++k) f[k] = 0.0f;
    const Frame fr(sh);
    const float p0 = sh.par[0], p1 = sh.par[1], p2 = sh.par[2], p3 = sh.par[3];
    const float p4 = sh.par[4], p5 = sh.par[5], p6 = sh.par[6], p7 = sh.par[7];
    for (int64_t i = threadIdx.x; i < n; i += kThreads) {
        if (!take(m, i)) continue;
        float x, y, X, Y;
        fr.apply(c[i], x, y, X, Y);
        const float w = fmaf(p6, x, fmaf(p7, y, 1.0f));
        const float iw = 1.0f / w;
        const float u = fmaf(p0, x, fmaf(p1, y, p2)) * iw;
        const float v = fmaf(p3, x, fmaf(p4, y, p5)) * iw;
        const float ru = u - X, rv = v - Y;
        const float gu = iw * ru, gv = iw * rv, gw = iw * fmaf(u, ru, v * rv);
        a.f[0] = fmaf(gu, x, a.f[0]); a.f[1] = fmaf(gu, y, a.f[1]); a.f[2] += gu;
        a.f[3] = fmaf(gv, x, a.f[3]); a.f[4] = fmaf(gv, y, a.f[4]); a.f[5] += gv;
        a.f[6] = fmaf(-gw, x, a.f[6]); a.f[7] = fmaf(-gw, y, a.f[7]);
        a.f[8] = fmaf(ru, ru, fmaf(rv, rv, a.f[8]));
        a.tick();
        const float q = iw * iw;
        const float xx = x * x, xy = x * y, yy = y * y;
        const float qu = q * u, qv = q * v, qr = q * fmaf(u, u, v * v);
        f[0] = fmaf(q, xx, f[0]); f[1] = fmaf(q, xy, f[1]); f[2] = fmaf(q, yy, f[2]);
        f[3] = fmaf(q, x, f[3]);  f[4] = fmaf(q, y, f[4]);  f[5] += q;
        f[6] = fmaf(qu, xx, f[6]); f[7] = fmaf(qu, xy, f[7]); f[8] = fmaf(qu, yy, f[8]);
        f[9] = fmaf(qu, x, f[9]); f[10] = fmaf(qu, y, f[10]);
        f[11] = fmaf(qv, xx, f[11]); f[12] = fmaf(qv, xy, f[12]); f[13] = fmaf(qv, yy, f[13]);
        f[14] = fmaf(qv, x, f[14]); f[15] = fmaf(qv, y, f[15]);
        f[16] = fmaf(qr, xx, f[16]); f[17] = fmaf(qr, xy, f[17]); f[18] = fmaf(qr, yy, f[18]);
    }
    a.flush();
    block_reduce<kDF_LM, kF_LM>(a.s, f, sh);
}

// J^T J (8x8, FP32) from the FP32 sums of lm_pass: blocks
// sum q xb xb^T (twice), -sum q u xb b^T, -sum q v xb b^T and
// sum q (u^2 + v^2) b b^T.
__device__ void lm_assemble(const float *s, float A[64])
{
    // index of the moment {xx, xy, yy, x, y, 1} of xb_i xb_j
    const int mi[3][3] = {{0, 1, 3}, {1, 2, 4}, {3, 4, 5}};
    for (int i = 0; i < 64; ++i) A[i] = 0.0f;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A[i * 8 + j] = s[mi[i][j]];
            A[(3 + i) * 8 + 3 + j] = s[mi[i][j]];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 2; ++j) {
            const int k = mi[i][j];   // one of xx, xy, yy, x, y
            A[i * 8 + 6 + j] = A[(6 + j) * 8 + i] = -s[6 + k];
            A[(3 + i) * 8 + 6 + j] = A[(6 + j) * 8 + 3 + i] = -s[11 + k];
        }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) A[(6 + i) * 8 + 6 + j] = s[16 + mi[i][j]];
}

__device__ void write_empty(float *H_out, float *rms, int p, float rms_value)
{
    if (threadIdx.x < 9) H_out[9 * (int64_t)p + threadIdx.x] = 0.0f;
    if (threadIdx.x == 0 && rms) rms[p] = rms_value;
}

__global__ void __launch_bounds__(kThreads, 2)
refit_kernel(const float4 *__restrict__ corr, const int64_t *__restrict__ offsets,
             const uint8_t *__restrict__ mask, int lm_iters, float *__restrict__ H_out,
             int32_t *__restrict__ n_used, float *__restrict__ rms)
{
    __shared__ Shared sh;
    const int p = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const bool leader = threadIdx.x < 32;          // warp 0 runs the small solves
    const int64_t o0 = offsets[p];
    int64_t n = offsets[p + 1] - o0;
    if (n < 0) n = 0;
    const float4 *c = corr + o0;
    const uint8_t *m = mask ? mask + o0 : nullptr;
    float none[1] = {0.0f};

    // Pass 1: count and centroids.
    {
        DFAcc<5> a;
        a.zero();
        for (int64_t i = threadIdx.x; i < n; i += kThreads) {
            if (!take(m, i)) continue;
            const float4 q = c[i];
            a.f[0] += 1.0f; a.f[1] += q.x; a.f[2] += q.y; a.f[3] += q.z; a.f[4] += q.w;
            a.tick();
        }
        a.flush();
        block_reduce<5, 1>(a.s, none, sh);
    }
    const double cnt = sh.sum[0];
    const int64_t used = (int64_t)(cnt + 0.5);
    if (threadIdx.x == 0 && n_used) n_used[p] = (int32_t)used;
    if (used < 4) {
        write_empty(H_out, rms, p, 0.0f);
        return;
    }
    __syncthreads();                                // all have read sh.sum
    if (threadIdx.x == 0) {
        sh.mu1x = (float)(sh.sum[1] / cnt); sh.mu1y = (float)(sh.sum[2] / cnt);
        sh.mu2x = (float)(sh.sum[3] / cnt); sh.mu2y = (float)(sh.sum[4] / cnt);
    }
    __syncthreads();

    // Pass 2: mean distances to the centroids -> scales.
    {
        DFAcc<2> a;
        a.zero();
        const float m1x = sh.mu1x, m1y = sh.mu1y, m2x = sh.mu2x, m2y = sh.mu2y;
        for (int64_t i = threadIdx.x; i < n; i += kThreads) {
            if (!take(m, i)) continue;
            const float4 q = c[i];
            const float dx = q.x - m1x, dy = q.y - m1y, dX = q.z - m2x, dY = q.w - m2y;
            a.f[0] += sqrtf(fmaf(dx, dx, dy * dy));
            a.f[1] += sqrtf(fmaf(dX, dX, dY * dY));
            a.tick();
        }
        a.flush();
        block_reduce<2, 1>(a.s, none, sh);
    }
    if (threadIdx.x == 0) {
        const double d1 = sh.sum[0], d2 = sh.sum[1];
        sh.s1 = d1 > 0.0 ? (float)(1.4142135623730951 * cnt / d1) : 1.0f;
        sh.s2 = d2 > 0.0 ? (float)(1.4142135623730951 * cnt / d2) : 1.0f;
    }
    __syncthreads();

    // Pass 3: moments of the normalised points for the Eq. 2 normal matrix:
    // S_w = sum w {xx, xy, yy, x, y, 1} for w = 1, X, Y, X^2 + Y^2.
    {
        DFAcc<kDF_DLT> a;
        a.zero();
        const Frame fr(sh);
        for (int64_t i = threadIdx.x; i < n; i += kThreads) {
            if (!take(m, i)) continue;
            float x, y, X, Y;
            fr.apply(c[i], x, y, X, Y);
            const float mo[6] = {x * x, x * y, y * y, x, y, 1.0f};
            const float R = fmaf(X, X, Y * Y);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                a.f[k] += mo[k];
                a.f[6 + k] = fmaf(X, mo[k], a.f[6 + k]);
                a.f[12 + k] = fmaf(Y, mo[k], a.f[12 + k]);
                a.f[18 + k] = fmaf(R, mo[k], a.f[18 + k]);
            }
            a.tick();
        }
        a.flush();
        block_reduce<kDF_DLT, 1>(a.s, none, sh);
    }

    // DLT by the leader warp.  Rows of Eq. 2 per point: (xb, 0, -X xb) and
    // (0, -xb, Y xb), so M has blocks S_1 (twice), -S_X, -S_Y and S_R.
    if (leader) {
        for (int i = lane; i < 81; i += 32) sh.M[i] = 0.0;
        __syncwarp();
        if (lane < 9) {
            const int mi[3][3] = {{0, 1, 3}, {1, 2, 4}, {3, 4, 5}};
            const int i = lane / 3, j = lane % 3, k = mi[i][j];
            sh.M[i * 9 + j] = sh.sum[k];
            sh.M[(3 + i) * 9 + 3 + j] = sh.sum[k];
            sh.M[i * 9 + 6 + j] = -sh.sum[6 + k];
            sh.M[(6 + j) * 9 + i] = -sh.sum[6 + k];
            sh.M[(3 + i) * 9 + 6 + j] = -sh.sum[12 + k];
            sh.M[(6 + j) * 9 + 3 + i] = -sh.sum[12 + k];
            sh.M[(6 + i) * 9 + 6 + j] = sh.sum[18 + k];
        }
        __syncwarp();
        double dmax = lane < 9 ? sh.M[lane * 10] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        // pivot floor 2^-44 max diag: a shift far below the eigenvalue gap
        const bool ok = warp_cholesky<9, double>(sh.M, sh.L9, sh.r9, dmax * 5.684341886080802e-14);
        // diag(M^-1)_k = |L^-1 e_k|^2: lane k solves L z = e_k on its own
        double dk = -1.0;
        if (ok && lane < 9) {
            double z[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                double s = i == lane ? 1.0 : 0.0;
#pragma unroll
                for (int j = 0; j < i; ++j) s -= sh.L9[i * 9 + j] * z[j];
                z[i] = s * sh.r9[i];
            }
            dk = 0.0;
#pragma unroll
            for (int i = 0; i < 9; ++i) dk += z[i] * z[i];
        }
        int kb = lane;
        double best = dk;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int okb = __shfl_xor_sync(0xffffffffu, kb, o);
            if (ob > best || (ob == best && okb < kb)) { best = ob; kb = okb; }
        }
        double x = lane == kb ? 1.0 : 0.0;
        for (int it = 0; ok && it < kInvIters; ++it) {
            double y = warp_chol_solve<9, double>(sh.L9, sh.r9, x);
            const double ny = warp_sum_d(y * y), dot = warp_sum_d(y * x);
            y *= (dot < 0 ? -1.0 : 1.0) / sqrt(ny);
            double ch = fabs(y - x);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ch = fmax(ch, __shfl_xor_sync(0xffffffffu, ch, o));
            x = y;
            if (ch < 1e-11) break;      // far below the FP32 output
        }
        if (lane < 9) sh.v[lane] = ok ? x : 0.0;
        __syncwarp();
        // LM gauge h33 = 1 needs the normalised h33 away from zero (v has unit norm)
        const bool gauge = ok && fabs(sh.v[8]) >= 1e-3;
        if (gauge && lane < 8) {
            sh.pd[lane] = sh.v[lane] / sh.v[8];
            sh.par[lane] = (float)sh.pd[lane];
        }
        if (lane == 0) sh.go = gauge ? 1 : (ok ? 0 : -1);
    }
    __syncthreads();
    if (sh.go < 0) {                                // factorisation failed: no fit
        write_empty(H_out, rms, p, -1.0f);
        return;
    }

    // Levenberg-Marquardt: one pass at the start (it also gives the residual
    // of the DLT when lm_iters = 0), then one pass per trial step.
    bool lm_ok = false;
    if (sh.go) {
        lm_pass(c, m, n, sh);
        if (threadIdx.x == 0) {
            lm_assemble(sh.sumf, sh.A);
            for (int k = 0; k < 8; ++k) sh.g[k] = sh.sum[k];
            sh.F = 0.5 * sh.sum[8];
            float dmax = 0.0f;
            for (int k = 0; k < 8; ++k) dmax = fmaxf(dmax, sh.A[k * 9]);
            sh.mu = (double)(kTau * dmax);
            sh.nu = 2.0;
            sh.go = isfinite(sh.F) && isfinite(sh.mu) && sh.mu > 0.0 ? 1 : 0;
        }
        __syncthreads();
        lm_ok = sh.go != 0;
        __syncthreads();
        for (int it = 0; lm_ok && it < lm_iters; ++it) {
            // Trial step (J^T J + mu I) d = -g by the leader warp.
            if (leader) {
                if (lane < 8) {
                    for (int k = 0; k < 8; ++k) sh.S8[lane * 8 + k] = sh.A[lane * 8 + k];
                    sh.S8[lane * 9] += (float)sh.mu;
                }
                __syncwarp();
                const bool ok = warp_cholesky<8, float>(sh.S8, sh.L8, sh.r8, 0.0f);
                int go = 2;                 // not positive definite: a rejected step
                if (ok) {
                    const float dl = warp_chol_solve<8, float>(sh.L8, sh.r8, lane < 8 ? (float)-sh.g[lane] : 0.0f);
                    const double dd = lane < 8 ? (double)dl : 0.0;
                    const double pp = lane < 8 ? sh.pd[lane] : 0.0;
                    const double nd = warp_sum_d(dd * dd), np = warp_sum_d(pp * pp);
                    if (!(sqrt(nd) > kEpsStep * (sqrt(np) + kEpsStep))) {
                        go = 0;             // below FP32 resolution (or not finite): converged
                    } else {
                        go = 1;
                        if (lane < 8) {
                            sh.d[lane] = dd;
                            sh.par[lane] = (float)(pp + dd);
                        }
                    }
                }
                if (lane == 0) {
                    if (go == 2) {
                        sh.mu *= sh.nu;
                        sh.nu *= 2.0;
                        if (!isfinite(sh.mu)) go = 0;
                    }
                    sh.go = go;
                }
            }
            __syncthreads();
            const int go = sh.go;
            __syncthreads();                // all have read go before it changes
            if (go == 0) break;
            if (go == 2) continue;
            lm_pass(c, m, n, sh);
            if (threadIdx.x == 0) {
                const double Fn = 0.5 * sh.sum[8];
                double pred = 0.0;
                for (int k = 0; k < 8; ++k) pred += sh.d[k] * (sh.mu * sh.d[k] - sh.g[k]);
                pred *= 0.5;
                const double rho = (sh.F - Fn) / pred;
                const double noise = kCostNoise * sh.F;
                const bool accept = isfinite(Fn) && (rho > 0.0 || (pred <= noise && Fn <= sh.F + noise));
                if (accept) {
                    for (int k = 0; k < 8; ++k) { sh.pd[k] += sh.d[k]; sh.g[k] = sh.sum[k]; }
                    lm_assemble(sh.sumf, sh.A);
                    sh.F = Fn;
                    const double t = rho > 0.0 && rho < 1.0 ? 2.0 * rho - 1.0 : 1.0;
                    sh.mu *= fmax(1.0 / 3.0, 1.0 - t * t * t);
                    sh.nu = 2.0;
                } else {
                    sh.mu *= sh.nu;
                    sh.nu *= 2.0;
                }
            }
            __syncthreads();                // the update is visible to the next trial
        }
    }
    __syncthreads();

    // Back to pixels: H = T2^-1 Hn T1, unit Frobenius norm.
    if (threadIdx.x == 0) {
        double hn[9];
        if (lm_ok) {
            for (int k = 0; k < 8; ++k) hn[k] = sh.pd[k];
            hn[8] = 1.0;
        } else {
            for (int k = 0; k < 9; ++k) hn[k] = sh.v[k];
        }
        const double s1 = sh.s1, s2 = sh.s2;
        const double a1x = sh.mu1x, a1y = sh.mu1y, a2x = sh.mu2x, a2y = sh.mu2y;
        // Hn T1: columns scale by s1, the third picks up -s1 mu1.
        double B[9];
        for (int r = 0; r < 3; ++r) {
            B[r * 3 + 0] = hn[r * 3 + 0] * s1;
            B[r * 3 + 1] = hn[r * 3 + 1] * s1;
            B[r * 3 + 2] = hn[r * 3 + 2] - s1 * (hn[r * 3 + 0] * a1x + hn[r * 3 + 1] * a1y);
        }
        // T2^-1 B: rows 0, 1 scaled by 1/s2 plus mu2 times row 2.
        double h[9];
        for (int col = 0; col < 3; ++col) {
            h[0 + col] = B[0 + col] / s2 + a2x * B[6 + col];
            h[3 + col] = B[3 + col] / s2 + a2y * B[6 + col];
            h[6 + col] = B[6 + col];
        }
        store_frob(h, H_out + 9 * (int64_t)p);
        if (rms) rms[p] = lm_ok ? (float)(sqrt(2.0 * sh.F / cnt) / s2) : -1.0f;
    }
}

}  // namespace
}  // namespace aca

extern "C" aca_status aca_refit(const float *corr, const int64_t *offsets, const uint8_t *mask, int32_t P,
                                int32_t lm_iters, float *H, int32_t *n_used, float *rms, void *stream)
{
    using namespace aca;
    if (P < 0) return set_error(ACA_ERR_INVALID_ARG, "aca_refit: P = %d < 0", (int)P);
    if (lm_iters < 0 || lm_iters > 10000)
        return set_error(ACA_ERR_INVALID_ARG, "aca_refit: lm_iters = %d outside [0, 10000]", (int)lm_iters);
    if (P == 0) return ACA_OK;
    if (!corr || !offsets || !H) return set_error(ACA_ERR_INVALID_ARG, "aca_refit: null corr, offsets or H");
    if (!aligned16(corr)) return set_error(ACA_ERR_INVALID_ARG, "aca_refit: corr must be 16-byte aligned");
    refit_kernel<<<P, kThreads, 0, as_stream(stream)>>>(reinterpret_cast<const float4 *>(corr), offsets, mask,
                                                        lm_iters, H, n_used, rms);
    return check_launch("aca_refit");
}
