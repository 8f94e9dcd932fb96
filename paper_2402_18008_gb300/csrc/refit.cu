// Refit of one homography per problem on all of its masked correspondences:
// the global optimisation with all inliers that ends the RANSAC pipeline
// (Sec. 6.2, stage 5).  One block per problem:
//   1. Hartley normalisation of each side: centroid to the origin, mean
//      distance sqrt(2) (the centroids in a first pass over the points, the
//      mean distances in a second);
//   2. normalised DLT: the 9x9 normal matrix M of the two Eq. 2 rows of every
//      point (from moments of the centred points taken in the same second
//      pass and scaled afterwards), its eigenvector of the smallest eigenvalue by inverse
//      iteration on a Cholesky factor, started from e_k with k the largest
//      diagonal entry of M^-1 (sum_j v_j[k]^2 / lambda_j, dominated by the
//      smallest eigenvalue's vector, so e_k has a component of at least 1/3
//      along it);
//   3. Levenberg-Marquardt on the reprojection error in the normalised frames
//      (the eight entries of H with h33 = 1), with the damping schedule of
//      Madsen, Nielsen & Tingleff, "Methods for non-linear least squares
//      problems" (2004), Alg. 3.16, with tau = 1e-6, the value they give
//      for a start believed close to the minimiser; when the first trial
//      step is rejected the start was not that close, and mu becomes their
//      value for a poorer start, 1e-3 max diag(J^T J) (nu unchanged).  Each
//      trial step is one pass.
//
// Precision and speed on GB300, where FP64 runs at 1/64 of the FP32 rate and
// each FP64 instruction (conversions included) of a serial chain costs
// hundreds of cycles:
//   - per-point arithmetic is FP32 on O(1) normalised coordinates;
//   - sums whose cancellation matters (the DLT moments, the gradient J^T r
//     and the cost) are double-float: FP32 partials over chunks of 8 points,
//     TwoSum accumulation, then per warp a transposition through shared
//     memory (lane k adds up value k of the 32 lanes; in two rounds for the
//     26 sums of the DLT pass) and a sum over the warps, all in a fixed
//     order (deterministic); J^T J, which only shapes the step, is summed in
//     FP32;
//   - the DLT eigenvector is refined to double-float accuracy (FP32 factor,
//     double-float residuals) when it is the result (lm_iters = 0), and is
//     FP32 when it only starts LM, which converges to the same minimiser
//     from either start;
//   - the 8x8 LM steps are FP32 (an inexact step only slows the iteration;
//     its fixed point is set by the gradient); the parameters and the cost
//     are double-float, and so is the map back to pixels, whose translation
//     column cancels; nothing on the LM path uses FP64;
//   - the small solves run in registers, every lane of the leader warp
//     computing the same values (no shuffle or shared-memory access in
//     their dependent chains);
//   - the cost of a trial point carries FP32 rounding noise of about 2^-16
//     relative, so near the optimum, where the predicted decrease is below
//     that noise, a step is accepted unless the cost rises by more than the
//     noise: the gain ratio could not tell such steps apart; after two such
//     accepted steps in a row that also moved the parameters by less than
//     2^-20 LM stops, since what further steps change is rounding (without
//     that, a few pairs random-walked at the noise floor through the whole
//     step budget; the size condition keeps slow linear convergence, as on
//     sets with many outliers, going).
#include <math.h>

#include <map>
#include <mutex>

#include "common.cuh"
#include "fp32.cuh"
#include "pdl.cuh"

namespace aca {
namespace {

constexpr int kThreads = 256;         // 2 blocks (of <= 128 registers a thread) per SM
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 8;
constexpr int kPad = 33;              // transposition row stride (floats per value, padded)
constexpr int kRefineMax = 16;        // refinement steps of the DLT eigenvector (lm_iters = 0), at most
constexpr int kBisect = 12;           // bisection steps for its shift, when it needs one
constexpr float kSlow = 0.01f;        // contraction per step above which the refinement shifts
constexpr float kTau = 1e-6f;         // mu0 = tau * max diag(J^T J): the value given for a start
                                      // close to the minimiser (the DLT of the same points)
constexpr float kTauPoor = 1e-3f;     // mu after a rejected first trial: the value for a poorer start
constexpr float kEpsStep = 5.9604644775390625e-8f;   // 2^-24: parameters are used in FP32
constexpr float kCostNoise = 1.52587890625e-05f;     // 2^-16: FP32 noise of the cost, relative
constexpr int kQuietSteps = 2;        // LM stops after this many accepted quiet steps in a row
constexpr float kQuietStep = 9.5367431640625e-07f;   // 2^-20: a quiet step's size, relative to the parameters

constexpr int kDF_DLT = 24;           // moments of the normalised points (the DLT)
constexpr int kDF_P2 = kDF_DLT + 2;   // double-float sums of pass 2 (moments + 2 distance sums)
constexpr int kDF_LM = 9;             // gradient (8) and cost (1)
constexpr int kF_LM = 19;             // J^T J moments
constexpr int kTr = kDF_LM * 2 * kPad + kF_LM * kPad;   // transposition floats per warp (LM pass)
static_assert(kDF_LM + kF_LM <= 32, "one lane per LM sum");

struct Shared {
    float tr[kWarps][kTr];            // per-warp transposition scratch
    DF wpart[kWarps][kDF_P2];         // per-warp double-float sums
    float wpartf[kWarps][kF_LM];
    DF sum[kDF_P2];                   // block sums (leader warp), renormalised
    float sumf[kF_LM];
    DF mdf[kDF_DLT];                  // the DLT moments of the normalised points (lm_iters = 0)
    DF Mdf[45];                       // the DLT normal matrix from them, packed lower triangle
    DF hn[9];                         // the DLT fit in the normalised frames
    float par[8];                     // parameters broadcast to the pass
    float mu1x, mu1y, s1, mu2x, mu2y, s2, cnt;
    int64_t used;
    int go;                           // leader -> block decision
    // Levenberg-Marquardt state (leader warp)
    float Asum[kF_LM];                // the FP32 sums of J^T J at pd
    float g[8];                       // J^T r at pd
    DF F;                             // ||r||^2 / 2 at pd
    DF pd[8];                         // parameters
    float d[8], mu, nu;               // step, damping
    float mu_poor;                    // kTauPoor * max diag(J^T J) at the start
    int it;                           // trial steps taken
    int quiet;                        // consecutive accepted quiet steps (small, and below the cost's noise)
    int small;                        // the evaluated step is below kQuietStep of the parameters
};

// Double-float accumulator: FP32 partials per chunk of kChunk slots, then
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
    // after `slots` more slots (the same count in every lane)
    __device__ void tick(int slots)
    {
        c += slots;
        if (c >= kChunk) flush();
    }
};

__device__ __forceinline__ DF df_renorm(DF x)
{
    const float s = F_ADD(x.h, x.l);
    return DF{s, F_SUB(x.l, F_SUB(s, x.h))};
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <typename T>
__device__ __forceinline__ T warp_max(T x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Per-warp sums of a pass: each lane writes its K double-float and KF FP32
// values to the warp's scratch; lane k < K adds up double-float value k over
// the 32 lanes, lane K + k value k of the FP32 ones; results to wpart.  The
// caller then synchronises the block and the leader warp calls leader_sums.
template <int K, int KF>
__device__ void warp_partials(const DF (&s)[K], const float *f, Shared &sh)
{
    static_assert(K * 2 * kPad + KF * kPad <= kTr, "pass does not fit the transposition scratch");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *t = sh.tr[warp];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        t[(k * kPad + lane) * 2] = s[k].h;
        t[(k * kPad + lane) * 2 + 1] = s[k].l;
    }
#pragma unroll
    for (int k = 0; k < KF; ++k) t[K * 2 * kPad + k * kPad + lane] = f[k];
    __syncwarp();
    if (lane < K) {
        const float *r = t + lane * kPad * 2;
        DF a{r[0], r[1]};
        for (int i = 1; i < 32; ++i) a = df_add(a, DF{r[2 * i], r[2 * i + 1]});
        sh.wpart[warp][lane] = df_renorm(a);
    } else if (lane < K + KF) {
        const float *r = t + K * 2 * kPad + (lane - K) * kPad;
        float a = r[0];
        for (int i = 1; i < 32; ++i) a += r[i];
        sh.wpartf[warp][lane - K] = a;
    }
}

// Per-warp sums of the double-float values [K0, K0 + KN) of s by
// transposition, for passes with more values than the scratch holds at once
// (the DLT moments: two rounds, once per problem); same order as
// warp_partials.
template <int K0, int KN, int K>
__device__ void warp_partials_part(const DF (&s)[K], Shared &sh)
{
    static_assert(KN * 2 * kPad <= kTr && K0 + KN <= K, "round does not fit the transposition scratch");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *t = sh.tr[warp];
#pragma unroll
    for (int k = 0; k < KN; ++k) {
        t[(k * kPad + lane) * 2] = s[K0 + k].h;
        t[(k * kPad + lane) * 2 + 1] = s[K0 + k].l;
    }
    __syncwarp();
    if (lane < KN) {
        const float *r = t + lane * kPad * 2;
        DF a{r[0], r[1]};
        for (int i = 1; i < 32; ++i) a = df_add(a, DF{r[2 * i], r[2 * i + 1]});
        sh.wpart[warp][K0 + lane] = df_renorm(a);
    }
    __syncwarp();
}

// Leader warp, after the block barrier: sums over the warps into sh.sum
// (double-float) and sh.sumf; visible to the leader warp on return.
template <int K, int KF>
__device__ void leader_sums(Shared &sh)
{
    const int lane = threadIdx.x & 31;
    if (lane < K) {
        DF a = sh.wpart[0][lane];
#pragma unroll
        for (int w = 1; w < kWarps; ++w) a = df_renorm(df_add(a, sh.wpart[w][lane]));
        sh.sum[lane] = df_renorm(a);
    } else if (lane < K + KF) {
        float a = sh.wpartf[0][lane - K];
#pragma unroll
        for (int w = 1; w < kWarps; ++w) a += sh.wpartf[w][lane - K];
        sh.sumf[lane - K] = a;
    }
    __syncwarp();
}

// Small dense algebra in registers, run redundantly by every lane of the
// leader warp: each lane holds the whole packed matrix, all lanes execute the
// same instructions on the same values (so they agree bit for bit), and no
// step of the dependent chain is a shuffle or a shared-memory access.  Those
// go through the SM's memory-instruction queue, which the other resident
// block's point loads keep full; a chain of shuffles there runs an order of
// magnitude slower than on an idle SM.  Packed lower triangle, row-major:
// entry (i, j), j <= i, at tri(i, j).
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// In-place Cholesky L L^T of the packed n x n matrix a (right-looking: after
// column j the trailing block holds S - sum_{k <= j} l_k l_k^T), pivots below
// `floor` raised to it; rd[j] = 1 / L[j][j].  False on a non-positive or
// non-finite pivot.  The pivot's reciprocal square root is the hardware
// approximation (a few ulp): every factor here only steers an iteration
// (the LM step, the DLT start, the refinement's preconditioner), and it
// halves the dependent chain of a column.
template <int n>
__device__ __forceinline__ bool reg_cholesky(float (&a)[n * (n + 1) / 2], float (&rd)[n], float floor)
{
    bool ok = true;
#pragma unroll
    for (int j = 0; j < n; ++j) {
        float d = a[tri(j, j)];
        if (d < floor) d = floor;
        ok = ok && d > 0.0f && isfinite(d);
        const float r = rsqrtf(d), l = d * r;
        a[tri(j, j)] = l;
        rd[j] = r;
#pragma unroll
        for (int i = j + 1; i < n; ++i) a[tri(i, j)] *= r;
#pragma unroll
        for (int i = j + 1; i < n; ++i)
#pragma unroll
            for (int k = j + 1; k <= i; ++k) a[tri(i, k)] = fmaf(-a[tri(i, j)], a[tri(k, j)], a[tri(i, k)]);
    }
    return ok;
}

// x := (L L^T)^-1 x with the factor of reg_cholesky.
template <int n>
__device__ __forceinline__ void reg_chol_solve(const float (&a)[n * (n + 1) / 2], const float (&rd)[n], float (&x)[n])
{
#pragma unroll
    for (int i = 0; i < n; ++i) {
#pragma unroll
        for (int k = 0; k < i; ++k) x[i] = fmaf(-a[tri(i, k)], x[k], x[i]);
        x[i] *= rd[i];
    }
#pragma unroll
    for (int i = n - 1; i >= 0; --i) {
#pragma unroll
        for (int k = i + 1; k < n; ++k) x[i] = fmaf(-a[tri(k, i)], x[k], x[i]);
        x[i] *= rd[i];
    }
}

// x[lane] for lane < n (else 0) without an indexed register access.
template <int n>
__device__ __forceinline__ float lane_pick(const float (&x)[n], int lane)
{
    float v = 0.0f;
#pragma unroll
    for (int i = 0; i < n; ++i) v = lane == i ? x[i] : v;
    return v;
}

__device__ __forceinline__ bool take(const uint8_t *mask, int64_t i) { return mask == nullptr || mask[i] != 0; }

// The block's problem: its correspondences and mask bytes in global memory,
// and a copy of the first nr of them (points and mask bytes) in shared
// memory, filled by the first pass.  The later passes read that copy, so
// for problems that fit it (most of them) only the first pass touches
// global memory; the rest of a larger problem is read from global memory
// (L2) on every pass.
extern __shared__ __align__(16) unsigned char s_pts[];   // cap points, then cap mask bytes

struct Points {
    const float4 *c;
    const uint8_t *m;                 // null: every point is used
    int64_t n;
    int nr;                           // points in the shared copy
    int cap;                          // its capacity
    __device__ float4 *sc() const { return reinterpret_cast<float4 *>(s_pts); }
    __device__ uint8_t *sm() const { return s_pts + (size_t)cap * sizeof(float4); }
};

// Calls f(q, t) for every slot of the block's problem, and step(U) after
// each U slots: the block's threads stride over the points, all of them
// taking the same number of steps, and t says whether the slot holds a used
// point (q is zero otherwise), so the per-point code runs without divergence
// and the accumulators' chunk flushes (in step, one copy of the code a loop)
// happen on the same step in every lane; f must make an unused slot add
// nothing.  Each thread keeps U loads in flight (the passes are otherwise
// bound by one memory round trip per step).  A correspondence is loaded
// whether or not its mask byte is set, so both loads are in flight at once;
// the masked-out points share cache sectors with the used ones.
template <int U, class Fn, class Step>
__device__ __forceinline__ void for_global(const Points &P, int64_t from, bool fill, Fn &&f, Step &&step)
{
    for (int64_t b0 = from; b0 < P.n; b0 += U * kThreads) {
        float4 q[U];
        bool t[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t i = b0 + (int64_t)(u * kThreads) + threadIdx.x;
            const bool in = i < P.n;
            q[u] = in ? P.c[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            t[u] = in && take(P.m, i);
        }
        if (fill) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = b0 + (int64_t)(u * kThreads) + threadIdx.x;
                if (i < P.nr) {
                    P.sc()[i] = q[u];
                    P.sm()[i] = t[u] ? 1 : 0;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) f(t[u] ? q[u] : make_float4(0.0f, 0.0f, 0.0f, 0.0f), t[u]);
        step(U);
    }
}

constexpr int kUnroll = 4;

// The first pass: every point from global memory, eight loads in flight a
// thread (first touch: HBM latency), filling the shared copy.
template <class Fn, class Step>
__device__ __forceinline__ void for_points_fill(const Points &P, Fn &&f, Step &&step)
{
    for_global<8>(P, 0, true, f, step);
}

// A later pass: the shared copy (US loads in flight a thread), then the rest
// from global memory (UG).
template <int US = kUnroll, int UG = kUnroll, class Fn, class Step>
__device__ __forceinline__ void for_points(const Points &P, Fn &&f, Step &&step)
{
    for (int b0 = 0; b0 < P.nr; b0 += US * kThreads) {
        float4 q[US];
        bool t[US];
#pragma unroll
        for (int u = 0; u < US; ++u) {
            const int i = b0 + u * kThreads + (int)threadIdx.x;
            const bool in = i < P.nr;
            q[u] = in ? P.sc()[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            t[u] = in && P.sm()[i] != 0;
        }
#pragma unroll
        for (int u = 0; u < US; ++u) f(t[u] ? q[u] : make_float4(0.0f, 0.0f, 0.0f, 0.0f), t[u]);
        step(US);
    }
    for_global<UG>(P, P.nr, false, f, step);
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

// One LM pass at the parameters in sh.par: per-warp sums of, with
// xb = (x, y, 1), b = (x, y), q = 1/w^2:
//   double-float: g = J^T r (u rows: r_u xb / w; v rows: r_v xb / w;
//                 perspective: -(u r_u + v r_v) b / w) and ||r||^2;
//   FP32: sum q {xx, xy, yy, x, y, 1}, sum q u {xx, xy, yy, x, y},
//         sum q v {...}, sum q (u^2 + v^2) {xx, xy, yy}, the blocks of J^T J.
// Ends with a block barrier; the leader warp then calls leader_sums.
__device__ void lm_pass(const Points &P, Shared &sh)
{
    DFAcc<kDF_LM> a;
    a.zero();
    float f[kF_LM];
#pragma unroll
    for (int k = 0; k < kF_LM; ++k) f[k] = 0.0f;
    const Frame fr(sh);
    const float p0 = sh.par[0], p1 = sh.par[1], p2 = sh.par[2], p3 = sh.par[3];
    const float p4 = sh.par[4], p5 = sh.par[5], p6 = sh.par[6], p7 = sh.par[7];
    for_points(P, [&](float4 pt, bool t) {
        float x, y, X, Y;
        fr.apply(pt, x, y, X, Y);
        const float w = fmaf(p6, x, fmaf(p7, y, 1.0f));
        // an unused slot: 1/w = 0 zeroes every gradient and J^T J term
        const float iw = t ? 1.0f / w : 0.0f;
        const float u = fmaf(p0, x, fmaf(p1, y, p2)) * iw;
        const float v = fmaf(p3, x, fmaf(p4, y, p5)) * iw;
        const float ru = u - X, rv = v - Y;
        const float gu = iw * ru, gv = iw * rv, gw = iw * fmaf(u, ru, v * rv);
        a.f[0] = fmaf(gu, x, a.f[0]); a.f[1] = fmaf(gu, y, a.f[1]); a.f[2] += gu;
        a.f[3] = fmaf(gv, x, a.f[3]); a.f[4] = fmaf(gv, y, a.f[4]); a.f[5] += gv;
        a.f[6] = fmaf(-gw, x, a.f[6]); a.f[7] = fmaf(-gw, y, a.f[7]);
        a.f[8] += t ? fmaf(ru, ru, rv * rv) : 0.0f;
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
    }, [&](int slots) { a.tick(slots); });
    a.flush();
    warp_partials<kDF_LM, kF_LM>(a.s, f, sh);
    __syncthreads();
}

// Moment index of xb_i xb_j, xb = (x, y, 1), in {xx, xy, yy, x, y, 1}.
__host__ __device__ constexpr int mom(int i, int j)
{
    return i == 2 ? (j == 2 ? 5 : 3 + j) : (j == 2 ? 3 + i : i + j);
}

// Entry (r, c), r >= c, of the DLT normal matrix in the 24 moments S_1, S_X,
// S_Y, S_R (6 each): 1 + index, negated for a negative entry, 0 for zero.
__host__ __device__ constexpr int dlt_code(int r, int c)
{
    return r < 3   ? 1 + mom(r, c)
           : r < 6 ? (c < 3 ? 0 : 1 + mom(r - 3, c - 3))
           : c < 3 ? -(1 + 6 + mom(c, r - 6))
           : c < 6 ? -(1 + 12 + mom(c - 3, r - 6))
                   : 1 + 18 + mom(r - 6, c - 6);
}

// Entry (r, c), r >= c, of J^T J (8 x 8) in the 19 FP32 sums of lm_pass:
// blocks sum q xb xb^T (twice), -sum q u xb b^T, -sum q v xb b^T and
// sum q (u^2 + v^2) b b^T; same code convention.
__host__ __device__ constexpr int jtj_code(int r, int c)
{
    return r < 3   ? 1 + mom(r, c)
           : r < 6 ? (c < 3 ? 0 : 1 + mom(r - 3, c - 3))
           : c < 3 ? -(1 + 6 + mom(c, r - 6))
           : c < 6 ? -(1 + 11 + mom(c - 3, r - 6))
                   : 1 + 16 + mom(r - 6, c - 6);
}

// The packed matrix from its sums: the DLT normal matrix (n = 9) or J^T J
// (n = 8).
template <int n, int K>
__device__ __forceinline__ void fill_packed(const float (&m)[K], float (&a)[n * (n + 1) / 2])
{
    static_assert((n == 9 && K == kDF_DLT) || (n == 8 && K == kF_LM), "DLT (9, 24 sums) or J^T J (8, 19 sums)");
#pragma unroll
    for (int r = 0; r < n; ++r)
#pragma unroll
        for (int c = 0; c <= r; ++c) {
            const int k = n == 9 ? dlt_code(r, c) : jtj_code(r, c);
            a[tri(r, c)] = k == 0 ? 0.0f : k > 0 ? m[k - 1] : -m[-k - 1];
        }
}

// Leader warp, every lane: the FP32 normalised DLT from the 24 moments of
// the normalised points: M, its Cholesky factor (pivot floor 2^-20 of the
// largest diagonal entry: near FP32's rounding of M, far below the
// eigenvalue gap), the start e_k with k the largest diagonal entry of M^-1
// (the squared column norms of L^-1), then three inverse-iteration steps
// (error ratio lambda1 / lambda2 per step).  False if the factorisation
// failed.
__device__ __forceinline__ bool dlt_fp32(const float (&m)[kDF_DLT], float (&a)[45], float (&rd)[9], float (&x)[9])
{
    fill_packed<9>(m, a);
    float dmax = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) dmax = fmaxf(dmax, a[tri(k, k)]);
    if (!reg_cholesky<9>(a, rd, dmax * 9.5367431640625e-07f)) return false;
    float best = -1.0f;
    int kb = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        float z[9], dk = 0.0f;
#pragma unroll
        for (int i = k; i < 9; ++i) {
            float t = i == k ? 1.0f : 0.0f;
#pragma unroll
            for (int j = k; j < i; ++j) t = fmaf(-a[tri(i, j)], z[j], t);
            z[i] = t * rd[i];
            dk = fmaf(z[i], z[i], dk);
        }
        if (dk > best) {
            best = dk;
            kb = k;
        }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) x[i] = i == kb ? 1.0f : 0.0f;
    for (int it = 0; it < 3; ++it) {
        float y[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) y[i] = x[i];
        reg_chol_solve<9>(a, rd, y);
        float ny = 0.0f, dot = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            ny = fmaf(y[i], y[i], ny);
            dot = fmaf(y[i], x[i], dot);
        }
        const float sc = (dot < 0.0f ? -1.0f : 1.0f) / sqrtf(ny);
#pragma unroll
        for (int i = 0; i < 9; ++i) x[i] = y[i] * sc;
    }
    return true;
}

__device__ __forceinline__ bool dlt_start(const float (&m)[kDF_DLT], float (&x)[9])
{
    float a[45], rd[9];
    return dlt_fp32(m, a, rd, x);
}

// (a.h + a.l)(b.h + b.l) to double-float accuracy (the a.l b.l term is below it).
__device__ __forceinline__ DF df_mul2(DF a, DF b)
{
    const DF p = df_prod(a.h, b.h);
    return DF{p.h, fmaf(a.h, b.l, fmaf(a.l, b.h, p.l))};
}

// a / b in double-float: the quotient's leading part, then the remainder's.
__device__ __forceinline__ DF df_div2(DF a, DF b)
{
    const float q = a.h / b.h;
    const DF r = df_sub(a, df_mul2(b, DF{q, 0.0f}));
    return DF{q, df_round(r) / b.h};
}

// Leader warp, every lane: the DLT eigenvector when it is the result, to
// double-float accuracy without FP64 (fac: 72 floats of scratch, for the
// FP32 factor and M v).  The FP32 start of dlt_fp32, then steps of
// eigenvector refinement: with the Rayleigh quotient
// lambda = v^T M v / v^T v and the residual r = M v - lambda v, both in
// double-float from the double-float matrix Mdf (shared, packed), the
// correction solves (M - sigma I) d = r with the FP32 factor and keeps the
// part of d orthogonal to v: v := v - (d - (d.v / v.v) v).  Against the
// exact correction (M - lambda I)^-1 r this errs by
// (lambda - sigma) / (lambda_j - sigma) on each other eigendirection j and
// by FP32 rounding relative to the complement's conditioning, so each step
// shrinks the error by about
// max((lambda_min - sigma) / (lambda_2 - sigma), 2^-24 lambda_max / lambda_2),
// The first steps use sigma = 0, which suffices for inlier sets
// (lambda_min / lambda_2 ~ 1e-4); when a step shrinks the correction by less
// than kSlow (a DLT over sets with many outliers, where lambda_min is near
// lambda_2 and unshifted inverse iteration crawls), sigma moves to just
// below lambda_min (bisection on whether M - sigma I factors, from the
// Rayleigh quotient down), the factor with it, and three inverse-iteration
// steps with that factor bring v close before refining on.  Steps until the
// correction is below 2^-36 of v (far below what the FP32 result resolves,
// above the double-float residual's floor of about 2^-48 lambda_max /
// lambda_2; two or three steps for inlier sets), kRefineMax at most.
// The factor of M - sigma I (pivot floor 2^-20 of M's largest diagonal
// entry) to the scratch; false if it failed.
__device__ __forceinline__ bool store_factor(const float (&m)[kDF_DLT], float sigma, float *fac)
{
    float a[45], rd[9];
    fill_packed<9>(m, a);
    float dmax = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        dmax = fmaxf(dmax, a[tri(k, k)]);
        a[tri(k, k)] -= sigma;
    }
    const bool ok = reg_cholesky<9>(a, rd, dmax * 9.5367431640625e-07f);
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int e = 0; e < 45; ++e) fac[e] = a[e];
#pragma unroll
        for (int i = 0; i < 9; ++i) fac[45 + i] = rd[i];
    }
    __syncwarp();
    return ok;
}

// The largest sigma in [0, hi] at which M - sigma I still factors in FP32
// (every pivot positive), by kBisect bisection steps: M's smallest
// eigenvalue lies within FP32 rounding of M above it.
__device__ __forceinline__ float shift_below_min(const float (&m)[kDF_DLT], float hi)
{
    float lo = 0.0f;
    for (int b = 0; b < kBisect; ++b) {
        const float mid = 0.5f * (lo + hi);
        float a[45], rd[9];
        fill_packed<9>(m, a);
#pragma unroll
        for (int k = 0; k < 9; ++k) a[tri(k, k)] -= mid;
        if (reg_cholesky<9>(a, rd, 0.0f)) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool dlt_refined(const DF *Mdf, const float (&m)[kDF_DLT], float *fac, DF (&v)[9])
{
    {
        float a[45], rd[9], x[9];
        if (!dlt_fp32(m, a, rd, x)) return false;
        // the factor to the scratch (every lane writes the same values)
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int e = 0; e < 45; ++e) fac[e] = a[e];
#pragma unroll
            for (int i = 0; i < 9; ++i) fac[45 + i] = rd[i];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = DF{x[i], 0.0f};
    }
    __syncwarp();
    const int lane = threadIdx.x & 31;
    bool shifted = false;
    float prev = 0.0f;
    for (int it = 0; it < kRefineMax; ++it) {
        // w = M v: lane i < 9 forms row i, through the scratch to every lane
        {
            const int i = lane < 9 ? lane : 0;
            DF t{0.0f, 0.0f};
#pragma unroll
            for (int j = 0; j < 9; ++j) t = df_add(t, df_mul2(Mdf[i >= j ? tri(i, j) : tri(j, i)], v[j]));
            if (lane < 9) {
                fac[54 + 2 * lane] = t.h;
                fac[55 + 2 * lane] = t.l;
            }
        }
        __syncwarp();
        DF w[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) w[i] = DF{fac[54 + 2 * i], fac[55 + 2 * i]};
        __syncwarp();
        DF num{0.0f, 0.0f}, den{0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            num = df_add(num, df_mul2(v[i], w[i]));
            den = df_add(den, df_mul2(v[i], v[i]));
        }
        const DF lam = df_div2(num, den);
        float d[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = df_round(df_sub(w[i], df_mul2(lam, v[i])));
        {
            float a[45], rd[9];
#pragma unroll
            for (int e = 0; e < 45; ++e) a[e] = fac[e];
#pragma unroll
            for (int i = 0; i < 9; ++i) rd[i] = fac[45 + i];
            reg_chol_solve<9>(a, rd, d);
        }
        float dv = 0.0f, vv = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            dv = fmaf(d[i], v[i].h, dv);
            vv = fmaf(v[i].h, v[i].h, vv);
        }
        const float c = dv / vv;
        float dmax = 0.0f, vmax = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const float di = fmaf(c, v[i].h, -d[i]);
            dmax = fmaxf(dmax, fabsf(di));
            vmax = fmaxf(vmax, fabsf(v[i].h));
            v[i] = df_renorm(df_add(v[i], DF{di, 0.0f}));
        }
        if (!(dmax > 1.4551915228366852e-11f * vmax)) break;      // 2^-36; also ends on NaN
        // slow contraction (lambda_min not small against lambda_2): shift
        // the factor to just below lambda_min, the Rayleigh quotient bounding
        // it from above
        if (!shifted && it >= 1 && dmax > kSlow * prev) {
            shifted = true;
            const float rq = df_round(lam);
            const float sigma = shift_below_min(m, rq > 0.0f ? rq : 0.0f);
            if (!store_factor(m, sigma, fac)) return false;
            // v is still far from the eigenvector: three FP32 inverse-iteration
            // steps with the shifted factor (error ratio
            // (lambda_min - sigma) / (lambda_2 - sigma) per step) before the
            // refinement resumes
            float a[45], rd[9], x[9];
#pragma unroll
            for (int e = 0; e < 45; ++e) a[e] = fac[e];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                rd[i] = fac[45 + i];
                x[i] = v[i].h;
            }
            for (int k = 0; k < 3; ++k) {
                float y[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) y[i] = x[i];
                reg_chol_solve<9>(a, rd, y);
                float ny = 0.0f, dot = 0.0f;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    ny = fmaf(y[i], y[i], ny);
                    dot = fmaf(y[i], x[i], dot);
                }
                const float sc = (dot < 0.0f ? -1.0f : 1.0f) / sqrtf(ny);
#pragma unroll
                for (int i = 0; i < 9; ++i) x[i] = y[i] * sc;
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) v[i] = DF{x[i], 0.0f};
        }
        prev = dmax;
    }
    return true;
}

// v[lane] for lane < 9 (else zero) without an indexed register access.
__device__ __forceinline__ DF lane_pick_df(const DF (&v)[9], int lane)
{
    DF r{0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < 9; ++i) r = lane == i ? v[i] : r;
    return r;
}

// Leader warp: the DLT as the result (lm_iters = 0).  Double-float moments
// of the normalised points and the normal matrix from them, the refined
// eigenvector; writes sh.hn and, when the gauge h33 = 1 is usable, the LM
// parameters sh.pd / sh.par.  Returns 0 (the factorisation failed), 1 (no
// gauge) or 2.
__device__ __forceinline__ int dlt_result(Shared &sh, float s1, float s2)
{
    const int lane = threadIdx.x & 31;
    constexpr int dm[6] = {2, 2, 2, 1, 1, 0}, dw[4] = {0, 1, 1, 2};
    if (lane < kDF_DLT) {
        const int am = dm[lane % 6], aw = dw[lane / 6];
        const float fa = am == 0 ? 1.0f : (am == 1 ? s1 : s1 * s1), fb = aw == 0 ? 1.0f : (aw == 1 ? s2 : s2 * s2);
        sh.mdf[lane] = df_mul(sh.sum[lane], fa * fb);
    }
    __syncwarp();
    for (int e = lane; e < 45; e += 32) {
        int r = 0;
        while (tri(r + 1, 0) <= e) ++r;
        const int k = dlt_code(r, e - tri(r, 0));
        sh.Mdf[e] = k == 0 ? DF{0.0f, 0.0f} : (k > 0 ? sh.mdf[k - 1] : df_neg(sh.mdf[-k - 1]));
    }
    __syncwarp();
    float mo[kDF_DLT];
#pragma unroll
    for (int k = 0; k < kDF_DLT; ++k) mo[k] = df_round(sh.mdf[k]);
    DF v[9];
    const bool fact = dlt_refined(sh.Mdf, mo, sh.tr[0], v);
    float n2 = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) n2 = fmaf(v[i].h, v[i].h, n2);
    // LM gauge h33 = 1 needs the normalised h33 away from zero
    const bool gauge = fact && fabsf(v[8].h) >= 1e-3f * sqrtf(n2);
    if (lane < 9) sh.hn[lane] = fact ? lane_pick_df(v, lane) : DF{0.0f, 0.0f};
    if (gauge && lane < 8) {
        const DF pk = df_div2(lane_pick_df(v, lane), v[8]);
        sh.pd[lane] = pk;
        sh.par[lane] = pk.h;
    }
    __syncwarp();
    return gauge ? 2 : (fact ? 1 : 0);
}


// Leader warp, after the first pass: the LM state at the start (gradient,
// J^T J sums, cost, damping mu0 = tau * max diag(J^T J)); false if the cost
// or the damping is not finite and positive.
__device__ __forceinline__ bool lm_start(Shared &sh)
{
    const int lane = threadIdx.x & 31;
    if (lane < kF_LM) sh.Asum[lane] = sh.sumf[lane];
    if (lane < 8) sh.g[lane] = df_round(sh.sum[lane]);
    // largest diagonal entry of J^T J: sums q xx, q yy, q and q (u^2 + v^2) {xx, yy}
    const float *f = sh.sumf;
    const float dmax = fmaxf(fmaxf(fmaxf(f[0], f[2]), fmaxf(f[5], f[16])), fmaxf(f[18], 0.0f));
    const DF s8 = sh.sum[8];
    const DF F{0.5f * s8.h, 0.5f * s8.l};
    const float mu = kTau * dmax;
    if (lane == 0) {
        sh.F = F;
        sh.mu = mu;
        sh.mu_poor = kTauPoor * dmax;
        sh.nu = 2.0f;
        sh.it = 0;
        sh.quiet = 0;
    }
    __syncwarp();
    return isfinite(F.h) && isfinite(mu) && mu > 0.0f;
}

// Leader warp: the next trial step (J^T J + mu I) d = -g, counting every
// trial (a non-positive-definite matrix is a rejected step).  Returns 1
// (evaluate pd + d, in sh.par) or 0 (no more trials: the budget is spent, the
// step is below the FP32 resolution of the parameters, the last kQuietSteps
// accepted steps were quiet (each below 2^-20 of the parameters and
// predicting a decrease below the cost's FP32 noise), or the damping is no
// longer finite).  Every lane factors and solves in registers.
__device__ __forceinline__ int lm_trial(Shared &sh, int budget)
{
    const int lane = threadIdx.x & 31;
    float m[kF_LM], g[8], p[8];
#pragma unroll
    for (int k = 0; k < kF_LM; ++k) m[k] = sh.Asum[k];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        g[k] = sh.g[k];
        p[k] = sh.pd[k].h;
    }
    float mu = sh.mu, nu = sh.nu;
    int it = sh.it, go = 0;
    float d[8];
    for (;;) {
        if (it >= budget || sh.quiet >= kQuietSteps || !(isfinite(mu) && mu > 0.0f)) break;
        float a[36], rd[8];
        fill_packed<8>(m, a);
#pragma unroll
        for (int k = 0; k < 8; ++k) a[tri(k, k)] += mu;
        const bool ok = reg_cholesky<8>(a, rd, 0.0f);
        ++it;
        if (!ok) {
            if (it == 1) {
                mu = sh.mu_poor;
            } else {
                mu *= nu;
                nu *= 2.0f;
            }
            continue;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) d[k] = -g[k];
        reg_chol_solve<8>(a, rd, d);
        float nd = 0.0f, np = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            nd = fmaf(d[k], d[k], nd);
            np = fmaf(p[k], p[k], np);
        }
        go = sqrtf(nd) > kEpsStep * (sqrtf(np) + kEpsStep) ? 1 : 0;
        if (lane == 0) sh.small = sqrtf(nd) <= kQuietStep * (sqrtf(np) + kQuietStep);
        break;
    }
    if (go && lane < 8) {
        const float dl = lane_pick<8>(d, lane);
        sh.d[lane] = dl;
        sh.par[lane] = df_round(df_add(sh.pd[lane], DF{dl, 0.0f}));
    }
    if (lane == 0) {
        sh.mu = mu;
        sh.nu = nu;
        sh.it = it;
    }
    __syncwarp();
    return go;
}

// Leader warp: gain ratio of the evaluated step; accept or reject it.
__device__ __forceinline__ void lm_update(Shared &sh)
{
    const int lane = threadIdx.x & 31;
    const DF F = sh.F, sn = sh.sum[8];
    const DF Fn{0.5f * sn.h, 0.5f * sn.l};
    const float mu = sh.mu, nu = sh.nu;
    float pred = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float dk = sh.d[k];
        pred = fmaf(dk, fmaf(mu, dk, -sh.g[k]), pred);
    }
    pred *= 0.5f;
    const float dF = df_round(df_sub(F, Fn));            // the decrease, from the double-float costs
    const float rho = dF / pred;
    const float noise = kCostNoise * F.h;
    const bool accept = isfinite(Fn.h) && (rho > 0.0f || (pred <= noise && -dF <= noise));
    __syncwarp();
    if (accept) {
        if (lane < 8) {
            sh.pd[lane] = df_renorm(df_add(sh.pd[lane], DF{sh.d[lane], 0.0f}));
            sh.g[lane] = df_round(sh.sum[lane]);
        }
        if (lane < kF_LM) sh.Asum[lane] = sh.sumf[lane];
        if (lane == 0) {
            sh.F = Fn;
            sh.quiet = pred <= noise && sh.small ? sh.quiet + 1 : 0;
            const float t = rho > 0.0f && rho < 1.0f ? 2.0f * rho - 1.0f : 1.0f;
            sh.mu = mu * fmaxf(1.0f / 3.0f, 1.0f - t * t * t);
            sh.nu = 2.0f;
        }
    } else if (lane == 0) {
        if (sh.it == 1) {                           // the first trial: a poorer start
            sh.mu = sh.mu_poor;
        } else {
            sh.mu = mu * nu;
            sh.nu = nu * 2.0f;
        }
    }
    __syncwarp();
}

// (x.h + x.l) / b: the quotient's leading part, then the remainder's
// (TwoProduct makes x - q b exact up to x.l's rounding).
__device__ __forceinline__ DF df_div(DF x, float b)
{
    const float q = x.h / b;
    const DF r = df_sub(x, df_prod(q, b));
    return DF{q, df_round(r) / b};
}

// Leader warp, every lane: H = T2^-1 Hn T1 in pixels, in double-float (the
// translation columns cancel), with unit Frobenius norm and the sign that
// makes h33 > 0 (or, when |h33| < 1e-6 |H|, the first entry of largest
// magnitude > 0); lane i writes entry i.
__device__ __forceinline__ void leader_store(const Shared &sh, const DF (&hn)[9], float *out)
{
    const int lane = threadIdx.x & 31;
    const float s1 = sh.s1, s2 = sh.s2, a1x = sh.mu1x, a1y = sh.mu1y, a2x = sh.mu2x, a2y = sh.mu2y;
    // B = Hn T1: columns 0, 1 scale by s1, column 2 picks up -s1 (h_r0 mu1x + h_r1 mu1y)
    DF B[9];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        B[3 * r] = df_mul(hn[3 * r], s1);
        B[3 * r + 1] = df_mul(hn[3 * r + 1], s1);
        B[3 * r + 2] = df_sub(hn[3 * r + 2], df_mul(df_add(df_mul(hn[3 * r], a1x), df_mul(hn[3 * r + 1], a1y)), s1));
    }
    // H = T2^-1 B: rows 0, 1 are B_r / s2 + mu2 B_2, row 2 is B_2
    float h[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        h[c] = df_round(df_add(df_div(B[c], s2), df_mul(B[6 + c], a2x)));
        h[3 + c] = df_round(df_add(df_div(B[3 + c], s2), df_mul(B[6 + c], a2y)));
        h[6 + c] = df_round(B[6 + c]);
    }
    float n2 = 0.0f, ab = -1.0f, hb = 0.0f;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        n2 = fmaf(h[k], h[k], n2);
        if (fabsf(h[k]) > ab) {
            ab = fabsf(h[k]);
            hb = h[k];
        }
    }
    const float nrm = sqrtf(n2);
    if (lane < 9) {
        if (!(nrm > 0.0f) || !isfinite(nrm)) {
            out[lane] = 0.0f;
        } else {
            const float sgn = fabsf(h[8]) >= 1e-6f * nrm ? (h[8] > 0.0f ? 1.0f : -1.0f) : (hb > 0.0f ? 1.0f : -1.0f);
            out[lane] = sgn * lane_pick<9>(h, lane) / nrm;
        }
    }
}

// Longest first: block b takes the problem of rank b in the order of
// decreasing size class (size = correspondences, class = octave and quarter
// octave: 4 log2(N) rounded down), then increasing index.  The largest
// problems set the kernel's length; started in the first wave they finish
// while the small ones fill the SMs.  Every block ranks all P problems
// (two passes over the offsets), so above kOrderMaxP problems the natural
// order is used.
constexpr int kClasses = 128;
constexpr int32_t kOrderMaxP = 1 << 16;

__device__ __forceinline__ int size_class(int64_t N)
{
    if (N <= 0) return 0;
    const uint64_t u = (uint64_t)N;
    const int e = 63 - __clzll((long long)u);                 // floor(log2 N)
    const int f = e >= 2 ? (int)((u >> (e - 2)) & 3u) : (int)((u << (2 - e)) & 3u);
    const int c = 4 * e + f;
    return c < kClasses ? c : kClasses - 1;
}

__device__ __forceinline__ int32_t longest_first(const int64_t *__restrict__ offsets, int32_t P, int32_t b, int32_t *hist,
                                 int32_t *scratch)
{
    for (int k = threadIdx.x; k < kClasses; k += kThreads) hist[k] = 0;
    __syncthreads();
    for (int32_t q = threadIdx.x; q < P; q += kThreads) atomicAdd(&hist[size_class(offsets[q + 1] - offsets[q])], 1);
    __syncthreads();
    if (threadIdx.x < 32) {
        // class of rank b, classes in decreasing order: lane l holds classes
        // 127 - 4l .. 124 - 4l; a warp scan gives the count above each
        const int lane = threadIdx.x;
        int32_t c[4], tot = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = hist[kClasses - 1 - 4 * lane - u];
            tot += c[u];
        }
        int32_t incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int32_t above = incl - tot;                             // counts of the classes before this lane's
        const unsigned hit = __ballot_sync(0xffffffffu, above <= b && b < incl);
        if (lane == __ffs(hit) - 1) {
            int u = 0;
            while (u < 3 && above + c[u] <= b) above += c[u++];
            scratch[0] = kClasses - 1 - 4 * lane - u;
            scratch[1] = b - above;                             // rank within the class
            scratch[2] = -1;
        }
    }
    __syncthreads();
    const int kb = scratch[0];
    const int32_t j = scratch[1];
    int32_t before = 0;                                         // class members of lower index so far
    for (int32_t base = 0; base < P && scratch[2] < 0; base += kThreads) {
        const int32_t q = base + (int32_t)threadIdx.x;
        const bool mine = q < P && size_class(offsets[q + 1] - offsets[q]) == kb;
        const unsigned bal = __ballot_sync(0xffffffffu, mine);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) scratch[4 + warp] = __popc(bal);
        __syncthreads();
        int32_t wbefore = before;
        for (int w = 0; w < warp; ++w) wbefore += scratch[4 + w];
        if (mine && wbefore + __popc(bal & ((1u << lane) - 1u)) == j) scratch[2] = q;
        for (int w = 0; w < kWarps; ++w) before += scratch[4 + w];
        __syncthreads();
    }
    return scratch[2];
}

__device__ void write_empty(float *H_out, float *rms, int p, float rms_value)
{
    if (threadIdx.x < 9) H_out[9 * (int64_t)p + threadIdx.x] = 0.0f;
    if (threadIdx.x == 0 && rms) rms[p] = rms_value;
}

__global__ void __launch_bounds__(kThreads, 2)
refit_kernel(const float4 *__restrict__ corr, const int64_t *__restrict__ offsets,
             const uint8_t *__restrict__ mask, int lm_iters, float *__restrict__ H_out,
             int32_t *__restrict__ n_used, float *__restrict__ rms, int cap)
{
    __shared__ Shared sh;
    __shared__ int32_t s_hist[kClasses], s_scr[4 + kWarps];
    grid_launch_dependents();
    grid_dependency_wait();                 // may follow a RANSAC finish kernel that writes the mask
    const int32_t P = gridDim.x;
    const int p = P <= kOrderMaxP ? longest_first(offsets, P, blockIdx.x, s_hist, s_scr) : (int)blockIdx.x;
    const int lane = threadIdx.x & 31;
    const bool leader = threadIdx.x < 32;          // warp 0 runs the small solves
    const int64_t o0 = offsets[p];
    int64_t n = offsets[p + 1] - o0;
    if (n < 0) n = 0;
    const Points pts{corr + o0, mask ? mask + o0 : nullptr, n, (int)(n < cap ? n : cap), cap};

    // Pass 1: count and centroids.
    {
        DFAcc<5> a;
        a.zero();
        for_points_fill(pts, [&](float4 q, bool t) {
            a.f[0] += t ? 1.0f : 0.0f; a.f[1] += q.x; a.f[2] += q.y; a.f[3] += q.z; a.f[4] += q.w;
        }, [&](int slots) { a.tick(slots); });
        a.flush();
        warp_partials<5, 0>(a.s, nullptr, sh);
        __syncthreads();
        if (leader) {
            leader_sums<5, 0>(sh);
            if (lane == 0) {
                const DF c0 = sh.sum[0];                    // an exact integer
                const int64_t used = (int64_t)c0.h + (int64_t)c0.l;
                const float cnt = (float)used;
                sh.used = used;
                sh.cnt = cnt;
                sh.mu1x = df_round(sh.sum[1]) / cnt; sh.mu1y = df_round(sh.sum[2]) / cnt;
                sh.mu2x = df_round(sh.sum[3]) / cnt; sh.mu2y = df_round(sh.sum[4]) / cnt;
            }
        }
        __syncthreads();
    }
    const int64_t used = sh.used;
    if (threadIdx.x == 0 && n_used) n_used[p] = (int32_t)used;
    if (used < 4) {
        write_empty(H_out, rms, p, 0.0f);
        return;
    }

    // Pass 2: mean distances to the centroids (-> the scales s1, s2) and the
    // moments of the centred points, S_w = sum w {xx, xy, yy, x, y, 1} for
    // w = 1, X, Y, X^2 + Y^2; those of the normalised points follow by
    // scaling each by s1^(degree in x, y) s2^(degree in X, Y).
    {
        DFAcc<kDF_P2> a;
        a.zero();
        const float m1x = sh.mu1x, m1y = sh.mu1y, m2x = sh.mu2x, m2y = sh.mu2y;
        for_points<2, kUnroll>(pts, [&](float4 q, bool t) {
            // an unused slot: zero centred coordinates and weight
            const float x = t ? q.x - m1x : 0.0f, y = t ? q.y - m1y : 0.0f;
            const float X = t ? q.z - m2x : 0.0f, Y = t ? q.w - m2y : 0.0f;
            // distances by the hardware reciprocal square root (a few ulp: they
            // only set the normalising scales); zero for an unused slot (the
            // argument floored at the smallest normal), without the
            // special-case path of a correctly rounded sqrt(0)
            const float r1 = fmaf(x, x, y * y), R = fmaf(X, X, Y * Y);
            a.f[kDF_DLT] += r1 * rsqrtf(fmaxf(r1, 1.17549435e-38f));
            a.f[kDF_DLT + 1] += R * rsqrtf(fmaxf(R, 1.17549435e-38f));
            const float mo[6] = {x * x, x * y, y * y, x, y, t ? 1.0f : 0.0f};
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                a.f[k] += mo[k];
                a.f[6 + k] = fmaf(X, mo[k], a.f[6 + k]);
                a.f[12 + k] = fmaf(Y, mo[k], a.f[12 + k]);
                a.f[18 + k] = fmaf(R, mo[k], a.f[18 + k]);
            }
        }, [&](int slots) { a.tick(slots); });
        a.flush();
        warp_partials_part<0, kDF_P2 / 2>(a.s, sh);
        warp_partials_part<kDF_P2 / 2, kDF_P2 - kDF_P2 / 2>(a.s, sh);
        __syncthreads();
    }

    // DLT, then the LM set-up and first trial, by the leader warp.  FP64 runs
    // at 1/64 of the FP32 rate on this part, and each FP64 instruction of a
    // serial chain costs hundreds of cycles, so none is used: FP32 and
    // double-float only.
    if (leader) {
        leader_sums<kDF_P2, 0>(sh);
        const float cnt = sh.cnt;
        const float d1 = df_round(sh.sum[kDF_DLT]), d2 = df_round(sh.sum[kDF_DLT + 1]);
        const float s1 = d1 > 0.0f ? 1.41421356f * cnt / d1 : 1.0f;
        const float s2 = d2 > 0.0f ? 1.41421356f * cnt / d2 : 1.0f;
        if (lane == 0) {
            sh.s1 = s1;
            sh.s2 = s2;
        }
        // the factor s1^(degree in x, y) s2^(degree in X, Y) of moment k
        const float f1[3] = {1.0f, s1, s1 * s1}, f2[3] = {1.0f, s2, s2 * s2};
        constexpr int dm[6] = {2, 2, 2, 1, 1, 0}, dw[4] = {0, 1, 1, 2};
        bool fact, gauge;                           // factorisation done; LM gauge h33 = 1 usable
        if (lm_iters == 0) {
            const int r = dlt_result(sh, s1, s2);
            fact = r != 0;
            gauge = r == 2;
        } else {
            // FP32 in registers: it only starts LM
            float mo[kDF_DLT];
#pragma unroll
            for (int k = 0; k < kDF_DLT; ++k) mo[k] = df_round(sh.sum[k]) * (f1[dm[k % 6]] * f2[dw[k / 6]]);
            float x[9];
            fact = dlt_start(mo, x);
            gauge = fact && fabsf(x[8]) >= 1e-3f;
            if (lane < 9) sh.hn[lane] = DF{fact ? lane_pick<9>(x, lane) : 0.0f, 0.0f};
            if (gauge && lane < 8) {
                const float pk = lane_pick<9>(x, lane) / x[8];
                sh.pd[lane] = DF{pk, 0.0f};
                sh.par[lane] = pk;
            }
        }
        if (lane == 0) sh.go = gauge ? 1 : (fact ? 0 : -1);
    }
    __syncthreads();
    if (sh.go < 0) {                                // factorisation failed: no fit
        write_empty(H_out, rms, p, -1.0f);
        return;
    }

    // Levenberg-Marquardt: a pass at the start (it also gives the residual of
    // the DLT when lm_iters = 0), then one pass per evaluated trial step.
    bool lm_ok = false;
    if (sh.go) {
        bool first = true;
        do {
            lm_pass(pts, sh);
            if (leader) {
                leader_sums<kDF_LM, kF_LM>(sh);
                bool ok = true;
                if (first) ok = lm_start(sh);
                else lm_update(sh);
                const int go = ok ? 1 + lm_trial(sh, lm_iters) : 0;
                if (lane == 0) sh.go = go;        // 0: no LM; 1: LM, no more steps; 2: evaluate
            }
            __syncthreads();
            if (first) lm_ok = sh.go != 0;
            first = false;
            // sh.go is rewritten by the leader only after the barrier in lm_pass
        } while (sh.go == 2);
    }

    // Back to pixels.
    if (leader) {
        DF hn[9];
        if (lm_ok) {
#pragma unroll
            for (int k = 0; k < 8; ++k) hn[k] = sh.pd[k];
            hn[8] = DF{1.0f, 0.0f};
        } else {
#pragma unroll
            for (int k = 0; k < 9; ++k) hn[k] = sh.hn[k];
        }
        leader_store(sh, hn, H_out + 9 * (int64_t)p);
        if (lane == 0 && rms) rms[p] = lm_ok ? sqrtf(2.0f * sh.F.h / sh.cnt) / sh.s2 : -1.0f;
    }
}

// The points a block keeps in shared memory: what is left of half an SM's
// shared memory (two blocks per SM) after the block's static part, in whole
// block strides, at 17 bytes a point (the float4 and its mask byte); fewer if
// two blocks would not fit.  Sets the kernel's dynamic shared memory limit;
// cached per device.
struct RefitLaunch {
    int cap;
    size_t smem;
};

RefitLaunch refit_launch()
{
    static std::mutex mu;
    static std::map<int, RefitLaunch> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(mu);
        const auto it = cache.find(dev);
        if (it != cache.end()) return it->second;
    }
    int per_sm = 0, reserved = 0, optin = 0;
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, refit_kernel);
    long avail = (long)per_sm / 2 - reserved - (long)fa.sharedSizeBytes;
    if (avail > (long)optin - (long)fa.sharedSizeBytes) avail = (long)optin - (long)fa.sharedSizeBytes;
    constexpr int kBytesPerPoint = (int)sizeof(float4) + 1;
    int cap = avail > 0 ? (int)(avail / kBytesPerPoint) / kThreads * kThreads : 0;
    for (; cap > 0; cap -= kThreads) {
        const size_t smem = (size_t)cap * kBytesPerPoint;
        if (cudaFuncSetAttribute(refit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
            blocks_per_sm(reinterpret_cast<const void *>(refit_kernel), kThreads, smem) >= 2)
            break;
    }
    cudaGetLastError();                     // a refused size above is not an error of this call
    const RefitLaunch r{cap, (size_t)cap * kBytesPerPoint};
    std::lock_guard<std::mutex> lock(mu);
    cache[dev] = r;
    return r;
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
    const RefitLaunch L = refit_launch();
    launch_after_previous(refit_kernel, dim3(P), dim3(kThreads), L.smem, as_stream(stream),
                          reinterpret_cast<const float4 *>(corr), offsets, mask, lm_iters, H, n_used, rms, L.cap);
    return check_launch("aca_refit");
}
