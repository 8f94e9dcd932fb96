// RANSAC with ACA hypotheses, many problems of uneven size per launch
// (Sec. 2.2: sample a minimal set, solve, verify against all
// correspondences, keep the best; Sec. 6.2 runs this with the solvers of
// the paper plugged in).
//
// Kernels (all on the caller's stream, no host synchronisation):
//  1. ransac_prep_kernel    one block: per-problem prefix sums of hypotheses
//                           and work items (with 64 or more problems, items
//                           laid out largest problem first), resets the work
//                           counter;
//  2. zero_counts_kernel    clears the per-hypothesis counts;
//  3. ransac_score_kernel   persistent grid; each block repeatedly takes an
//                           item (problem p, hypotheses h0..h0+HB-1, points
//                           i0..i0+T-1) from one atomic counter, samples and
//                           solves its HB hypotheses (Philox + ACA) into shared
//                           memory while the whole block stages the point
//                           slice in shared memory, then scores: lane l of
//                           every warp holds hypotheses l, l+32, ... in
//                           registers, each warp walks its share of the slice
//                           (every lane reads the same point: a shared-memory
//                           broadcast) and counts inliers with a division-free
//                           test; warp partials are summed in shared memory and
//                           added to the global count with one atomic per
//                           hypothesis;
//  4. ransac_finish_kernel  one block per problem: argmax (ties to the lowest
//                           index), re-solve of the winner with the same
//                           device code (bit-identical H), inlier mask, outputs.
// There are no inter-block waits: progress only needs the atomics.  Kernels
// 2-4 are launched as programmatic dependents of their predecessor (they are
// scheduled while it runs and wait for it with griddepcontrol.wait before
// touching its data), which hides the launch gaps of short problems.
//
// With the online adaptive stop (ransac_aca_adaptive, Sec. 6.2: the loop
// count follows from the best inlier ratio so far), the same scoring loop
// runs with three changes:
//  - items are ordered in rounds, round r holding chunk r (hypotheses
//    r*HB .. r*HB+HB-1) of every problem that has one, so that a problem's
//    earlier chunks are finished while its later ones wait in the queue;
//  - the block that finishes the last slice of a chunk takes the chunk's best
//    count c at index j and lowers the problem's bound to max(j + 1, K(c)),
//    K being the required number of hypotheses; a chunk starting at or after
//    the bound is skipped: the sequential loop is certain to stop before it
//    (the best over hypotheses 0..h0-1 is at least c, so K at h0 is at most
//    K(c) <= h0).  A dead chunk stays dead, so the block that draws one checks
//    the next 31 problems of the round as well and moves the work counter
//    past the whole run of dead ones in a single atomicMax;
//  - the scoring runs in two epochs: chunk 0 of every problem, then a
//    one-block re-plan that keeps, per problem, only the chunks before its
//    current bound (a bound only decreases, so a stale one keeps a superset
//    of the live chunks), then the scoring of those;
//  - the finish kernel finds the sequential stop index from the prefix
//    maxima of the counts (the stop condition i >= K(best of 0..i-1) is
//    monotone in i) and takes the argmax before it.
// Every output is deterministic: counts before the stop are complete sums,
// everything after it is reported as not evaluated.
#include "aca_math.cuh"
#include "common.cuh"
#include "pdl.cuh"
#include "philox.cuh"

namespace aca {

// Done counters.  One thread of a block adds to the counter after a
// __syncthreads, with acquire-release semantics at GPU scope: the release
// half publishes the block's stores (ordered before the add by the barrier),
// the acquire half makes the stores that the other blocks published before
// their adds visible to the block after the next __syncthreads.  The same
// pattern as a grid-wide barrier, with the fences folded into the add.
__device__ __forceinline__ uint32_t atomic_add_acq_rel(uint32_t *p, uint32_t v)
{
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Degenerate-sample rule: on either side one of the triples (M,N,P),
// (M,Q,P), (M,N,Q), (N,P,Q) has |cross(a,b)| <= 1e-3 |a||b| for its edge
// vectors a, b (sine of the angle at most 1e-3).
__device__ __forceinline__ bool triple_degenerate(float cr, float ax, float ay, float bx, float by)
{
    const float tau2 = 1e-6f;
    const float la = sq2(ax, ay), lb = sq2(bx, by);
    return F_MUL(cr, cr) <= F_MUL(F_MUL(tau2, la), lb);
}

__device__ __forceinline__ bool sample_degenerate(const AcaParts &p)
{
    return triple_degenerate(p.fA1, p.MN1x, p.MN1y, p.MP1x, p.MP1y) ||
           triple_degenerate(p.Q3x, p.MQ1x, p.MQ1y, p.MP1x, p.MP1y) ||
           triple_degenerate(p.Q3y, p.MN1x, p.MN1y, p.MQ1x, p.MQ1y) ||
           triple_degenerate(p.t1, p.NP1x, p.NP1y, p.NQ1x, p.NQ1y) ||
           triple_degenerate(p.fA2, p.MN2x, p.MN2y, p.MP2x, p.MP2y) ||
           triple_degenerate(p.Q4x, p.MQ2x, p.MQ2y, p.MP2x, p.MP2y) ||
           triple_degenerate(p.Q4y, p.MN2x, p.MN2y, p.MQ2x, p.MQ2y) ||
           triple_degenerate(p.t2, p.NP2x, p.NP2y, p.NQ2x, p.NQ2y);
}

// Hypothesis h of a problem whose N >= 4 correspondences start at `c`:
// sample, reject degenerate samples (a non-finite coordinate, or a triple
// near collinear), solve by ACA and scale H by a power of
// two so that its largest entry lies in [1, 2) (exact; keeps the squared
// residuals of the test far from overflow).  Returns false if degenerate.
__device__ __forceinline__ bool make_hypothesis(const float4 *__restrict__ c, uint32_t N, uint64_t seed,
                                                uint32_t prob, uint32_t h, float H[9])
{
    uint32_t idx[4];
    sample4(seed, prob, h, N, idx);
    const float4 m = c[idx[0]], n = c[idx[1]], p4 = c[idx[2]], q = c[idx[3]];
    const Set s{m.x, m.y, n.x, n.y, p4.x, p4.y, q.x, q.y, m.z, m.w, n.z, n.w, p4.z, p4.w, q.z, q.w};
    // a sample with a non-finite coordinate is degenerate: x * 0 is 0 for
    // every finite x and NaN otherwise
    const float *sv = &s.M1x;
    float z = 0.0f;
#pragma unroll
    for (int k = 0; k < 16; ++k) z = F_FMA(sv[k], 0.0f, z);
    if (!(z == 0.0f))
        return false;
    AcaParts p;
    aca_parts(s, p);
    if (sample_degenerate(p))
        return false;
    aca_compose(s, p, true, H);
    const float sc = pow2_inv_scale(max_abs9(H));
#pragma unroll
    for (int i = 0; i < 9; ++i)
        H[i] = F_MUL(H[i], sc);
    return true;
}

// Forward transfer error test without division: with (u, v, w) = H (x, y, 1),
// e = (X w - u)^2 + (Y w - v)^2 - thr^2 w^2 and the point is an inlier when
// e < 0, i.e. ||(X, Y) - (u/w, v/w)|| < thr (e < 0 forces w != 0).  The FP32
// evaluation is strict; a point with e == 0 exactly lies within rounding of
// the threshold.  The threshold is folded into the data so that the FMA pipe,
// which bounds the scoring loop, does 11 operations per pair of tests
// instead of 12: the hypothesis is kept as G = (-h11, -h12, -h13, -h21, -h22,
// -h23, t h31, t h32, t h33) with t = thr (so w' = t w), and the target point
// as (Xs, Ys) = (X, Y) RN(1/t), so that Xs w' = X w up to two roundings
// (about 1e-7 relative, far inside the parity band):
//   w' = g6 x + g7 y + g8, -u = g0 x + g1 y + g2, -v = g3 x + g4 y + g5,
//   du = Xs w' - u, dv = Ys w' - v, e = du^2 + (dv^2 + w' (-w')),
// the sign flip of w' being an integer operation.  e is never -0 (each step
// adds a non-negative square to a sum that is not -0), so its sign bit is
// exactly (e < 0) and counting is a shift and an add.  The same operations,
// in the same order, run lane-wise on f32x2 pairs in the scoring loop
// (inlier2) and on scalars in the epilogue (inlier): packed FP32
// instructions round each lane exactly like the scalar ones, so counts and
// masks agree bit for bit.
__device__ __forceinline__ void to_test_form(float G[9], const float H[9], float thr)
{
#pragma unroll
    for (int i = 0; i < 6; ++i) G[i] = -H[i];
    G[6] = F_MUL(thr, H[6]);
    G[7] = F_MUL(thr, H[7]);
    G[8] = F_MUL(thr, H[8]);
}

// RN(1/thr), the factor of the stored target coordinates.
__device__ __forceinline__ float target_scale(float thr) { return F_DIV(1.0f, thr); }

__device__ __forceinline__ int inlier(const float G[9], float4 c, float rthr)
{
    const float w = F_FMA(G[6], c.x, F_FMA(G[7], c.y, G[8]));
    const float nu = F_FMA(G[0], c.x, F_FMA(G[1], c.y, G[2]));
    const float nv = F_FMA(G[3], c.x, F_FMA(G[4], c.y, G[5]));
    const float du = F_FMA(F_MUL(c.z, rthr), w, nu);
    const float dv = F_FMA(F_MUL(c.w, rthr), w, nv);
    const float e = F_FMA(du, du, F_FMA(dv, dv, F_MUL(w, -w)));
    return (int)(__float_as_uint(e) >> 31);
}

// Packed FP32 pair operations (sm_100+ f32x2 instructions; one instruction
// per pair, each lane rounded to nearest like the scalar operation).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// Sign flip of both lanes (an integer operation, off the FMA pipe).
__device__ __forceinline__ float2 neg2(float2 a)
{
    return make_float2(__uint_as_float(__float_as_uint(a.x) ^ 0x80000000u),
                       __uint_as_float(__float_as_uint(a.y) ^ 0x80000000u));
}

// Two points (lane a, lane b) against one hypothesis given as broadcast pairs
// g[i] = (G[i], G[i]); p = (x_a, x_b, y_a, y_b), q = (Xs_a, Xs_b, Ys_a, Ys_b)
// with the scaled target coordinates of the test form above.
__device__ __forceinline__ int inlier2(const float2 g[9], float4 p, float4 q)
{
    const float2 x = make_float2(p.x, p.y), y = make_float2(p.z, p.w);
    const float2 X = make_float2(q.x, q.y), Y = make_float2(q.z, q.w);
    const float2 w = fma2(g[6], x, fma2(g[7], y, g[8]));
    const float2 nu = fma2(g[0], x, fma2(g[1], y, g[2]));
    const float2 nv = fma2(g[3], x, fma2(g[4], y, g[5]));
    const float2 du = fma2(X, w, nu);
    const float2 dv = fma2(Y, w, nv);
    const float2 e = fma2(du, du, fma2(dv, dv, mul2(w, neg2(w))));
    return (int)((__float_as_uint(e.x) >> 31) + (__float_as_uint(e.y) >> 31));
}

struct Workspace {
    int64_t *hyp_off;            // [P+1] prefix of the hypothesis counts, problem order
    int64_t *item_off;           // [P+1] prefix of the work items over `order` (fixed counts)
    unsigned long long *counter; // [1] work counter
    int32_t *flags;              // [1] 1 = counts capacity exceeded
    unsigned *done;              // [1] blocks finished (one-launch path); zero between calls
    unsigned long long *best;    // [kFusedMaxP] packed best (count, ~index) per problem (one-launch
                                 // path, whole-range items); zero between calls
    int32_t *order;              // [P] scoring order of the problems (fixed counts): largest N first
    int32_t *counts;             // [capacity]
    int64_t capacity;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Every layout starts with the same 256-byte control block (work counter,
// overflow flag, the one-launch path's done counter and per-problem best),
// so that a workspace shared by calls of different sizes and kinds keeps the
// one-launch path's state in one place, written by nothing but that path,
// which leaves it zero.
static void carve_control(char *b, Workspace &w)
{
    w.counter = reinterpret_cast<unsigned long long *>(b);
    w.flags = reinterpret_cast<int32_t *>(b + 8);
    w.done = reinterpret_cast<unsigned *>(b + 16);
    w.best = reinterpret_cast<unsigned long long *>(b + 32);
}

static Workspace carve(void *base, int32_t P, size_t bytes)
{
    Workspace w;
    char *b = static_cast<char *>(base);
    carve_control(b, w);
    size_t o = 256;
    w.hyp_off = reinterpret_cast<int64_t *>(b + o);
    o += align256(sizeof(int64_t) * (size_t)(P + 1));
    w.item_off = reinterpret_cast<int64_t *>(b + o);
    o += align256(sizeof(int64_t) * (size_t)(P + 1));
    w.order = reinterpret_cast<int32_t *>(b + o);
    o += align256(sizeof(int32_t) * (size_t)P);
    w.counts = reinterpret_cast<int32_t *>(b + o);
    w.capacity = bytes > o ? (int64_t)((bytes - o) / sizeof(int32_t)) : 0;
    return w;
}

static size_t header_bytes(int32_t P)
{
    return 2 * align256(sizeof(int64_t) * (size_t)(P + 1)) + 256 + align256(sizeof(int32_t) * (size_t)P);
}

// Extra workspace of the adaptive variant (after the standard header).
struct AdaptiveWs {
    int64_t *chunk_off;    // [P+1] prefix of C_p, the chunks of HB hypotheses of problem p
    int32_t *order;        // [P] problems by C_p, largest first
    int64_t *spref;        // [P+1] prefix of the slice counts S_p over `order`
    int64_t *round_off;    // [rb+1] first item of round r
    int32_t *round_cnt;    // [rb+1] problems in round r (those with C_p > r)
    int32_t *cursor;       // [rb+1] counting-sort cursors
    int32_t *rounds;       // [1] rounds of the current epoch
    int32_t *chunk_lo;     // [1] chunk index of round 0 of the current epoch
    int32_t *kbound;       // [P] the stop is certain before this hypothesis index
    int32_t *chunk_done;   // [cb] completed slices per chunk
    int32_t *prefix;       // [capacity] inclusive prefix maxima of the counts (finish)
    int64_t rb, cb;        // capacities (bounds for HB = 32)
    double log_fail;       // log(1 - confidence)
};

// Layout: standard header, adaptive arrays, counts (total_hyps), prefix.
static size_t adaptive_bytes(int32_t P, int64_t total, int64_t *rb, int64_t *cb, size_t *counts_at)
{
    const int64_t r = total / 32 + 2, c = total / 32 + (int64_t)P + 1;
    size_t o = header_bytes(P);
    o += align256(sizeof(int64_t) * (size_t)(P + 1));    // chunk_off
    o += align256(sizeof(int32_t) * (size_t)P);          // order
    o += align256(sizeof(int64_t) * (size_t)(P + 1));    // spref
    o += align256(sizeof(int64_t) * (size_t)(r + 1));    // round_off
    o += 2 * align256(sizeof(int32_t) * (size_t)(r + 1));// round_cnt, cursor
    o += 256;                                            // rounds
    o += align256(sizeof(int32_t) * (size_t)P);          // kbound
    o += align256(sizeof(int32_t) * (size_t)c);          // chunk_done
    if (counts_at) *counts_at = o;
    o += 2 * align256(sizeof(int32_t) * (size_t)total);  // counts, prefix
    if (rb) *rb = r;
    if (cb) *cb = c;
    return o;
}

static void carve_adaptive(void *base, int32_t P, int64_t total, Workspace &w, AdaptiveWs &a)
{
    char *b = static_cast<char *>(base);
    size_t counts_at = 0;
    adaptive_bytes(P, total, &a.rb, &a.cb, &counts_at);
    carve_control(b, w);                                   // done: unused by the adaptive variant
    size_t o = 256;
    w.hyp_off = reinterpret_cast<int64_t *>(b + o);
    o += align256(sizeof(int64_t) * (size_t)(P + 1));
    w.item_off = reinterpret_cast<int64_t *>(b + o);
    o += align256(sizeof(int64_t) * (size_t)(P + 1));
    w.order = reinterpret_cast<int32_t *>(b + o);          // unused by the adaptive variant
    o += align256(sizeof(int32_t) * (size_t)P);
    a.chunk_off = reinterpret_cast<int64_t *>(b + o);
    o += align256(sizeof(int64_t) * (size_t)(P + 1));
    a.order = reinterpret_cast<int32_t *>(b + o);
    o += align256(sizeof(int32_t) * (size_t)P);
    a.spref = reinterpret_cast<int64_t *>(b + o);
    o += align256(sizeof(int64_t) * (size_t)(P + 1));
    a.round_off = reinterpret_cast<int64_t *>(b + o);
    o += align256(sizeof(int64_t) * (size_t)(a.rb + 1));
    a.round_cnt = reinterpret_cast<int32_t *>(b + o);
    o += align256(sizeof(int32_t) * (size_t)(a.rb + 1));
    a.cursor = reinterpret_cast<int32_t *>(b + o);
    o += align256(sizeof(int32_t) * (size_t)(a.rb + 1));
    a.rounds = reinterpret_cast<int32_t *>(b + o);
    a.chunk_lo = a.rounds + 1;
    o += 256;
    a.kbound = reinterpret_cast<int32_t *>(b + o);
    o += align256(sizeof(int32_t) * (size_t)P);
    a.chunk_done = reinterpret_cast<int32_t *>(b + o);
    o += align256(sizeof(int32_t) * (size_t)a.cb);
    w.counts = reinterpret_cast<int32_t *>(b + counts_at);
    w.capacity = total;
    a.prefix = reinterpret_cast<int32_t *>(b + counts_at + align256(sizeof(int32_t) * (size_t)total));
}

// Required number of hypotheses for the best count c of N at confidence p
// (log_fail = log(1 - p)): K = ceil(log(1 - p) / log(1 - w^4)), w = c / N,
// clamped to [1, cap]; c <= 0 gives cap (Sec. 6.2).
__device__ int32_t adaptive_k(int32_t c, int64_t N, int32_t cap, double log_fail)
{
    if (c <= 0 || N <= 0) return cap;
    const double w = __ddiv_rn((double)c, (double)N);
    const double w2 = __dmul_rn(w, w);
    const double w4 = __dmul_rn(w2, w2);
    if (w4 >= 1.0) return 1;
    const double den = log1p(-w4);
    if (!(den < 0.0)) return cap;
    const double r = ceil(__ddiv_rn(log_fail, den));
    if (!(r < (double)cap)) return cap;
    return r < 1.0 ? 1 : (int32_t)r;
}

// Inclusive block scan of int64 (blockDim.x == 1024).
__device__ int64_t block_scan_incl(int64_t v, int64_t *warp_tot)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int64_t t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    if (wid > 0) v += warp_tot[wid - 1];
    return v;
}

// Size class of a problem for the scoring order: floor(log2 N), 0..31.
__device__ __forceinline__ int n_class(int64_t N)
{
    if (N <= 1) return 0;
    const int c = 63 - __clzll((unsigned long long)N);
    return c < 31 ? c : 31;
}

// Set-up of the fixed-count variant (one block of 1024 threads): hypothesis
// prefix sums in problem order, the scoring order, the work-item prefix sums
// over that order, the work counter.  With `by_size`, the scoring order is
// problems by size class, largest first (a counting sort; the order within
// a class follows the atomics and only affects speed), so that the last
// items handed out are the short ones of small problems and the final wave
// ends evenly (512 pairs: 0.691 -> 0.678 ms).  Small batches keep the
// problem order and the single pass (the sort's extra passes cost a one-pair
// RANSAC 2 us of its 18).
__global__ void __launch_bounds__(1024) ransac_prep_kernel(const int64_t *__restrict__ offsets,
                                                           const int32_t *__restrict__ n_hyp, int32_t P, int HB,
                                                           int T, Workspace ws, bool zero_here, bool by_size)
{
    __shared__ int64_t wt_a[32], wt_b[32];
    __shared__ int64_t carry_a, carry_b;
    __shared__ int32_t s_base[32];
    grid_launch_dependents();
    if (threadIdx.x == 0) {
        carry_a = 0;
        carry_b = 0;
        ws.hyp_off[0] = 0;
        ws.item_off[0] = 0;
        *ws.counter = 0ull;
        *ws.flags = 0;
    }
    if (threadIdx.x < 32) s_base[threadIdx.x] = 0;
    __syncthreads();
    for (int32_t base = 0; base < P; base += 1024) {
        const int32_t p = base + (int32_t)threadIdx.x;
        int64_t k = 0, items = 0;
        if (p < P) {
            k = n_hyp[p] > 0 ? n_hyp[p] : 0;
            const int64_t N = offsets[p + 1] - offsets[p];
            if (by_size) {
                atomicAdd(&s_base[n_class(N)], 1);
            } else {
                ws.order[p] = p;
                if (N >= 4 && k > 0)
                    items = ((k + HB - 1) / HB) * ((N + T - 1) / T);
            }
        }
        const int64_t ia = block_scan_incl(k, wt_a);
        const int64_t ib = by_size ? 0 : block_scan_incl(items, wt_b);
        if (p < P) {
            ws.hyp_off[p + 1] = carry_a + ia;
            if (!by_size) ws.item_off[p + 1] = carry_b + ib;
        }
        __syncthreads();
        if (threadIdx.x == 1023) {
            carry_a += ia;
            carry_b += ib;
        }
        __syncthreads();
    }
    if (by_size) {
        if (threadIdx.x == 0) {
            // first position of each class, largest class first
            int32_t acc = 0;
            for (int c = 31; c >= 0; --c) {
                const int32_t n = s_base[c];
                s_base[c] = acc;
                acc += n;
            }
        }
        __syncthreads();
        for (int32_t p = threadIdx.x; p < P; p += 1024)
            ws.order[atomicAdd(&s_base[n_class(offsets[p + 1] - offsets[p])], 1)] = p;
        __syncthreads();
        for (int32_t base = 0; base < P; base += 1024) {
            const int32_t j = base + (int32_t)threadIdx.x;
            int64_t items = 0;
            if (j < P) {
                const int32_t p = ws.order[j];
                const int64_t k = n_hyp[p] > 0 ? n_hyp[p] : 0;
                const int64_t N = offsets[p + 1] - offsets[p];
                if (N >= 4 && k > 0)
                    items = ((k + HB - 1) / HB) * ((N + T - 1) / T);
            }
            const int64_t ib = block_scan_incl(items, wt_b);
            if (j < P) ws.item_off[j + 1] = carry_b + ib;
            __syncthreads();
            if (threadIdx.x == 1023) carry_b += ib;
            __syncthreads();
        }
    }
    if (threadIdx.x == 0 && carry_a > ws.capacity) {
        *ws.flags = 1;
        ws.item_off[P] = 0;   // nothing to score
    }
    if (zero_here) {          // small workspaces: clear the counts here, no extra launch
        const int64_t lim = carry_a < ws.capacity ? carry_a : ws.capacity;
        for (int64_t i = threadIdx.x; i < lim; i += blockDim.x)
            ws.counts[i] = 0;
    }
}

// Round lists of one epoch of the adaptive variant (all 1024 threads of the
// block): the epoch scores chunks lo .. hi-1 of each problem, and of those
// only the ones before the problem's current bound (chunk c is dead once
// c * HB >= kbound, and kbound only decreases, so a bound read at any time
// drops dead chunks only).  Problem p gets C'_p = min(C_p, ceil(kbound / HB),
// hi) - lo live chunks (at least 0); the problems are sorted by C'_p, largest
// first (counting sort; the order among equal C'_p follows the atomics and
// only affects speed), so that round r, which holds chunk lo + r of every
// problem with C'_p > r, is a prefix of that order.  Resets the work counter.
__device__ void build_rounds(const int64_t *__restrict__ offsets, int32_t P, int HB, int T, int32_t lo, int32_t hi,
                             Workspace ws, AdaptiveWs aw, int64_t *wt_a, int64_t *wt_b, int64_t &carry_a,
                             int64_t &carry_b, int32_t &s_rounds)
{
    auto live_chunks = [&](int32_t p) -> int32_t {
        const int64_t C = aw.chunk_off[p + 1] - aw.chunk_off[p];
        const int64_t kb = aw.kbound[p];
        int64_t c = (kb + HB - 1) / HB;
        c = c < C ? c : C;
        c = c < hi ? c : hi;
        return c > lo ? (int32_t)(c - lo) : 0;
    };
    if (threadIdx.x == 0) s_rounds = 0;
    __syncthreads();
    for (int32_t p = threadIdx.x; p < P; p += 1024) {
        const int32_t c = live_chunks(p);
        if (c > 0) atomicMax(&s_rounds, c);
    }
    __syncthreads();
    const int32_t R = s_rounds;
    // histogram of C'_p over 0..R
    for (int32_t c = threadIdx.x; c <= R; c += 1024) aw.round_cnt[c] = 0;
    __syncthreads();
    for (int32_t p = threadIdx.x; p < P; p += 1024)
        atomicAdd(&aw.round_cnt[live_chunks(p)], 1);
    __syncthreads();
    // descending exclusive prefix: #{p : C'_p > c}; it is both the size of
    // round c and the first position of bin c in the order
    if (threadIdx.x == 0) carry_a = 0;
    __syncthreads();
    for (int32_t base = 0; base <= R; base += 1024) {
        const int32_t c = R - (base + (int32_t)threadIdx.x);
        const int64_t v = c >= 0 ? aw.round_cnt[c] : 0;
        const int64_t incl = block_scan_incl(v, wt_a);
        __syncthreads();                        // every thread has read its bin
        if (c >= 0) {
            const int32_t above = (int32_t)(carry_a + incl - v);
            aw.round_cnt[c] = above;
            aw.cursor[c] = above;
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry_a += incl;
        __syncthreads();
    }
    for (int32_t p = threadIdx.x; p < P; p += 1024) {
        const int32_t c = live_chunks(p);
        if (c > 0) aw.order[atomicAdd(&aw.cursor[c], 1)] = p;
    }
    __syncthreads();
    // slice prefix over the order, then the round offsets
    const int32_t n1 = R > 0 ? aw.round_cnt[0] : 0;
    if (threadIdx.x == 0) {
        carry_a = 0;
        carry_b = 0;
        aw.spref[0] = 0;
        aw.round_off[0] = 0;
    }
    __syncthreads();
    for (int32_t base = 0; base < n1; base += 1024) {
        const int32_t j = base + (int32_t)threadIdx.x;
        int64_t v = 0;
        if (j < n1) {
            const int32_t p = aw.order[j];
            v = (offsets[p + 1] - offsets[p] + T - 1) / T;
        }
        const int64_t incl = block_scan_incl(v, wt_a);
        if (j < n1) aw.spref[j + 1] = carry_a + incl;
        __syncthreads();
        if (threadIdx.x == 1023) carry_a += incl;
        __syncthreads();
    }
    for (int32_t base = 0; base < R; base += 1024) {
        const int32_t r = base + (int32_t)threadIdx.x;
        const int64_t v = r < R ? aw.spref[aw.round_cnt[r]] : 0;
        const int64_t incl = block_scan_incl(v, wt_b);
        if (r < R) aw.round_off[r + 1] = carry_b + incl;
        __syncthreads();
        if (threadIdx.x == 1023) carry_b += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *aw.rounds = R;
        *aw.chunk_lo = lo;
        *ws.counter = 0ull;
    }
}

// Set-up of the adaptive variant (one block of 1024 threads): the hypothesis
// and chunk offsets, the bounds (initially the cap) and the round lists of
// the first epoch (chunks 0 .. hi-1).
__global__ void __launch_bounds__(1024) ransac_prep_adaptive_kernel(const int64_t *__restrict__ offsets,
                                                                    const int32_t *__restrict__ max_hyp, int32_t P,
                                                                    int HB, int T, int32_t hi, Workspace ws,
                                                                    AdaptiveWs aw)
{
    __shared__ int64_t wt_a[32], wt_b[32];
    __shared__ int64_t carry_a, carry_b;
    __shared__ int32_t s_rounds;
    grid_launch_dependents();
    if (threadIdx.x == 0) {
        carry_a = carry_b = 0;
        s_rounds = 0;
        ws.hyp_off[0] = 0;
        aw.chunk_off[0] = 0;
        *ws.counter = 0ull;
        *ws.flags = 0;
        *aw.rounds = 0;
        aw.round_off[0] = 0;
    }
    __syncthreads();
    for (int32_t base = 0; base < P; base += 1024) {
        const int32_t p = base + (int32_t)threadIdx.x;
        int64_t k = 0, C = 0;
        if (p < P) {
            k = max_hyp[p] > 0 ? max_hyp[p] : 0;
            const int64_t N = offsets[p + 1] - offsets[p];
            if (N >= 4 && k > 0)
                C = (k + HB - 1) / HB;
            aw.kbound[p] = (int32_t)k;
            if (C > 0) atomicMax(&s_rounds, (int32_t)(C < 0x7fffffff ? C : 0x7fffffff));
        }
        const int64_t ia = block_scan_incl(k, wt_a);
        const int64_t ic = block_scan_incl(C, wt_b);
        if (p < P) {
            ws.hyp_off[p + 1] = carry_a + ia;
            aw.chunk_off[p + 1] = carry_b + ic;
        }
        __syncthreads();
        if (threadIdx.x == 1023) {
            carry_a += ia;
            carry_b += ic;
        }
        __syncthreads();
    }
    if (carry_a > ws.capacity || (int64_t)s_rounds > aw.rb || carry_b > aw.cb) {
        if (threadIdx.x == 0) *ws.flags = 1;    // nothing is scored (rounds stay 0)
        return;
    }
    __syncthreads();
    build_rounds(offsets, P, HB, T, 0, hi, ws, aw, wt_a, wt_b, carry_a, carry_b, s_rounds);
}

// Round lists of a later epoch (chunks lo .. hi-1), from the bounds the
// previous epochs left.  Waits for the previous kernel.
__global__ void __launch_bounds__(1024) ransac_replan_adaptive_kernel(const int64_t *__restrict__ offsets, int32_t P,
                                                                      int HB, int T, int32_t lo, int32_t hi,
                                                                      Workspace ws, AdaptiveWs aw)
{
    __shared__ int64_t wt_a[32], wt_b[32];
    __shared__ int64_t carry_a, carry_b;
    __shared__ int32_t s_rounds;
    grid_launch_dependents();
    grid_dependency_wait();
    if (*ws.flags) return;
    build_rounds(offsets, P, HB, T, lo, hi, ws, aw, wt_a, wt_b, carry_a, carry_b, s_rounds);
}

// Clears the counts and the chunk completion counters of the adaptive
// variant.  Their sizes are the workspace's, known before the set-up kernel
// runs, so the clearing overlaps the set-up; each block awaits the set-up's
// completion before it exits, and the scoring kernel awaits this one.
__global__ void zero_adaptive_kernel(Workspace ws, AdaptiveWs aw)
{
    grid_launch_dependents();
    const int64_t nc = ws.capacity, nk = aw.cb;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += stride) ws.counts[i] = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += stride) aw.chunk_done[i] = 0;
    grid_dependency_wait();
}

__global__ void zero_counts_kernel(Workspace ws, int32_t P)
{
    grid_launch_dependents();
    grid_dependency_wait();
    const int64_t total = ws.hyp_off[P];
    const int64_t lim = total < ws.capacity ? total : ws.capacity;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < lim; i += (int64_t)gridDim.x * blockDim.x)
        ws.counts[i] = 0;
}

struct ItemInfo {
    int64_t item;
    int32_t p;
    uint32_t N;
    int64_t base;   // first correspondence of problem p
    int64_t hbase;  // first hypothesis slot of problem p
    int32_t h0, nh; // hypotheses of this item
    int32_t i0, ni; // points of this item
    int32_t slice;
    // adaptive variant only
    int32_t S;      // slices of problem p
    int32_t k;      // hypothesis cap of problem p
    int64_t cid;    // chunk id (completion counter)
};

// Largest p with item_off[p] <= item (item_off non-decreasing, p < P):
// 32-way search by one warp.
__device__ int32_t find_problem(const int64_t *__restrict__ item_off, int32_t P, int64_t item)
{
    int32_t lo = 0, hi = P;   // answer in [lo, hi)
    const int lane = threadIdx.x & 31;
    while (hi - lo > 1) {
        const int32_t stride = (hi - lo + 31) / 32;
        const int32_t q = lo + lane * stride;
        const bool ok = q < hi && item_off[q] <= item;
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        const int last = 31 - __clz((int)b);   // lane 0 always satisfies (item_off[lo] <= item)
        lo = lo + last * stride;
        hi = min(hi, lo + stride);
    }
    return lo;
}

template <int HPT, bool ADAPTIVE>
__global__ void __launch_bounds__(512) ransac_score_kernel(const float4 *__restrict__ corr,
                                                           const int64_t *__restrict__ offsets,
                                                           const int32_t *__restrict__ n_hyp, int32_t P, float thr,
                                                           uint64_t seed, uint32_t prob_base, int T, bool ordered,
                                                           Workspace ws,
                                                           AdaptiveWs aw)
{
    constexpr int HB = 32 * HPT;
    extern __shared__ float4 smem4[];
    const int W = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4 *tile = smem4;                                                   // [T/2][2]: point pairs
    float *Hs = reinterpret_cast<float *>(smem4 + T);                       // [HB][12]
    int32_t *red = reinterpret_cast<int32_t *>(Hs + HB * 12);               // [W][HB]
    __shared__ ItemInfo info;
    __shared__ int32_t s_last;
    const float rthr = target_scale(thr);
    const float nanv = __int_as_float(0x7fc00000);

    grid_launch_dependents();
    grid_dependency_wait();
    // adaptive: the items of the current epoch, round 0 = chunk lo
    const int32_t R = ADAPTIVE ? *aw.rounds : 0;
    const int32_t lo = ADAPTIVE ? *aw.chunk_lo : 0;
    const int64_t total = ADAPTIVE ? aw.round_off[R] : ws.item_off[P];
    for (;;) {
        if (wid == 0) {
            for (;;) {
                int64_t item = 0;
                if (lane == 0)
                    item = (int64_t)atomicAdd(ws.counter, 1ull);
                item = __shfl_sync(0xffffffffu, item, 0);
                if (item >= total) {
                    if (lane == 0)
                        info.item = item;
                    break;
                }
                int32_t p = 0, chunk = 0, slice = 0, j_fixed = 0;
                if constexpr (ADAPTIVE) {
                    // round r = chunk lo + r of every problem with more than
                    // r live chunks in this epoch
                    const int32_t r = find_problem(aw.round_off, R, item);
                    const int64_t rbase = aw.round_off[r];
                    const int64_t rem = item - rbase;
                    const int32_t cnt = aw.round_cnt[r];
                    const int32_t j = find_problem(aw.spref, cnt, rem);
                    p = aw.order[j];
                    chunk = lo + r;
                    slice = (int32_t)(rem - aw.spref[j]);
                    if (chunk > 0) {
                        // The stop is certain before hypothesis kbound[q] of
                        // problem q, and kbound only decreases: a chunk at or
                        // past it stays dead.  The lanes check problem j and
                        // the next 31 of this round; if j is dead, the work
                        // counter jumps past the run of dead problems (their
                        // items of round r are contiguous), so nobody claims
                        // them one by one.  Items of the run already claimed
                        // by other blocks are dropped by them in the same way.
                        const int32_t jj = j + lane;
                        const bool dead = jj < cnt && chunk * HB >= __ldcg(&aw.kbound[aw.order[jj]]);
                        const unsigned live = __ballot_sync(0xffffffffu, !dead);
                        if (!(live & 1u)) {
                            const int32_t run = live ? __ffs(live) - 1 : 32;   // dead: j .. j + run - 1
                            if (lane == 0)
                                atomicMax(ws.counter, (unsigned long long)(rbase + aw.spref[j + run]));
                            continue;
                        }
                    }
                } else {
                    j_fixed = find_problem(ws.item_off, P, item);
                    p = ordered ? ws.order[j_fixed] : j_fixed;   // the order is the identity unless sorted
                }
                if (lane == 0) {
                    const int64_t base = offsets[p];
                    const uint32_t N = (uint32_t)(offsets[p + 1] - base);
                    const int32_t k = n_hyp[p];
                    const int32_t S = (int32_t)((N + T - 1) / T);
                    if constexpr (!ADAPTIVE) {
                        const int64_t r = item - ws.item_off[j_fixed];
                        chunk = (int32_t)(r / S);
                        slice = (int32_t)(r % S);
                    }
                    info.item = item;
                    info.p = p;
                    info.N = N;
                    info.base = base;
                    info.hbase = ws.hyp_off[p];
                    info.h0 = chunk * HB;
                    info.nh = min(HB, k - chunk * HB);
                    info.i0 = slice * T;
                    info.ni = (int32_t)min((int64_t)T, (int64_t)N - (int64_t)slice * T);
                    info.slice = slice;
                    if constexpr (ADAPTIVE) {
                        info.S = S;
                        info.k = k;
                        info.cid = aw.chunk_off[p] + chunk;
                    }
                }
                break;
            }
        }
        __syncthreads();
        // copy the item to registers now: warp 0 rewrites `info` for the next
        // item as soon as it has passed this iteration's last barrier
        if (info.item >= total)
            break;
        const int32_t p = info.p, nh = info.nh, h0 = info.h0, ni = info.ni, i0 = info.i0, slice = info.slice;
        const uint32_t N = info.N;
        const int64_t hbase = info.hbase;
        const float4 *cp = corr + info.base;

        // hypotheses of this item -> shared memory (test form, see inlier)
        if ((int)threadIdx.x < HB) {
            float H[9], G[9];
            const int t = threadIdx.x;
            bool valid = false;
            if (t < nh) {
                valid = make_hypothesis(cp, N, seed, prob_base + (uint32_t)p, (uint32_t)(h0 + t), H);
                if (!valid && slice == 0)
                    ws.counts[hbase + h0 + t] = -1;
            }
            if (!valid) {
#pragma unroll
                for (int i = 0; i < 9; ++i) H[i] = 0.0f;   // scores nothing (w == 0)
            }
            to_test_form(G, H, thr);
#pragma unroll
            for (int i = 0; i < 9; ++i) Hs[t * 12 + i] = G[i];
            Hs[t * 12 + 9] = valid ? 1.0f : 0.0f;
        }
        // correspondence slice -> shared memory as interleaved pairs; an odd
        // tail is padded with a NaN point (never an inlier)
        const int npairs = (ni + 1) >> 1;
        for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
            const float4 a = cp[i0 + 2 * q];
            const float4 b = (2 * q + 1 < ni) ? cp[i0 + 2 * q + 1] : make_float4(nanv, nanv, nanv, nanv);
            tile[2 * q] = make_float4(a.x, b.x, a.y, b.y);
            tile[2 * q + 1] = make_float4(F_MUL(a.z, rthr), F_MUL(b.z, rthr), F_MUL(a.w, rthr), F_MUL(b.w, rthr));
        }
        __syncthreads();

        float2 g[HPT][9];
        int cnt[HPT];
#pragma unroll
        for (int j = 0; j < HPT; ++j) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float v = Hs[(lane + 32 * j) * 12 + i];
                g[j][i] = make_float2(v, v);
            }
            cnt[j] = 0;
        }
        int q = wid;
        for (; q + W < npairs; q += 2 * W) {
            const float4 p0 = tile[2 * q], q0 = tile[2 * q + 1];
            const float4 p1 = tile[2 * (q + W)], q1 = tile[2 * (q + W) + 1];
#pragma unroll
            for (int j = 0; j < HPT; ++j)
                cnt[j] += inlier2(g[j], p0, q0) + inlier2(g[j], p1, q1);
        }
        for (; q < npairs; q += W) {
            const float4 p0 = tile[2 * q], q0 = tile[2 * q + 1];
#pragma unroll
            for (int j = 0; j < HPT; ++j) cnt[j] += inlier2(g[j], p0, q0);
        }
#pragma unroll
        for (int j = 0; j < HPT; ++j) red[wid * HB + lane + 32 * j] = cnt[j];
        __syncthreads();
        if ((int)threadIdx.x < nh && Hs[threadIdx.x * 12 + 9] != 0.0f) {
            int s = 0;
            for (int w = 0; w < W; ++w) s += red[w * HB + threadIdx.x];
            if (s)
                atomicAdd(&ws.counts[hbase + h0 + threadIdx.x], s);
        }
        if constexpr (ADAPTIVE) {
            // the last slice of a chunk publishes the chunk's bound
            const int64_t cid = info.cid;
            const int32_t S = info.S, kcap = info.k;
            __syncthreads();
            if (threadIdx.x == 0)
                s_last = (int32_t)atomic_add_acq_rel(reinterpret_cast<uint32_t *>(&aw.chunk_done[cid]), 1u) == S - 1;
            __syncthreads();
            if (s_last && wid == 0) {
                int32_t bc = -2, bj = 0x7fffffff;
                for (int t = lane; t < nh; t += 32) {
                    const int32_t c = __ldcg(&ws.counts[hbase + h0 + t]);
                    if (c > bc) { bc = c; bj = t; }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const int32_t c2 = __shfl_xor_sync(0xffffffffu, bc, o), j2 = __shfl_xor_sync(0xffffffffu, bj, o);
                    if (c2 > bc || (c2 == bc && j2 < bj)) { bc = c2; bj = j2; }
                }
                if (lane == 0 && bc > 0) {
                    const int32_t K = adaptive_k(bc, (int64_t)N, kcap, aw.log_fail);
                    atomicMin(&aw.kbound[p], max(h0 + bj + 1, K));
                }
            }
        }
    }
}

// Inlier mask of one problem under the test-form hypothesis G, the block's
// threads striding over the points with four loads in flight each.
__device__ void write_mask(const float G[9], const float4 *__restrict__ c, int64_t N, float rthr, bool any,
                           uint8_t *__restrict__ out)
{
    for (int64_t i0 = threadIdx.x; i0 < N; i0 += 4 * (int64_t)blockDim.x) {
        float4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = i0 + u * (int64_t)blockDim.x;
            q[u] = any && i < N ? c[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = i0 + u * (int64_t)blockDim.x;
            if (i < N) out[i] = any ? (uint8_t)inlier(G, q[u], rthr) : (uint8_t)0;
        }
    }
}

__global__ void __launch_bounds__(256) ransac_finish_kernel(const float4 *__restrict__ corr,
                                                            const int64_t *__restrict__ offsets,
                                                            const int32_t *__restrict__ n_hyp, int32_t P, float thr,
                                                            uint64_t seed, uint32_t prob_base, Workspace ws,
                                                            float *__restrict__ best_H, int32_t *__restrict__ best_count,
                                                            int32_t *__restrict__ best_hyp,
                                                            int32_t *__restrict__ hyp_counts,
                                                            uint8_t *__restrict__ mask)
{
    grid_launch_dependents();
    grid_dependency_wait();
    const int32_t p = blockIdx.x;
    const int64_t base = offsets[p];
    const int64_t N = offsets[p + 1] - base;
    const int32_t k = n_hyp[p] > 0 ? n_hyp[p] : 0;
    const int64_t hb = ws.hyp_off[p];
    const bool overflow = *ws.flags != 0;
    __shared__ int32_t s_cnt[8], s_idx[8];
    __shared__ float sH[9];
    __shared__ int32_t s_best;

    int32_t bc = -1, bi = 0x7fffffff;
    if (!overflow && N >= 4) {
        // four counts in flight per thread (one L2 round trip per four)
        for (int32_t h0 = threadIdx.x; h0 < k; h0 += 4 * (int32_t)blockDim.x) {
            int32_t c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t h = h0 + u * (int32_t)blockDim.x;
                c[u] = h < k ? ws.counts[hb + h] : -1;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t h = h0 + u * (int32_t)blockDim.x;
                if (h >= k) break;
                if (hyp_counts) hyp_counts[hb + h] = c[u];
                if (c[u] > bc || (c[u] == bc && h < bi)) { bc = c[u]; bi = h; }
            }
        }
    } else if (!overflow && hyp_counts) {
        for (int32_t h = threadIdx.x; h < k; h += blockDim.x) hyp_counts[hb + h] = -1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int32_t c = __shfl_down_sync(0xffffffffu, bc, o), i = __shfl_down_sync(0xffffffffu, bi, o);
        if (c > bc || (c == bc && i < bi)) { bc = c; bi = i; }
    }
    if ((threadIdx.x & 31) == 0) { s_cnt[threadIdx.x >> 5] = bc; s_idx[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        bc = s_cnt[0]; bi = s_idx[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (s_cnt[w] > bc || (s_cnt[w] == bc && s_idx[w] < bi)) { bc = s_cnt[w]; bi = s_idx[w]; }
        if (overflow) { bi = -2; bc = 0; }
        else if (bc < 0) { bi = -1; bc = 0; }
        s_best = bi;
        float H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (bi >= 0)
            make_hypothesis(corr + base, (uint32_t)N, seed, prob_base + (uint32_t)p, (uint32_t)bi, H);
#pragma unroll
        for (int i = 0; i < 9; ++i) sH[i] = H[i];
        best_hyp[p] = bi;
        best_count[p] = bc;
        normalize_frob(H);
#pragma unroll
        for (int i = 0; i < 9; ++i) best_H[9 * p + i] = H[i];
    }
    __syncthreads();
    if (mask) {
        float H[9], G[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) H[i] = sH[i];
        to_test_form(G, H, thr);
        write_mask(G, corr + base, N, target_scale(thr), s_best >= 0, mask + base);
    }
}

// ---------------------------------------------------------------------------
// Small batches (at most kFusedMaxP problems, e.g. one image pair): the whole
// RANSAC in ONE launch.  The work is items (problem p, chunk of HB hypotheses,
// slice s of S point ranges); block b takes items b, b + G, b + 2G, ...
// (every block derives the item layout from offsets and n_hyp itself: no
// set-up kernel, no work counter).  An item issues the loads of its first
// tile of points, samples and solves its HB hypotheses meanwhile, walks its
// point range tile by tile (T points staged in shared memory at a time) and
// stores its partial counts with plain stores into the slot of its slice,
// part[s][hyp], so that no count needs clearing and no atomic adds are made;
// the slice-0 item also stores each hypothesis's H.  A block that has
// finished all of its items counts itself done (an acquire-release add); the last one sums
// the slots of every hypothesis, takes each problem's argmax (ties to the
// lowest index), writes the mask and the outputs from the winner's stored H
// (the bits its scoring used), and sets the done counter back to zero for
// the next call.  Nothing waits on
// another block.  The counts, the argmax, H and the mask are those of the
// multi-kernel path bit for bit: integer sums do not depend on the split.
// ---------------------------------------------------------------------------
constexpr int32_t kFusedMaxP = 8;
constexpr int kFusedSlices = 4;

// 32-bit words per hypothesis in the workspace: on the one-launch path one
// count slot per slice plus the hypothesis's 9 entries of H, else one count.
constexpr int kFusedWords = kFusedSlices + 9;
size_t ransac_count_slots(int32_t P) { return P <= kFusedMaxP ? (size_t)kFusedWords : 1; }

template <int HPT>
__global__ void __launch_bounds__(512) ransac_fused_kernel(const float4 *__restrict__ corr,
                                                           const int64_t *__restrict__ offsets,
                                                           const int32_t *__restrict__ n_hyp, int32_t P, float thr,
                                                           uint64_t seed, uint32_t prob_base, int T, Workspace ws,
                                                           float *__restrict__ best_H, int32_t *__restrict__ best_count,
                                                           int32_t *__restrict__ best_hyp,
                                                           int32_t *__restrict__ hyp_counts, uint8_t *__restrict__ mask)
{
    constexpr int HB = 32 * HPT;
    extern __shared__ float4 smem4[];
    const int W = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4 *tile = smem4;                                                   // [T/2][2]: point pairs
    float *Hs = reinterpret_cast<float *>(smem4 + T);                       // [HB][12]
    int32_t *red = reinterpret_cast<int32_t *>(Hs + HB * 12);               // [W][HB]
    __shared__ int64_t s_item0[kFusedMaxP + 1], s_hoff[kFusedMaxP + 1], s_off[kFusedMaxP + 1];
    __shared__ int32_t s_overflow, s_last, s_best, s_S;
    __shared__ int32_t s_cnt[16], s_idx[16];
    __shared__ float sH[9];
    const float rthr = target_scale(thr);
    const float nanv = __int_as_float(0x7fc00000);

    grid_launch_dependents();
    grid_dependency_wait();
    if (wid == 0) {
        int64_t k = 0, chunks = 0;
        if (lane < P) {
            const int64_t N = offsets[lane + 1] - offsets[lane];
            k = n_hyp[lane] > 0 ? n_hyp[lane] : 0;
            if (N >= 4 && k > 0)
                chunks = (k + HB - 1) / HB;
            s_off[lane] = offsets[lane];
        }
        if (lane == 0) s_off[P] = offsets[P];
        // whole point ranges per item when the hypothesis chunks alone fill
        // half of the grid, else kFusedSlices point ranges per chunk (every
        // block takes the same decision)
        int64_t allc = chunks;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) allc += __shfl_xor_sync(0xffffffffu, allc, o);
        const int S = 2 * allc >= (int64_t)gridDim.x ? 1 : kFusedSlices;
        int64_t ik = k, ii = chunks * S;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t a = __shfl_up_sync(0xffffffffu, ik, o), b = __shfl_up_sync(0xffffffffu, ii, o);
            if (lane >= o) { ik += a; ii += b; }
        }
        if (lane < P) { s_hoff[lane + 1] = ik; s_item0[lane + 1] = ii; }
        if (lane == 0) { s_hoff[0] = 0; s_item0[0] = 0; s_S = S; }
        const int64_t tot = __shfl_sync(0xffffffffu, ik, 31);
        // the counts hold S slots of tot values each, then 9 floats per
        // hypothesis (its H)
        if (lane == 0) s_overflow = tot > ws.capacity / kFusedWords;
    }
    __syncthreads();
    const int64_t total_items = s_overflow ? 0 : s_item0[P];
    const int64_t total_h = s_hoff[P];
    const int S = s_S;
    int32_t *part = ws.counts;                                              // [S][total_h] (S > 1)
    float *hst = reinterpret_cast<float *>(ws.counts + (int64_t)kFusedSlices * total_h);  // [total_h][9]

    for (int64_t item = blockIdx.x; item < total_items; item += gridDim.x) {
        int32_t p = 0;
        while (s_item0[p + 1] <= item) ++p;
        const int64_t r = item - s_item0[p];
        const int32_t chunk = (int32_t)(r / S), slice = (int32_t)(r % S);
        const int64_t base = s_off[p];
        const uint32_t N = (uint32_t)(s_off[p + 1] - base);
        const int64_t hbase = s_hoff[p];
        const int32_t k = (int32_t)(s_hoff[p + 1] - hbase);
        const int32_t h0 = chunk * HB, nh = min(HB, k - h0);
        const int64_t L = (((int64_t)N + S - 1) / S + 1) & ~(int64_t)1;     // even slice length
        const int64_t i0 = (int64_t)slice * L;
        const int64_t ni = max((int64_t)0, min(L, (int64_t)N - i0));
        const float4 *cp = corr + base;
        auto stage = [&](int64_t t0, int nt) {
            const int npairs = (nt + 1) >> 1;
            for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
                const int64_t i = i0 + t0 + 2 * q;
                const float4 a = cp[i];
                const float4 b = (2 * q + 1 < nt) ? cp[i + 1] : make_float4(nanv, nanv, nanv, nanv);
                tile[2 * q] = make_float4(a.x, b.x, a.y, b.y);
                tile[2 * q + 1] = make_float4(F_MUL(a.z, rthr), F_MUL(b.z, rthr), F_MUL(a.w, rthr), F_MUL(b.w, rthr));
            }
        };
        // the first tile's loads go out before the hypotheses are solved, so
        // that their latencies overlap
        if (ni > 0) stage(0, (int)min((int64_t)T, ni));

        // hypotheses of this item -> shared memory (test form, see inlier);
        // the slice-0 item also keeps each H for the final re-use
        if ((int)threadIdx.x < HB) {
            float H[9], G[9];
            const int t = threadIdx.x;
            bool valid = false;
            if (t < nh)
                valid = make_hypothesis(cp, N, seed, prob_base + (uint32_t)p, (uint32_t)(h0 + t), H);
            if (!valid) {
#pragma unroll
                for (int i = 0; i < 9; ++i) H[i] = 0.0f;   // scores nothing (w == 0)
            }
            if (slice == 0 && t < nh) {
#pragma unroll
                for (int i = 0; i < 9; ++i) hst[(hbase + h0 + t) * 9 + i] = H[i];
            }
            to_test_form(G, H, thr);
#pragma unroll
            for (int i = 0; i < 9; ++i) Hs[t * 12 + i] = G[i];
            Hs[t * 12 + 9] = valid ? 1.0f : 0.0f;
        }
        __syncthreads();          // first tile and Hs written
        int cnt[HPT];
        float2 g[HPT][9];
#pragma unroll
        for (int j = 0; j < HPT; ++j) {
            cnt[j] = 0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float v = Hs[(lane + 32 * j) * 12 + i];
                g[j][i] = make_float2(v, v);
            }
        }
        for (int64_t t0 = 0; t0 < ni; t0 += T) {
            const int nt = (int)min((int64_t)T, ni - t0);
            const int npairs = (nt + 1) >> 1;
            if (t0 > 0) {
                __syncthreads();  // the previous tile is consumed
                stage(t0, nt);
                __syncthreads();
            }
            int q = wid;
            for (; q + W < npairs; q += 2 * W) {
                const float4 p0 = tile[2 * q], q0 = tile[2 * q + 1];
                const float4 p1 = tile[2 * (q + W)], q1 = tile[2 * (q + W) + 1];
#pragma unroll
                for (int j = 0; j < HPT; ++j)
                    cnt[j] += inlier2(g[j], p0, q0) + inlier2(g[j], p1, q1);
            }
            for (; q < npairs; q += W) {
                const float4 p0 = tile[2 * q], q0 = tile[2 * q + 1];
#pragma unroll
                for (int j = 0; j < HPT; ++j) cnt[j] += inlier2(g[j], p0, q0);
            }
        }
#pragma unroll
        for (int j = 0; j < HPT; ++j) red[wid * HB + lane + 32 * j] = cnt[j];
        __syncthreads();
        int32_t c = -1;
        if ((int)threadIdx.x < nh) {
            c = 0;
            for (int w = 0; w < W; ++w) c += red[w * HB + threadIdx.x];
            // a degenerate sample is marked in slot 0 (its counts are 0)
            if (Hs[threadIdx.x * 12 + 9] == 0.0f) c = slice == 0 ? -1 : 0;
            if (S > 1)
                part[(int64_t)slice * total_h + hbase + h0 + threadIdx.x] = c;
            else if (hyp_counts)
                hyp_counts[hbase + h0 + threadIdx.x] = c;
        }
        if (S == 1 && (int)threadIdx.x < HB) {
            // whole range: the counts are final; the chunk's best (highest
            // count, then lowest index) joins the problem's packed maximum
            int32_t bi = (int)threadIdx.x < nh ? h0 + (int32_t)threadIdx.x : 0x7fffffff;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const int32_t c2 = __shfl_down_sync(0xffffffffu, c, o), i2 = __shfl_down_sync(0xffffffffu, bi, o);
                if (c2 > c || (c2 == c && i2 < bi)) { c = c2; bi = i2; }
            }
            if (lane == 0 && c >= 0)
                atomicMax(&ws.best[p], ((unsigned long long)(uint32_t)c << 32) | (unsigned long long)(0xffffffffu - (uint32_t)bi));
        }
        __syncthreads();          // Hs and red are rewritten by the next item
    }

    // the last block to finish takes the argmax of every problem
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomic_add_acq_rel(ws.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last)
        return;
    const bool overflow = s_overflow != 0;
    for (int32_t p = 0; p < P; ++p) {
        const int64_t base = s_off[p];
        const int64_t N = s_off[p + 1] - base;
        const int64_t hb = s_hoff[p];
        const int32_t k = (int32_t)(s_hoff[p + 1] - hb);
        int32_t bc = -1, bi = 0x7fffffff;
        if (!overflow && N >= 4 && S == 1) {
            // the packed maximum of the items (0: no valid hypothesis)
            if (threadIdx.x == 0) {
                const unsigned long long v = __ldcg(&ws.best[p]);
                if (v) { bc = (int32_t)(v >> 32); bi = (int32_t)(0xffffffffu - (uint32_t)v); }
            }
        } else if (!overflow && N >= 4) {
            // all slots of four hypotheses per thread in flight at once (one
            // L2 round trip per 4 x blockDim hypotheses)
            for (int32_t h0 = threadIdx.x; h0 < k; h0 += 4 * (int32_t)blockDim.x) {
                constexpr int SL = kFusedSlices;
                int32_t c[4][SL];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t h = h0 + u * (int32_t)blockDim.x;
#pragma unroll
                    for (int sl = 0; sl < SL; ++sl)
                        c[u][sl] = h < k ? __ldcg(&part[(int64_t)sl * total_h + hb + h]) : -1;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t h = h0 + u * (int32_t)blockDim.x;
                    if (h >= k) break;
                    int32_t t = c[u][0];
                    if (t >= 0) {
#pragma unroll
                        for (int sl = 1; sl < SL; ++sl) t += c[u][sl];
                    }
                    if (hyp_counts) hyp_counts[hb + h] = t;
                    if (t > bc) { bc = t; bi = h; }
                }
            }
        } else if (!overflow && hyp_counts) {
            for (int32_t h = threadIdx.x; h < k; h += blockDim.x) hyp_counts[hb + h] = -1;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int32_t c = __shfl_down_sync(0xffffffffu, bc, o), i = __shfl_down_sync(0xffffffffu, bi, o);
            if (c > bc || (c == bc && i < bi)) { bc = c; bi = i; }
        }
        if (lane == 0) { s_cnt[wid] = bc; s_idx[wid] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            bc = s_cnt[0]; bi = s_idx[0];
            for (int w = 1; w < W; ++w)
                if (s_cnt[w] > bc || (s_cnt[w] == bc && s_idx[w] < bi)) { bc = s_cnt[w]; bi = s_idx[w]; }
            if (overflow) { bi = -2; bc = 0; }
            else if (bc < 0) { bi = -1; bc = 0; }
            s_best = bi;
            float H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            if (bi >= 0) {        // the winner's H as its scoring item solved it
#pragma unroll
                for (int i = 0; i < 9; ++i) H[i] = __ldcg(&hst[(hb + bi) * 9 + i]);
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) sH[i] = H[i];
            best_hyp[p] = bi;
            best_count[p] = bc;
            normalize_frob(H);
#pragma unroll
            for (int i = 0; i < 9; ++i) best_H[9 * p + i] = H[i];
        }
        __syncthreads();
        if (mask) {
            float H[9], G[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) H[i] = sH[i];
            to_test_form(G, H, thr);
            write_mask(G, corr + base, N, target_scale(thr), s_best >= 0, mask + base);
        }
        __syncthreads();          // s_cnt, sH are reused by the next problem
    }
    if (threadIdx.x < kFusedMaxP)
        ws.best[threadIdx.x] = 0ull;
    if (threadIdx.x == 0)
        *ws.done = 0u;
}

// Adaptive finish, one block of 512 threads per problem: inclusive prefix
// maxima I of the counts, tile by tile (2048 hypotheses), until the stop is
// certain within the scanned part; the stop index is the first i in 1..k with
// i >= K(I[i-1]) (monotone in i: I does not decrease and K does not increase
// with the count), found by a 32-way search; the best is I at the stop and
// its first index.  Hypotheses at or after the stop are reported as -2.
__global__ void __launch_bounds__(512) ransac_finish_adaptive_kernel(
    const float4 *__restrict__ corr, const int64_t *__restrict__ offsets, const int32_t *__restrict__ max_hyp,
    float thr, uint64_t seed, uint32_t prob_base, Workspace ws, AdaptiveWs aw, float *__restrict__ best_H,
    int32_t *__restrict__ best_count, int32_t *__restrict__ best_hyp, int32_t *__restrict__ n_eval,
    int32_t *__restrict__ hyp_counts, uint8_t *__restrict__ mask)
{
    constexpr int kPer = 16, kTile = kPer * 512;
    grid_launch_dependents();
    grid_dependency_wait();
    const int32_t p = blockIdx.x;
    const int64_t base = offsets[p];
    const int64_t N = offsets[p + 1] - base;
    const int32_t k = max_hyp[p] > 0 ? max_hyp[p] : 0;
    const bool overflow = *ws.flags != 0;
    const int64_t hb = overflow ? 0 : ws.hyp_off[p];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ int32_t s_wmax[16], s_carry, s_end, s_istar, s_bi;
    __shared__ float sH[9];
    const int32_t *cnt = ws.counts + hb;
    int32_t *pre = aw.prefix + hb;

    if (threadIdx.x == 0) {
        s_carry = -2;
        s_end = 0;
        s_istar = 0;
        s_bi = 0x7fffffff;
    }
    __syncthreads();
    const bool active = !overflow && N >= 4 && k > 0;
    if (active) {
        // The stop is at or before the bound the scoring left: at i = kbound
        // the best of 0..i-1 is at least the count c_j that set it, and K is
        // non-increasing, so K(best) <= K(c_j) <= kbound.  The prefix maxima
        // are needed up to there only (every chunk before it was scored).
        const int32_t lim = min(k, max(1, aw.kbound[p]));
        for (int32_t t0 = 0; t0 < lim; t0 += kTile) {
            const int32_t b = t0 + kPer * (int32_t)threadIdx.x;
            int32_t m[kPer], run = -2;
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int32_t c = b + q < lim ? cnt[b + q] : -2;
                run = max(run, c);
                m[q] = run;
            }
            // exclusive max-scan of the thread maxima
            int32_t incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl = max(incl, t);
            }
            if (lane == 31) s_wmax[wid] = incl;
            __syncthreads();
            int32_t before = s_carry;
            for (int w = 0; w < wid; ++w) before = max(before, s_wmax[w]);
            const int32_t excl = __shfl_up_sync(0xffffffffu, incl, 1);
            if (lane > 0) before = max(before, excl);
#pragma unroll
            for (int q = 0; q < kPer; ++q)
                if (b + q < lim) pre[b + q] = max(before, m[q]);
            __syncthreads();
            if (threadIdx.x == 0) {
                int32_t tile_max = s_carry;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tile_max = max(tile_max, s_wmax[w]);
                s_carry = tile_max;
                s_end = lim;
            }
            __syncthreads();
        }
        // first i in [1, end] with the stop condition (it holds at end)
        if (wid == 0) {
            int32_t lo = 1, hi = s_end;
            while (lo < hi) {
                const int32_t st = (hi - lo + 30) / 31;    // lane 31 reaches hi: some lane holds
                const int32_t q = lo + lane * st;
                bool ok = true;
                if (q < hi) ok = q == k || q >= adaptive_k(pre[q - 1], N, k, aw.log_fail);
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                const int f = __ffs(bal) - 1;
                const int32_t nhi = min(hi, lo + f * st);
                lo = f > 0 ? lo + (f - 1) * st + 1 : lo;
                hi = nhi;
            }
            if (lane == 0) s_istar = lo;
        }
        __syncthreads();
        // first index of the best count before the stop: the first h with
        // pre[h] >= best (the prefix maxima do not decrease, and first reach
        // the best where it first occurs; it holds at istar - 1)
        if (wid == 0) {
            const int32_t best = pre[s_istar - 1];
            int32_t lo = 0, hi = s_istar - 1;
            while (lo < hi) {
                const int32_t st = (hi - lo + 30) / 31;
                const int32_t q = lo + lane * st;
                const bool ok = q >= hi || pre[q] >= best;
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                const int f = __ffs(bal) - 1;
                const int32_t nhi = min(hi, lo + f * st);
                lo = f > 0 ? lo + (f - 1) * st + 1 : lo;
                hi = nhi;
            }
            if (lane == 0) s_bi = lo;
        }
    }
    __syncthreads();
    const int32_t istar = s_istar;
    if (hyp_counts && !overflow) {
#pragma unroll 4
        for (int32_t h = threadIdx.x; h < k; h += blockDim.x)
            hyp_counts[hb + h] = !active ? -1 : (h < istar ? cnt[h] : -2);
    }
    if (threadIdx.x == 0) {
        int32_t bi = -1, bc = 0;
        if (overflow) {
            bi = -2;
        } else if (active && s_bi != 0x7fffffff && pre[istar - 1] >= 0) {
            bi = s_bi;
            bc = pre[istar - 1];
        }
        s_bi = bi;
        float H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (bi >= 0)
            make_hypothesis(corr + base, (uint32_t)N, seed, prob_base + (uint32_t)p, (uint32_t)bi, H);
#pragma unroll
        for (int i = 0; i < 9; ++i) sH[i] = H[i];
        best_hyp[p] = bi;
        best_count[p] = bc;
        if (n_eval) n_eval[p] = overflow ? 0 : istar;
        normalize_frob(H);
#pragma unroll
        for (int i = 0; i < 9; ++i) best_H[9 * p + i] = H[i];
    }
    __syncthreads();
    if (mask) {
        float H[9], G[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) H[i] = sH[i];
        to_test_form(G, H, thr);
        write_mask(G, corr + base, N, target_scale(thr), s_bi >= 0, mask + base);
    }
}

__global__ void sample_indices_kernel(uint32_t N, int32_t n_hyp, uint64_t seed, uint32_t prob, int4 *__restrict__ idx)
{
    for (int32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < n_hyp; h += gridDim.x * blockDim.x) {
        uint32_t i[4];
        sample4(seed, prob, (uint32_t)h, N, i);
        idx[h] = make_int4((int)i[0], (int)i[1], (int)i[2], (int)i[3]);
    }
}

}  // namespace aca

using namespace aca;

extern "C" aca_status aca_sample_indices(int64_t N, int32_t n_hyp, uint64_t seed, uint32_t problem, int32_t *idx,
                                         void *stream)
{
    if (N < 4 || N >= (int64_t(1) << 31))
        return set_error(ACA_ERR_INVALID_ARG, "aca_sample_indices: need 4 <= N < 2^31");
    if (n_hyp < 0)
        return set_error(ACA_ERR_INVALID_ARG, "aca_sample_indices: n_hyp < 0");
    if (n_hyp == 0)
        return ACA_OK;
    if (!idx || !aligned16(idx))
        return set_error(ACA_ERR_INVALID_ARG, "aca_sample_indices: idx must be non-null and 16-byte aligned");
    const int threads = 256;
    const int grid = resident_grid(sample_indices_kernel, threads, 0, (n_hyp + threads - 1) / threads);
    sample_indices_kernel<<<grid, threads, 0, as_stream(stream)>>>((uint32_t)N, n_hyp, seed, problem,
                                                                  reinterpret_cast<int4 *>(idx));
    return check_launch("aca_sample_indices");
}

extern "C" size_t ransac_aca_workspace_size(int32_t P, int64_t total_hyps)
{
    if (P < 0 || total_hyps < 0)
        return 0;
    return header_bytes(P) + align256(sizeof(int32_t) * (size_t)total_hyps * ransac_count_slots(P));
}

extern "C" aca_status ransac_aca(const float *corr, const int64_t *offsets, const int32_t *n_hyp, int32_t P,
                                 const aca_ransac_params *params, float *best_H, int32_t *best_count,
                                 int32_t *best_hyp, int32_t *hyp_counts, uint8_t *inlier_mask, void *workspace,
                                 size_t workspace_bytes, void *stream)
{
    if (P < 0)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca: P < 0");
    if (P == 0)
        return ACA_OK;
    if (!corr || !offsets || !n_hyp || !params || !best_H || !best_count || !best_hyp || !workspace)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca: null pointer");
    if (!aligned16(corr))
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca: corr must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca: workspace must be 256-byte aligned");
    if (workspace_bytes < header_bytes(P))
        return set_error(ACA_ERR_WORKSPACE, "ransac_aca: workspace smaller than %zu bytes", header_bytes(P));
    if (!(params->threshold_px > 0.0f))
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca: threshold_px must be > 0");
    const int W = params->block_warps ? params->block_warps : 8;
    const int HPT = params->hyps_per_thread ? params->hyps_per_thread : 2;
    const int T = params->tile_points ? params->tile_points : 1024;
    if (W < 1 || W > 16)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca: block_warps must be in 1..16");
    if (HPT != 1 && HPT != 2 && HPT != 4)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca: hyps_per_thread must be 1, 2 or 4");
    if (T < 32 || T > 8192 || T % 32 != 0)   // even: the tile holds point pairs
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca: tile_points must be a multiple of 32 in 32..8192");
    if (32 * HPT > 32 * W)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca: need hyps_per_thread <= block_warps");
    const int HB = 32 * HPT;
    const cudaStream_t st = as_stream(stream);
    const Workspace ws = carve(workspace, P, workspace_bytes);
    const size_t smem = (size_t)T * 16 + (size_t)HB * 12 * 4 + (size_t)W * HB * 4;
    const int threads = 32 * W;
    const float4 *c4 = reinterpret_cast<const float4 *>(corr);
    aca_status s = ACA_OK;

    if (P <= kFusedMaxP) {
        // small batches: everything in one launch (ransac_fused_kernel)
#define ACA_FUSED(HPTV)                                                                                       \
    {                                                                                                          \
        auto k = ransac_fused_kernel<HPTV>;                                                                    \
        if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                                     (int)smem) != cudaSuccess)                                \
            return set_error(ACA_ERR_CUDA, "ransac_aca: cannot reserve %zu bytes of shared memory", smem);    \
        const int grid = params->grid_blocks > 0 ? params->grid_blocks : resident_grid(k, threads, smem, 1 << 30); \
        launch_after_previous(k, dim3(grid), dim3(threads), smem, st, c4, offsets, n_hyp, P, params->threshold_px, \
                              params->seed, params->problem_base, T, ws, best_H, best_count, best_hyp, hyp_counts, \
                              inlier_mask);                                                                    \
    }
        if (HPT == 1) ACA_FUSED(1)
        else if (HPT == 2) ACA_FUSED(2)
        else ACA_FUSED(4)
#undef ACA_FUSED
        return check_launch("ransac_aca (one launch)");
    }

    // counts of small workspaces are cleared by the prep kernel itself
    const bool zero_in_prep = ws.capacity <= 65536;
    const bool by_size = P >= 64;     // problems by size, largest first (ransac_prep_kernel)
    ransac_prep_kernel<<<1, 1024, 0, st>>>(offsets, n_hyp, P, HB, T, ws, zero_in_prep, by_size);
    s = check_launch("ransac_aca (prep)");
    if (s != ACA_OK) return s;
    if (!zero_in_prep) {
        const int threads = 256;
        const int grid = resident_grid(zero_counts_kernel, threads, 0, (ws.capacity + threads - 1) / threads);
        launch_after_previous(zero_counts_kernel, dim3(grid), dim3(threads), 0, st, ws, P);
        if ((s = check_launch("ransac_aca (zero)")) != ACA_OK) return s;
    }
#define ACA_SCORE(HPTV)                                                                                       \
    {                                                                                                          \
        auto k = ransac_score_kernel<HPTV, false>;                                                             \
        if (smem > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                                                     (int)smem) != cudaSuccess)                                \
            return set_error(ACA_ERR_CUDA, "ransac_aca: cannot reserve %zu bytes of shared memory", smem);    \
        const int grid = params->grid_blocks > 0 ? params->grid_blocks : resident_grid(k, threads, smem, 1 << 30); \
        launch_after_previous(k, dim3(grid), dim3(threads), smem, st, c4, offsets, n_hyp, P,                   \
                              params->threshold_px, params->seed, params->problem_base, T, by_size, ws,      \
                              AdaptiveWs{});                                                                   \
    }
    if (HPT == 1) ACA_SCORE(1)
    else if (HPT == 2) ACA_SCORE(2)
    else ACA_SCORE(4)
#undef ACA_SCORE
    if ((s = check_launch("ransac_aca (score)")) != ACA_OK) return s;
    launch_after_previous(ransac_finish_kernel, dim3(P), dim3(256), 0, st, c4, offsets, n_hyp, P,
                          params->threshold_px, params->seed, params->problem_base, ws, best_H, best_count, best_hyp,
                          hyp_counts, inlier_mask);
    return check_launch("ransac_aca (finish)");
}

extern "C" size_t ransac_aca_adaptive_workspace_size(int32_t P, int64_t total_max_hyps)
{
    if (P < 0 || total_max_hyps < 0)
        return 0;
    return adaptive_bytes(P, total_max_hyps, nullptr, nullptr, nullptr);
}

extern "C" aca_status ransac_aca_adaptive(const float *corr, const int64_t *offsets, const int32_t *max_hyp,
                                          int32_t P, int64_t total_max_hyps, const aca_ransac_params *params,
                                          double confidence, float *best_H, int32_t *best_count, int32_t *best_hyp,
                                          int32_t *n_evaluated, int32_t *hyp_counts, uint8_t *inlier_mask,
                                          void *workspace, size_t workspace_bytes, void *stream)
{
    if (P < 0 || total_max_hyps < 0)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca_adaptive: P < 0 or total_max_hyps < 0");
    if (P == 0)
        return ACA_OK;
    if (!corr || !offsets || !max_hyp || !params || !best_H || !best_count || !best_hyp || !workspace)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca_adaptive: null pointer");
    if (!aligned16(corr))
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca_adaptive: corr must be 16-byte aligned");
    if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca_adaptive: workspace must be 256-byte aligned");
    const size_t need = adaptive_bytes(P, total_max_hyps, nullptr, nullptr, nullptr);
    if (workspace_bytes < need)
        return set_error(ACA_ERR_WORKSPACE, "ransac_aca_adaptive: workspace smaller than %zu bytes", need);
    if (!(params->threshold_px > 0.0f))
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca_adaptive: threshold_px must be > 0");
    if (!(confidence > 0.0 && confidence < 1.0))
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca_adaptive: confidence must be in (0, 1)");
    const int W = params->block_warps ? params->block_warps : 8;
    const int HPT = params->hyps_per_thread ? params->hyps_per_thread : 2;
    const int T = params->tile_points ? params->tile_points : 1024;
    if (W < 1 || W > 16)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca_adaptive: block_warps must be in 1..16");
    if (HPT != 1 && HPT != 2 && HPT != 4)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca_adaptive: hyps_per_thread must be 1, 2 or 4");
    if (T < 32 || T > 8192 || T % 32 != 0)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca_adaptive: tile_points must be a multiple of 32 in 32..8192");
    if (HPT > W)
        return set_error(ACA_ERR_INVALID_ARG, "ransac_aca_adaptive: need hyps_per_thread <= block_warps");
    const int HB = 32 * HPT;
    const cudaStream_t st = as_stream(stream);
    Workspace ws;
    AdaptiveWs aw;
    carve_adaptive(workspace, P, total_max_hyps, ws, aw);
    aw.log_fail = log(1.0 - confidence);

    // Epochs: chunk 0 of every problem first, then the chunks still before
    // each problem's bound, re-planned from the bounds the first epoch left.
    // Measured on 512 pairs with a cap of 16384: claiming the dead chunks of
    // the full-cap item space one by one cost 13 % of the batch; the re-plan
    // boundary costs about 4 %; a first epoch of 1, 2, 3 or 4 chunks gave
    // the same time within 1 %, and a third epoch was slower.
    constexpr int32_t kEpochEnd[] = {1, 0x7fffffff};
    constexpr int kEpochs = (int)(sizeof(kEpochEnd) / sizeof(kEpochEnd[0]));
    // The first epoch scores chunk 0 only (about 1.4 waves of items over the
    // resident blocks); items of a quarter tile balance its last wave
    // better: 1.320 against 1.333 ms on 512 pairs (half a tile: 1.323).
    constexpr int kFirstEpochTileDiv = 4;
    const int Te[kEpochs] = {(T / kFirstEpochTileDiv) < 32 ? 32 : ((T / kFirstEpochTileDiv) & ~31), T};
    ransac_prep_adaptive_kernel<<<1, 1024, 0, st>>>(offsets, max_hyp, P, HB, Te[0], kEpochEnd[0], ws, aw);
    aca_status s = check_launch("ransac_aca_adaptive (prep)");
    if (s != ACA_OK) return s;
    {
        const int threads = 256;
        const int64_t work = total_max_hyps > aw.cb ? total_max_hyps : aw.cb;
        const int grid = resident_grid(zero_adaptive_kernel, threads, 0, (work + threads - 1) / threads);
        launch_after_previous(zero_adaptive_kernel, dim3(grid), dim3(threads), 0, st, ws, aw);
        if ((s = check_launch("ransac_aca_adaptive (zero)")) != ACA_OK) return s;
    }
    const size_t smem = (size_t)T * 16 + (size_t)HB * 12 * 4 + (size_t)W * HB * 4;
    const int threads = 32 * W;
    const float4 *c4 = reinterpret_cast<const float4 *>(corr);
    auto score = [&](auto kernel, int Tk) -> aca_status {
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return set_error(ACA_ERR_CUDA, "ransac_aca_adaptive: cannot reserve %zu bytes of shared memory", smem);
        const int grid = params->grid_blocks > 0 ? params->grid_blocks : resident_grid(kernel, threads, smem, 1 << 30);
        launch_after_previous(kernel, dim3(grid), dim3(threads), smem, st, c4, offsets, max_hyp, P,
                              params->threshold_px, params->seed, params->problem_base, Tk, false, ws, aw);
        return check_launch("ransac_aca_adaptive (score)");
    };
    for (int e = 0; e < kEpochs; ++e) {
        if (e > 0) {
            launch_after_previous(ransac_replan_adaptive_kernel, dim3(1), dim3(1024), 0, st, offsets, P, HB, Te[e],
                                  kEpochEnd[e - 1], kEpochEnd[e], ws, aw);
            if ((s = check_launch("ransac_aca_adaptive (replan)")) != ACA_OK) return s;
        }
        s = HPT == 1 ? score(ransac_score_kernel<1, true>, Te[e])
                     : HPT == 2 ? score(ransac_score_kernel<2, true>, Te[e]) : score(ransac_score_kernel<4, true>, Te[e]);
        if (s != ACA_OK) return s;
    }
    launch_after_previous(ransac_finish_adaptive_kernel, dim3(P), dim3(512), 0, st, c4, offsets, max_hyp,
                          params->threshold_px, params->seed, params->problem_base, ws, aw, best_H, best_count,
                          best_hyp, n_evaluated, hyp_counts, inlier_mask);
    return check_launch("ransac_aca_adaptive (finish)");
}
