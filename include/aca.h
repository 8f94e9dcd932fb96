/*
 * aca.h - C ABI of the GB300 (sm_103a) minimal-homography library.
 *
 * Batched 4-point homography solvers from "Fast and Interpretable 2D
 * Homography Decomposition: Similarity-Kernel-Similarity and
 * Affine-Core-Affine Transformations" (arXiv 2402.18008), the RANSAC
 * hypothesis scoring they feed, and the derivative of ACA for networks that
 * regress 4-point offsets.
 *
 * Conventions shared by every call
 * --------------------------------
 * - All array arguments are DEVICE pointers owned by the caller (for example
 *   the storage of torch tensors).  The library allocates no memory and keeps
 *   no pointer after the call returns.
 * - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL = the
 *   legacy default stream) and is asynchronous: results are valid once the
 *   stream has been synchronised.  Calls contain no host synchronisation and
 *   can be captured in a CUDA graph.
 * - Argument errors are detected on the host before anything is launched and
 *   returned as ACA_ERR_INVALID_ARG; a failed launch returns ACA_ERR_CUDA.
 *   aca_last_error() then returns a message (thread-local, valid until the
 *   next call on the same thread).
 * - Homographies are 3x3, row-major h11 h12 h13 h21 ... h33, and map source
 *   to target points: x2 ~ H x1 up to scale (the problem statement of
 *   Sec. 2.1, Eq. 1).
 * - Minimal sets are stored as 16 planes of `ld` floats ("SoA"): plane
 *   p = side*8 + point*2 + coord, side 0 = source, 1 = target, point 0..3 =
 *   M, N, P, Q (M, N, P are the three anchor points of Sec. 4.2, Q the
 *   fourth correspondence), coord 0 = x, 1 = y.  Outputs use 9 planes of
 *   `ld` floats.  n <= ld.  Entries n..ld-1 of outputs are not written.
 *   When `ld` is a multiple of 4 and every plane pointer is 16-byte aligned
 *   the kernels use 16-byte vector accesses; otherwise a scalar variant runs.
 */
#ifndef ACA_GB300_H
#define ACA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ACA_OK = 0,
    ACA_ERR_INVALID_ARG = -1, /* null pointer, bad size, misaligned workspace */
    ACA_ERR_CUDA = -2,        /* a CUDA runtime call failed (message in aca_last_error) */
    ACA_ERR_WORKSPACE = -3,   /* workspace too small */
    ACA_ERR_TIMEOUT = -4      /* reserved: a device-side wait gave up (no current kernel waits) */
} aca_status;

typedef enum {
    ACA_NORM_NONE = 0, /* the division-free H of Eq. 24 / Eq. 28-29, unscaled */
    ACA_NORM_H33 = 1,  /* divided by h33 (Sec. 3.4: one division, eight multiplications) */
    ACA_NORM_FROB = 2  /* unit Frobenius norm, h33 > 0 (or, if |h33| < 1e-6 |H|,
                          the entry of largest magnitude > 0) */
} aca_norm;

/* Flag bits written per set when `flags` is not NULL. */
#define ACA_FLAG_SRC_ANCHORS 1u /* M1 N1 P1: 2*area / longest side < 1 px */
#define ACA_FLAG_TGT_ANCHORS 2u /* M2 N2 P2: 2*area / longest side < 1 px */
#define ACA_FLAG_OTHER_TRIPLE 4u /* a triple containing Q (either side) < 1 px */
#define ACA_FLAG_NON_FINITE 8u   /* a non-finite input or output value */

/*
 * aca_solve - batched ACA minimal solve (Sec. 4, Eq. 20-29; composition
 * Eq. 24; no division unless a normalisation is requested).
 *   pts   [16][ld] float, SoA minimal sets (see above), read-only.
 *   H     [9][ld] float, output homographies.
 *   flags [ld] uint8 or NULL: per-set ACA_FLAG_* bits.  Degenerate sets are
 *         not errors: ACA has no division, so H stays finite (rank-deficient).
 *   pts, H and flags may each be device memory or host memory the device can
 *   address (page-locked, e.g. cudaHostAlloc or cudaHostRegister): the
 *   kernel then reads the sets from and writes H to host memory itself, over
 *   the host link, with no staging copy (zero-copy; on GB300 the link, not
 *   HBM, then bounds the call).
 *   n     number of sets, 0 <= n <= ld (n = 0 launches nothing).
 *   norm  ACA_NORM_*; ACA_NORM_NONE returns the paper's unnormalised H (the
 *         function aca_backward differentiates).
 */
aca_status aca_solve(const float *pts, float *H, uint8_t *flags, int64_t n, int64_t ld, int32_t norm,
                     void *stream);

/*
 * sks_solve - batched SKS minimal solve (Sec. 3, Eq. 4-14: two similarities
 * from the anchor pair M, N, a 4-parameter kernel H_K from P and Q).  Same
 * layout, flags and normalisations as aca_solve.  The paper's SKS divides
 * by P3.y, Q3.y and Q7.x^2 - Q7.y^2; the library evaluates Eq. 11-13 over
 * their common denominator without a division, so a set where one of them
 * vanishes (M, N and P or Q collinear, or P, Q and M or N collinear, on
 * either side) gives a finite but degenerate H.  Such sets are near
 * collinear triples, which the flag bits report as for aca_solve.
 */
aca_status sks_solve(const float *pts, float *H, uint8_t *flags, int64_t n, int64_t ld, int32_t norm,
                     void *stream);

/*
 * aca_rect_solve - ACA for a rectangle source (Sec. 5.3, Eq. 39-42 and
 * Algorithm 1): source M1 = (x0, y0) upper-left corner, N1 upper-right,
 * Q1 lower-right, P1 lower-left, width w, aspect ratio r = width / height.
 *   tgt [8][ld] float: target corners M2 N2 P2 Q2 as x, y planes.
 *   H   [9][ld] float: Eq. 42's H (unnormalised; equal up to scale to the
 *       general aca_solve on the same corners).
 */
aca_status aca_rect_solve(const float *tgt, float x0, float y0, float w, float r, float *H, int64_t n,
                          int64_t ld, void *stream);

/*
 * aca_affine_solve - batched affine map from three correspondences by the
 * affine-decomposition of Sec. 5.2 (Eq. 38): H_A = H_A2^-1 H_A1, the ACA
 * chain with the identity core.
 *   pts [12][ld] float: M1 N1 P1 (source) then M2 N2 P2 (target), x/y planes.
 *   H   [9][ld] float: row-major; with ACA_NORM_NONE the division-free form
 *       with third row (0, 0, f_A1), f_A1 = M1N1 x M1P1; ACA_NORM_H33 gives
 *       the usual affine matrix with third row (0, 0, 1).  A collinear
 *       anchor triple gives f_A1 = 0 (singular map, non-finite with H33).
 */
aca_status aca_affine_solve(const float *pts, float *H, int64_t n, int64_t ld, int32_t norm, void *stream);

/*
 * aca_backward - vector-Jacobian product of the unnormalised ACA H
 * (aca_solve with ACA_NORM_NONE, Eq. 24-29) with respect to the 8 target
 * coordinates, the source points held fixed.  ACA uses only +, -, * (the
 * paper notes it is naturally differentiable, Sec. 5.3), so H is a
 * polynomial of degree 3 in the target coordinates and the derivative is
 * exact up to rounding.
 *   pts      [16][ld] float: the sets of the forward call.
 *   grad_H   [9][ld] float: dL/dH.
 *   grad_tgt [8][ld] float: output dL/d(M2.x, M2.y, N2.x, N2.y, P2.x, P2.y,
 *            Q2.x, Q2.y).
 */
aca_status aca_backward(const float *pts, const float *grad_H, float *grad_tgt, int64_t n, int64_t ld,
                        void *stream);

/*
 * aca_rect_backward - the same product for aca_rect_solve's H (Eq. 42).
 *   tgt [8][ld], grad_H [9][ld] in; grad_tgt [8][ld] out.
 */
aca_status aca_rect_backward(const float *tgt, float x0, float y0, float w, float r, const float *grad_H,
                             float *grad_tgt, int64_t n, int64_t ld, void *stream);

/*
 * RANSAC with ACA hypotheses (Sec. 2.2 and Sec. 6.2: sample 4 -> solve ->
 * verify -> keep the best), many problems in one launch.
 *
 *   corr      [total][4] float: correspondences (x1, y1, x2, y2), the points of
 *             problem p at rows offsets[p] .. offsets[p+1]-1; 16-byte aligned.
 *   offsets   [P+1] int64, offsets[0] = 0, non-decreasing (device memory).
 *   n_hyp     [P] int32 >= 0: hypotheses for problem p (device memory).
 *   P         number of problems (>= 0).
 *   params    thresholds, seed and launch tuning (see aca_ransac_params).
 *   best_H    [P][9] float: best hypothesis, unit Frobenius norm, sign fixed
 *             as ACA_NORM_FROB; zeros when the problem has no valid sample.
 *   best_count[P] int32: its inlier count (0 when none).
 *   best_hyp  [P] int32: its hypothesis index in 0..n_hyp[p]-1, or -1 when
 *             every sample was degenerate or n_hyp[p] = 0 or fewer than 4 points.
 *   hyp_counts[sum n_hyp] int32 or NULL: every hypothesis's inlier count,
 *             problem after problem; -1 for a degenerate sample.
 *   inlier_mask[total] uint8 or NULL: 1 for the inliers of the best hypothesis.
 *   workspace device memory of at least ransac_aca_workspace_size(P, sum n_hyp)
 *             bytes, 256-byte aligned.  With P <= 8 its first 256 bytes must
 *             be zero before the first call on it (e.g. cudaMemset once at
 *             allocation); every call leaves them zero.  Otherwise its
 *             contents need not be initialised.
 *
 * Work decomposition, P > 8: the (problem, block of 32*hyps_per_thread
 * hypotheses, slice of tile_points correspondences) items of all problems
 * are pulled by a persistent grid from one atomic counter; every item
 * samples and solves its hypotheses in registers (Philox + ACA), stages its
 * correspondence slice in shared memory and scores every hypothesis against
 * it; per-slice counts are summed with one atomic add per hypothesis; a last
 * kernel takes the argmax per problem, re-solves the winner and writes the
 * outputs.  P <= 8 (e.g. one image pair): everything in one launch; the
 * items (problem, block of hypotheses, one of 4 point ranges) are striped
 * over the resident blocks, each writes its partial counts to the slot of
 * its point range (and its hypotheses' H), and the last block to finish
 * sums them, takes the argmax and writes the outputs from the winner's
 * stored H.  Both give the same results bit for bit.
 *
 * Sampling: hypothesis h of problem p draws Philox4x32-10 (Salmon et al.,
 * SC'11) with counter (h, problem_base + p, 0, 0) and key (seed low 32 bits,
 * seed high 32 bits); the four 32-bit outputs u_k give ranks
 * j_k = floor(u_k (N - k) / 2^32) among the indices not drawn yet, which are
 * turned into distinct indices M, N, P, Q (k = 0..3) by stepping over the
 * earlier draws in ascending order.  The results do not depend on P, the
 * other problems or the launch tuning.
 * A sample is degenerate (scores -1) if, on either side, one of its triples
 * (M,N,P), (M,Q,P), (M,N,Q), (N,P,Q) has |cross(a, b)| <= 1e-3 |a| |b| for
 * its two edge vectors a, b.
 * Inlier test: with (u, v, w) = H (x1, y1, 1), a point is an inlier when
 * (u - x2 w)^2 + (v - y2 w)^2 - thr^2 w^2 < 0 in FP32 (H scaled by an exact
 * power of two), i.e. the forward transfer error ||x2 - (u/w, v/w)|| < thr
 * without a division; points exactly at the threshold are within rounding of
 * either outcome.  Best: highest count, ties to the lowest hypothesis index.
 */
typedef struct {
    float threshold_px;      /* inlier threshold in pixels (> 0) */
    uint32_t problem_base;   /* added to the problem index in the Philox counter */
    uint64_t seed;           /* Philox key */
    int32_t block_warps;     /* warps per block, 0 = default (8); 1..16 */
    int32_t hyps_per_thread; /* hypotheses per thread, 0 = default (2); 1, 2 or 4 */
    int32_t grid_blocks;     /* resident blocks of the persistent kernel, 0 = SMs x occupancy */
    int32_t tile_points;     /* correspondences per work item (P > 8) or per shared-memory
                                tile of a point range (P <= 8), staged in shared memory;
                                0 = default (1024); a multiple of 32, 32..8192 */
} aca_ransac_params;

/* Workspace bytes ransac_aca needs for P problems with total_hyps =
 * sum of n_hyp hypotheses (per-problem offsets plus one int32 count per
 * hypothesis; with P <= 8, four partial counts and the 9 entries of H per
 * hypothesis).  If the device-side sum of n_hyp exceeds what the workspace
 * holds, nothing is scored and every best_hyp is -2. */
size_t ransac_aca_workspace_size(int32_t P, int64_t total_hyps);

aca_status ransac_aca(const float *corr, const int64_t *offsets, const int32_t *n_hyp, int32_t P,
                      const aca_ransac_params *params, float *best_H, int32_t *best_count, int32_t *best_hyp,
                      int32_t *hyp_counts, uint8_t *inlier_mask, void *workspace, size_t workspace_bytes,
                      void *stream);

/*
 * ransac_aca_noalloc - ransac_aca without a caller workspace and without any
 * device allocation, for callers that may not allocate device memory: for
 * example a plugin whose host framework owns all device memory through its
 * own allocator, a latency-critical loop in which an allocation (which can
 * synchronise the device) is not allowed, or a service whose device-memory
 * budget is fixed at start-up.  The paper has no counterpart; this is a
 * deployment variant of the RANSAC call above.
 *
 * The scratch is a fixed array of ACA_NOALLOC_SCRATCH_BYTES inside the
 * library's device image, held by every GPU that loads the library until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress, with the device current) and caches it.
 * Under lazy module loading (the CUDA runtime's default) that lookup is also
 * what loads the module and reserves the array on the device, so the first
 * call on each device may allocate: make it once as a warm-up, outside any
 * region that must not allocate and before any stream capture (or set
 * CUDA_MODULE_LOADING=EAGER).  All calls share the array and
 * each call re-initialises it, so calls whose kernels may overlap on the GPU
 * race and must be serialised by the caller.
 *
 *   total_hyps must equal sum(n_hyp); a request that needs more than
 *   ACA_NOALLOC_SCRATCH_BYTES (ransac_aca_workspace_size(P, total_hyps))
 *   is rejected with ACA_ERR_WORKSPACE before anything is launched.  The
 *   count capacity is exactly total_hyps: if the device-side sum of n_hyp
 *   exceeds it, nothing is scored and every best_hyp is -2, as with a
 *   ransac_aca workspace of that size.  Other arguments, outputs and results
 *   are those of ransac_aca.
 */
#define ACA_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)
aca_status ransac_aca_noalloc(const float *corr, const int64_t *offsets, const int32_t *n_hyp, int32_t P,
                              int64_t total_hyps, const aca_ransac_params *params, float *best_H,
                              int32_t *best_count, int32_t *best_hyp, int32_t *hyp_counts, uint8_t *inlier_mask,
                              void *stream);

/*
 * aca_sample_indices - the minimal-set indices ransac_aca draws: for
 * h = 0..n_hyp-1, idx[h][0..3] = the distinct indices (M, N, P, Q) in [0, N)
 * of hypothesis h of problem `problem` (the Philox counter's second word,
 * i.e. problem_base + p) under `seed`.  Requires 4 <= N < 2^31.
 *   idx [n_hyp][4] int32 device memory.
 */
aca_status aca_sample_indices(int64_t N, int32_t n_hyp, uint64_t seed, uint32_t problem, int32_t *idx,
                              void *stream);

/*
 * ransac_aca_adaptive - ransac_aca with the online adaptive stop of the
 * paper's RANSAC loop (Sec. 6.2: the number of loops follows from the inlier
 * ratio, at a confidence that one 4-point sample is all inliers, with a cap).
 * For problem p the loop over hypotheses h = 0, 1, ... stops before h when
 *     h >= K(best count among hypotheses 0..h-1),
 *     K(c) = ceil(log(1 - confidence) / log(1 - (c / N)^4)), clamped to
 *            [1, max_hyp[p]] (c <= 0: max_hyp[p]),
 * or after max_hyp[p] hypotheses.  The result is that of this sequential loop
 * exactly: hypotheses are sampled, solved and scored as in ransac_aca (same
 * Philox streams, same counts), the best is the argmax over the evaluated
 * hypotheses (ties to the lowest index).  On the GPU, work on hypotheses the
 * loop is certain not to reach is skipped; which of them were scored does
 * not change any output.
 *   max_hyp    [P] int32 >= 0: the cap per problem (device memory).
 *   total_max_hyps  sum of max_hyp (sizes the workspace).
 *   confidence in (0, 1), e.g. 0.99.
 *   n_evaluated[P] int32 or NULL: the number of hypotheses the loop evaluated
 *              (0 when the problem has fewer than 4 points or max_hyp[p] = 0).
 *   hyp_counts [total_max_hyps] int32 or NULL: counts of the evaluated
 *              hypotheses (-1 degenerate), -2 for the ones after the stop.
 *   workspace  at least ransac_aca_adaptive_workspace_size(P, total_max_hyps)
 *              bytes, 256-byte aligned.
 * Other arguments, outputs and errors as ransac_aca; confidence outside
 * (0, 1) is ACA_ERR_INVALID_ARG.  Work order: the first hypothesis block of
 * every problem, then, re-planned from the bounds that block set, the blocks
 * still before each problem's bound, taken in rounds (round r = block r of
 * every problem that has one), so that a problem's earlier blocks finish
 * while its later ones wait.
 */
size_t ransac_aca_adaptive_workspace_size(int32_t P, int64_t total_max_hyps);

aca_status ransac_aca_adaptive(const float *corr, const int64_t *offsets, const int32_t *max_hyp, int32_t P,
                               int64_t total_max_hyps, const aca_ransac_params *params, double confidence,
                               float *best_H, int32_t *best_count, int32_t *best_hyp, int32_t *n_evaluated,
                               int32_t *hyp_counts, uint8_t *inlier_mask, void *workspace, size_t workspace_bytes,
                               void *stream);

/*
 * aca_refit - re-estimate one homography per problem from ALL of its masked
 * correspondences: the global optimisation with all inliers that follows
 * the RANSAC loop (Sec. 6.2, stage 5, where it is a Levenberg-Marquardt
 * minimisation).  Per problem:
 *   1. Hartley normalisation of each image (centroid to the origin, mean
 *      distance sqrt(2));
 *   2. the normalised DLT: h minimises the algebraic residual of the two
 *      Eq. 2 rows of every point under |h| = 1 (smallest eigenvector of the
 *      9x9 normal matrix: FP32 inverse iteration as the start of step 3;
 *      refined to double-float accuracy when it is the result, lm_iters = 0);
 *   3. lm_iters trial steps of Levenberg-Marquardt on the reprojection error
 *      sum_i |pi(H x1_i) - x2_i|^2 (eight entries with h33 = 1 in the
 *      normalised frames; damping of Madsen, Nielsen & Tingleff 2004,
 *      Alg. 3.16, mu0 = 1e-6 max diag(J^T J), 1e-3 max diag after a
 *      rejected first trial), stopping early once a step is below FP32 resolution, or
 *      after two accepted steps that each moved the parameters by less than
 *      2^-20 and predicted a decrease below the cost's FP32 noise.
 *      It is skipped when the normalised DLT has |h33| < 1e-3.
 *   corr     [total][4] float (x1, y1, x2, y2), the points of problem p at rows
 *            offsets[p] .. offsets[p+1]-1; 16-byte aligned (device memory).
 *   offsets  [P+1] int64, offsets[0] = 0, non-decreasing (device memory).
 *   mask     [total] uint8 or NULL: nonzero = use the point (e.g. the
 *            inlier_mask of ransac_aca); NULL uses every point.
 *   lm_iters 0..10000 trial steps (0: the normalised DLT only).
 *   H        [P][9] float out: row-major, unit Frobenius norm, h33 > 0 (or the
 *            largest entry > 0 when |h33| < 1e-6); all zeros for a problem
 *            with fewer than 4 used points.
 *   n_used   [P] int32 out or NULL: number of used points.
 *   rms      [P] float out or NULL: RMS reprojection error in pixels of the
 *            returned H over the used points (-1 when step 3 was skipped).
 * One block per problem, all buffers caller-owned, nothing allocated.
 * Points in general position are assumed: with all used points collinear
 * the minimiser is not unique and H is one of them.  Returns
 * ACA_ERR_INVALID_ARG for P < 0, lm_iters outside its range, a null or
 * misaligned buffer; ACA_ERR_CUDA if the launch fails.
 */
aca_status aca_refit(const float *corr, const int64_t *offsets, const uint8_t *mask, int32_t P, int32_t lm_iters,
                     float *H, int32_t *n_used, float *rms, void *stream);

/*
 * FP32 FMA throughput probe (a diagnostic, not part of the method): `blocks`
 * blocks of `threads` threads each run 8 independent FMA chains of `steps`
 * steps, as scalar FMAs (packed = 0) or as packed f32x2 FMAs (packed != 0),
 * and write one float per thread to `sink` (blocks * threads floats, device,
 * caller-owned).  Timing it gives the measured FP32 rate that the FP32-pipe
 * rooflines (Sec. 6.2's verification loop on the GPU) are stated against,
 * beside the rate derived from the SM count and the clock.
 * aca_fma_probe_flops returns the FLOPs of one launch (an FMA counts 2).
 * Returns ACA_ERR_INVALID_ARG for blocks < 1, threads not a multiple of 32
 * in 32..1024, steps not a positive multiple of 16, or a null sink.
 */
aca_status aca_fma_probe(int32_t packed, int32_t blocks, int32_t threads, int32_t steps, float *sink, void *stream);
int64_t aca_fma_probe_flops(int32_t packed, int32_t blocks, int32_t threads, int32_t steps);

/* Message describing the last non-OK status returned on this thread. */
const char *aca_last_error(void);

/* Library version string. */
const char *aca_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ACA_GB300_H */
