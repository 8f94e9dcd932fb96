// Batched minimal solvers: aca_solve (Sec. 4), sks_solve (Sec. 3) and
// aca_rect_solve (Sec. 5.3), one set per thread lane in registers.
//
// The work is a pure stream (64 B in, 36 B out per set, ~365 FP32
// instructions), bound by HBM bandwidth with the ALU close behind: each thread
// takes four adjacent sets as one float4 from each of the 16 SoA planes,
// solves them one after another in registers and writes nine float4 planes
// with streaming (evict-first) stores.  A persistent grid strides over the
// quads; each thread copies its next quad's 16 float4 into its own slots of a
// two-stage shared-memory ring (cp.async) while it solves the current one, so
// the loads of the next step are in flight during the arithmetic (ACA, and
// SKS without flags, which runs two sets per packed f32x2 instruction; the
// flagged SKS loads directly).  When the layout does not allow 16-byte
// accesses a scalar variant (one set per thread, coalesced 4-byte accesses)
// runs instead.
//
// Every kernel here is launched as a programmatic dependent of its stream
// predecessor and waits for it at entry (grid_dependency_wait), so its launch
// overlaps the predecessor's last blocks.  None triggers its own successor
// early: the successor is scheduled as this grid's blocks exit.  With the
// trigger at entry the successor's blocks sat resident beside the running
// grid, and calls of 2e4 to 1e6 sets took 10-40 % longer; without it, a
// 100-call graph of 1-set calls takes 1.15 us a call (1.3-1.5 without PDL),
// and the rectangle forward + backward pair on 65536 sets 3.3 us (4.1).
#include "aca_math.cuh"
#include "common.cuh"
#include "pdl.cuh"

namespace aca {

enum Solver { kAca = 0, kSks = 1 };

// With FINITE = false the flags leave out bit 8 (non-finite), which the
// caller then decides for several sets at once (solve_quad).
template <int SOLVER, int NORM, bool FLAGS, bool FINITE = true>
__device__ __forceinline__ void solve_one(const Set &s, float H[9], uint8_t &flag)
{
    if (SOLVER == kAca) {
        AcaParts p;
        aca_parts(s, p);
        aca_compose(s, p, NORM != ACA_NORM_NONE, H);
        if (NORM == ACA_NORM_H33) normalize_h33(H);
        if (NORM == ACA_NORM_FROB) normalize_frob(H);
        if (FLAGS) flag = FINITE ? aca_flags(s, p, H) : aca_geom_flags(s, p);
    } else {
        sks_solve(s, H);
        if (NORM == ACA_NORM_H33) normalize_h33(H);
        if (NORM == ACA_NORM_FROB) normalize_frob(H);
        if (FLAGS) {
            AcaParts p;
            aca_parts(s, p);
            flag = FINITE ? aca_flags(s, p, H) : aca_geom_flags(s, p);
        }
    }
}

// SKS on two sets at once, as packed pairs (fp32.cuh); the optional
// normalisation, which compares and divides, finishes per lane in scalar
// code, as in solve_one.
template <int NORM>
__device__ __forceinline__ void sks_solve_two(const SetT<P2> &s, P2 H[9])
{
    sks_solve(s, H);
    if (NORM != ACA_NORM_NONE) {
#pragma unroll
        for (int lane = 0; lane < 2; ++lane) {
            float h[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) h[k] = lane ? vhi(H[k]) : vlo(H[k]);
            if (NORM == ACA_NORM_H33) normalize_h33(h);
            if (NORM == ACA_NORM_FROB) normalize_frob(h);
#pragma unroll
            for (int k = 0; k < 9; ++k) H[k] = lane ? vpack(vlo(H[k]), h[k]) : vpack(h[k], vhi(H[k]));
        }
    }
}

// Four adjacent sets (one float4 from each input plane); nine float4 planes
// stored with streaming stores, element-wise on the last, partial quad.
// SKS without flags solves them as two packed pairs (sets 0-1 from the .x/.y
// lanes, sets 2-3 from .z/.w): 43.0 against 40.5 G sets/s one by one.  The
// ACA solve sits at the HBM stream either way (packed it measured 1 % lower),
// and the flagged solves lose more to the per-lane finish and to 210-240
// registers than packing saves (44.7 against 55.1 G sets/s), so they take
// the sets one by one.  Both forms give the same bits (fp32.cuh).
template <int SOLVER, int NORM, bool FLAGS>
__device__ __forceinline__ void solve_quad(const float4 (&v)[16], int64_t q, float *__restrict__ Hout,
                                           uint8_t *__restrict__ flags, int64_t n, int64_t ld)
{
    float4 h[9];
    uint32_t fl = 0;
    if constexpr (SOLVER == kSks && !FLAGS) {
#pragma unroll
        for (int jp = 0; jp < 2; ++jp) {
            SetT<P2> s;
            P2 *sv = &s.M1x;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                sv[k] = jp ? vpack(v[k].z, v[k].w) : vpack(v[k].x, v[k].y);
            P2 H[9];
            sks_solve_two<NORM>(s, H);
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                if (jp) vunpack(H[k], h[k].z, h[k].w);
                else vunpack(H[k], h[k].x, h[k].y);
            }
        }
    } else {
        // bit 8 (non-finite) of the four sets at once, in aca_flags' test
        // x * 0 + z, on packed pairs (sets 0-1 in the .x/.y lanes, 2-3 in
        // .z/.w) at half the instructions: the inputs first, the outputs below
        const P2 zero = vpack(0.0f, 0.0f);
        P2 z01 = zero, z23 = zero;
        if (FLAGS) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                z01 = vfma(vpack(v[k].x, v[k].y), zero, z01);
                z23 = vfma(vpack(v[k].z, v[k].w), zero, z23);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            Set s;
            float *sv = &s.M1x;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                sv[k] = (&v[k].x)[j];
            float H[9];
            uint8_t f = 0;
            solve_one<SOLVER, NORM, FLAGS, false>(s, H, f);
#pragma unroll
            for (int k = 0; k < 9; ++k)
                (&h[k].x)[j] = H[k];
            fl |= (uint32_t)f << (8 * j);
        }
        if (FLAGS) {
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                z01 = vfma(vpack(h[k].x, h[k].y), zero, z01);
                z23 = vfma(vpack(h[k].z, h[k].w), zero, z23);
            }
            float z[4];
            vunpack(z01, z[0], z[1]);
            vunpack(z23, z[2], z[3]);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (!(z[j] == 0.0f)) fl |= (uint32_t)kFlagNonFinite << (8 * j);
        }
    }
    const int64_t i0 = q << 2;
    if (i0 + 3 < n) {
        float4 *out = reinterpret_cast<float4 *>(Hout);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            st_stream(out + k * (ld >> 2) + q, h[k]);
        if (FLAGS)
            reinterpret_cast<uint32_t *>(flags)[q] = fl;
    } else {
        for (int j = 0; j < 4 && i0 + j < n; ++j) {
#pragma unroll
            for (int k = 0; k < 9; ++k)
                Hout[k * ld + i0 + j] = (&h[k].x)[j];
            if (FLAGS)
                flags[i0 + j] = (uint8_t)(fl >> (8 * j));
        }
    }
}

// Direct loads: 16 streaming float4 loads per quad, then the solves.
template <int SOLVER, int NORM, bool FLAGS>
__global__ void __launch_bounds__(256) solve_vec4_kernel(const float *__restrict__ pts, float *__restrict__ Hout,
                                                          uint8_t *__restrict__ flags, int64_t n, int64_t ld)
{
    grid_dependency_wait();
    const int64_t nq = (n + 3) >> 2;
    const int64_t ldq = ld >> 2;
    const float4 *in = reinterpret_cast<const float4 *>(pts);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        float4 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k)
            v[k] = ld_stream(in + k * ldq + q);
        solve_quad<SOLVER, NORM, FLAGS>(v, q, Hout, flags, n, ld);
    }
}

// 16-byte asynchronous copy global -> shared, cached in L2 only, and the
// group fences of the issuing thread.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Prefetching stream over quads: each thread copies its next quad's PLANES
// float4 into its own slots of a two-stage shared-memory ring while it
// solves the current quad, so the next loads are in flight during the
// arithmetic.  128 threads, 2 blocks per SM (2 x 128 beat 3 x 128, 4 x 128
// and 1 x 256 in a sweep of the ACA solve).
constexpr int kRingThreads = 128;
constexpr int kRingBlocksPerSm = 2;
template <int PLANES>
constexpr size_t ring_smem() { return 2 * PLANES * kRingThreads * sizeof(float4); }

template <int PLANES, typename QuadFn>
__device__ __forceinline__ void ring_stream(const float *__restrict__ pts, int64_t n, int64_t ld, QuadFn &&solve)
{
    extern __shared__ float4 ring[];   // [2 stages][PLANES][kRingThreads]
    const int64_t nq = (n + 3) >> 2;
    const int64_t ldq = ld >> 2;
    const float4 *in = reinterpret_cast<const float4 *>(pts);
    const int64_t stride = (int64_t)gridDim.x * kRingThreads;
    const int t = threadIdx.x;
    // a thread only ever reads the slots it filled itself, so its own
    // cp.async.wait_group is the only synchronisation needed
    auto fetch = [&](int64_t q, int stage) {
#pragma unroll
        for (int k = 0; k < PLANES; ++k) cp_async16(&ring[(stage * PLANES + k) * kRingThreads + t], in + k * ldq + q);
        cp_async_commit();
    };
    int64_t q = (int64_t)blockIdx.x * kRingThreads + t;
    int stage = 0;
    if (q < nq) fetch(q, 0);
    for (; q < nq; q += stride) {
        const int64_t qn = q + stride;
        if (qn < nq) {
            fetch(qn, stage ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        float4 v[PLANES];
#pragma unroll
        for (int k = 0; k < PLANES; ++k) v[k] = ring[(stage * PLANES + k) * kRingThreads + t];
        solve(v, q);
        stage ^= 1;
    }
}

// Launch of a ring kernel: opt in to its dynamic shared memory (a function
// attribute of the current device, set on every call: well under a
// microsecond against >= 8 us of work on this path), persistent grid.
template <int PLANES, int BLOCKS_PER_SM = kRingBlocksPerSm, typename K, typename... Args>
static aca_status launch_ring(K kernel, const char *name, int64_t n, cudaStream_t st, Args... args)
{
    const size_t smem = ring_smem<PLANES>();
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return set_error(ACA_ERR_CUDA, "%s: cannot reserve %zu bytes of shared memory", name, smem);
    const int64_t need = ((n + 3) / 4 + kRingThreads - 1) / kRingThreads;
    int64_t grid = (int64_t)sm_count() * BLOCKS_PER_SM;
    if (grid > need) grid = need;
    launch_after_previous(kernel, dim3((int)grid), dim3(kRingThreads), smem, st, args...);
    return ACA_OK;
}

template <int SOLVER, int NORM, bool FLAGS>
__global__ void __launch_bounds__(kRingThreads) solve_ring_kernel(const float *__restrict__ pts,
                                                                  float *__restrict__ Hout,
                                                                  uint8_t *__restrict__ flags, int64_t n, int64_t ld)
{
    grid_dependency_wait();
    ring_stream<16>(pts, n, ld, [&](const float4 (&v)[16], int64_t q) {
        solve_quad<SOLVER, NORM, FLAGS>(v, q, Hout, flags, n, ld);
    });
}

template <int SOLVER, int NORM, bool FLAGS>
__global__ void __launch_bounds__(256) solve_scalar_kernel(const float *__restrict__ pts, float *__restrict__ Hout,
                                                            uint8_t *__restrict__ flags, int64_t n, int64_t ld)
{
    grid_dependency_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Set s;
        float *sv = &s.M1x;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            sv[k] = ld_stream(pts + k * ld + i);
        float H[9];
        uint8_t f = 0;
        solve_one<SOLVER, NORM, FLAGS>(s, H, f);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            st_stream(Hout + k * ld + i, H[k]);
        if (FLAGS)
            flags[i] = f;
    }
}

template <int SOLVER, int NORM, bool FLAGS>
static aca_status launch_solve(const float *pts, float *H, uint8_t *flags, int64_t n, int64_t ld, cudaStream_t st)
{
    const int threads = 256;
    const bool vec = n >= kSmallBatch && (ld % 4 == 0) && aligned16(pts) && aligned16(H) &&
                     (!FLAGS || (reinterpret_cast<uintptr_t>(flags) & 3u) == 0);
    // The ACA solve (~365 instructions a set) sits at the HBM stream:
    // prefetching pays (0.95 -> 0.98 of copy bandwidth) at 2 blocks of 128
    // threads per SM.  With the flags (~490 instructions) the arithmetic
    // leads and a third block per SM pays (58.8 against 55.1 G sets/s with
    // direct loads).  SKS without flags, division-free and packed, runs best
    // on a ring grid of 4 blocks per SM, 3 resident (2^26 sets: 60.3 G sets/s
    // against 59.8 at 3; first measured 46.98 against 46.48 at 3, 45.26 at
    // 2 and 45.55 with direct loads); with flags it takes its sets one by
    // one on direct loads.
    constexpr bool kRing = SOLVER == kAca || !FLAGS;
    constexpr int kRingBlocks = SOLVER == kSks ? 4 : (FLAGS ? 3 : kRingBlocksPerSm);
    if (kRing && vec) {
        if constexpr (kRing) {
            const aca_status r = launch_ring<16, kRingBlocks>(solve_ring_kernel<SOLVER, NORM, FLAGS>,
                                                              SOLVER == kAca ? "aca_solve" : "sks_solve", n, st, pts,
                                                              H, flags, n, ld);
            if (r != ACA_OK)
                return r;
        }
    } else if (vec) {
        auto k = solve_vec4_kernel<SOLVER, NORM, FLAGS>;
        const int64_t nq = (n + 3) / 4;
        const int grid = resident_grid(k, threads, 0, (nq + threads - 1) / threads);
        launch_after_previous(k, dim3(grid), dim3(threads), 0, st, pts, H, flags, n, ld);
    } else {
        auto k = solve_scalar_kernel<SOLVER, NORM, FLAGS>;
        const int grid = resident_grid(k, threads, 0, (n + threads - 1) / threads);
        launch_after_previous(k, dim3(grid), dim3(threads), 0, st, pts, H, flags, n, ld);
    }
    return check_launch(SOLVER == kAca ? "aca_solve" : "sks_solve");
}

template <int SOLVER>
static aca_status dispatch_solve(const float *pts, float *H, uint8_t *flags, int64_t n, int64_t ld, int32_t norm,
                                 void *stream)
{
    const char *name = SOLVER == kAca ? "aca_solve" : "sks_solve";
    if (n < 0 || ld < n)
        return set_error(ACA_ERR_INVALID_ARG, "%s: need 0 <= n <= ld (n=%lld, ld=%lld)", name, (long long)n,
                         (long long)ld);
    if (norm < ACA_NORM_NONE || norm > ACA_NORM_FROB)
        return set_error(ACA_ERR_INVALID_ARG, "%s: unknown norm %d", name, norm);
    if (n == 0)
        return ACA_OK;
    if (!pts || !H)
        return set_error(ACA_ERR_INVALID_ARG, "%s: null pts or H", name);
    if (ld > (INT64_MAX / 16))
        return set_error(ACA_ERR_INVALID_ARG, "%s: ld too large", name);
    const cudaStream_t st = as_stream(stream);
#define ACA_CASE(NRM)                                                                              \
    if (norm == NRM)                                                                               \
        return flags ? launch_solve<SOLVER, NRM, true>(pts, H, flags, n, ld, st)                   \
                     : launch_solve<SOLVER, NRM, false>(pts, H, flags, n, ld, st);
    ACA_CASE(ACA_NORM_NONE)
    ACA_CASE(ACA_NORM_H33)
    ACA_CASE(ACA_NORM_FROB)
#undef ACA_CASE
    return ACA_ERR_INVALID_ARG;
}

// --------------------------------------------------------------------------
// Rectangle source (Eq. 42): 8 target planes in, 9 planes out.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) rect_vec4_kernel(const float *__restrict__ tgt, Rect R, float *__restrict__ Hout,
                                                         int64_t n, int64_t ld)
{
    grid_dependency_wait();
    const int64_t nq = (n + 3) >> 2, ldq = ld >> 2;
    const float4 *in = reinterpret_cast<const float4 *>(tgt);
    float4 *out = reinterpret_cast<float4 *>(Hout);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        float4 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            v[k] = ld_stream(in + k * ldq + q);
        float4 h[9];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float t[8], H[9];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                t[k] = (&v[k].x)[j];
            rect_solve(t, R, H);
#pragma unroll
            for (int k = 0; k < 9; ++k)
                (&h[k].x)[j] = H[k];
        }
        const int64_t i0 = q << 2;
        if (i0 + 3 < n) {
#pragma unroll
            for (int k = 0; k < 9; ++k)
                st_stream(out + k * ldq + q, h[k]);
        } else {
            for (int j = 0; j < 4 && i0 + j < n; ++j)
#pragma unroll
                for (int k = 0; k < 9; ++k)
                    Hout[k * ld + i0 + j] = (&h[k].x)[j];
        }
    }
}

__global__ void __launch_bounds__(256) rect_scalar_kernel(const float *__restrict__ tgt, Rect R,
                                                           float *__restrict__ Hout, int64_t n, int64_t ld)
{
    grid_dependency_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float t[8], H[9];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            t[k] = ld_stream(tgt + k * ld + i);
        rect_solve(t, R, H);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            st_stream(Hout + k * ld + i, H[k]);
    }
}

// --------------------------------------------------------------------------
// Affine map from three correspondences (Eq. 38): 12 planes in, 9 out.
// --------------------------------------------------------------------------
template <int NORM>
__device__ __forceinline__ void affine_one(const Set3 &s, float H[9])
{
    affine_solve(s, H);
    if (NORM == ACA_NORM_H33) normalize_h33(H);
    if (NORM == ACA_NORM_FROB) normalize_frob(H);
}

template <int NORM>
__device__ __forceinline__ void affine_quad(const float4 (&v)[12], int64_t q, float *__restrict__ Hout, int64_t n,
                                            int64_t ld)
{
    float4 h[9];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        Set3 s;
        float *sv = &s.M1x;
#pragma unroll
        for (int k = 0; k < 12; ++k)
            sv[k] = (&v[k].x)[j];
        float H[9];
        affine_one<NORM>(s, H);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            (&h[k].x)[j] = H[k];
    }
    const int64_t i0 = q << 2;
    if (i0 + 3 < n) {
        float4 *out = reinterpret_cast<float4 *>(Hout);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            st_stream(out + k * (ld >> 2) + q, h[k]);
    } else {
        for (int j = 0; j < 4 && i0 + j < n; ++j)
#pragma unroll
            for (int k = 0; k < 9; ++k)
                Hout[k * ld + i0 + j] = (&h[k].x)[j];
    }
}

template <int NORM>
__global__ void __launch_bounds__(kRingThreads) affine_ring_kernel(const float *__restrict__ pts,
                                                                   float *__restrict__ Hout, int64_t n, int64_t ld)
{
    grid_dependency_wait();
    ring_stream<12>(pts, n, ld, [&](const float4 (&v)[12], int64_t q) { affine_quad<NORM>(v, q, Hout, n, ld); });
}

template <int NORM>
__global__ void __launch_bounds__(256) affine_scalar_kernel(const float *__restrict__ pts, float *__restrict__ Hout,
                                                             int64_t n, int64_t ld)
{
    grid_dependency_wait();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Set3 s;
        float *sv = &s.M1x;
#pragma unroll
        for (int k = 0; k < 12; ++k)
            sv[k] = ld_stream(pts + k * ld + i);
        float H[9];
        affine_one<NORM>(s, H);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            st_stream(Hout + k * ld + i, H[k]);
    }
}

template <int NORM>
static aca_status launch_affine(const float *pts, float *H, int64_t n, int64_t ld, cudaStream_t st)
{
    const int threads = 256;
    if (n >= kSmallBatch && ld % 4 == 0 && aligned16(pts) && aligned16(H)) {
        const aca_status r = launch_ring<12>(affine_ring_kernel<NORM>, "aca_affine_solve", n, st, pts, H, n, ld);
        if (r != ACA_OK)
            return r;
    } else {
        auto k = affine_scalar_kernel<NORM>;
        const int grid = resident_grid(k, threads, 0, (n + threads - 1) / threads);
        launch_after_previous(k, dim3(grid), dim3(threads), 0, st, pts, H, n, ld);
    }
    return check_launch("aca_affine_solve");
}

}  // namespace aca

using namespace aca;

extern "C" aca_status aca_affine_solve(const float *pts, float *H, int64_t n, int64_t ld, int32_t norm, void *stream)
{
    if (n < 0 || ld < n)
        return set_error(ACA_ERR_INVALID_ARG, "aca_affine_solve: need 0 <= n <= ld");
    if (norm < ACA_NORM_NONE || norm > ACA_NORM_FROB)
        return set_error(ACA_ERR_INVALID_ARG, "aca_affine_solve: unknown norm %d", norm);
    if (n == 0)
        return ACA_OK;
    if (!pts || !H)
        return set_error(ACA_ERR_INVALID_ARG, "aca_affine_solve: null pts or H");
    const cudaStream_t st = as_stream(stream);
    if (norm == ACA_NORM_NONE) return launch_affine<ACA_NORM_NONE>(pts, H, n, ld, st);
    if (norm == ACA_NORM_H33) return launch_affine<ACA_NORM_H33>(pts, H, n, ld, st);
    return launch_affine<ACA_NORM_FROB>(pts, H, n, ld, st);
}

extern "C" aca_status aca_solve(const float *pts, float *H, uint8_t *flags, int64_t n, int64_t ld, int32_t norm,
                                void *stream)
{
    return dispatch_solve<kAca>(pts, H, flags, n, ld, norm, stream);
}

extern "C" aca_status sks_solve(const float *pts, float *H, uint8_t *flags, int64_t n, int64_t ld, int32_t norm,
                                void *stream)
{
    return dispatch_solve<kSks>(pts, H, flags, n, ld, norm, stream);
}

extern "C" aca_status aca_rect_solve(const float *tgt, float x0, float y0, float w, float r, float *H, int64_t n,
                                     int64_t ld, void *stream)
{
    if (n < 0 || ld < n)
        return set_error(ACA_ERR_INVALID_ARG, "aca_rect_solve: need 0 <= n <= ld");
    if (!(w > 0) || !(r > 0))
        return set_error(ACA_ERR_INVALID_ARG, "aca_rect_solve: width and aspect ratio must be > 0");
    if (n == 0)
        return ACA_OK;
    if (!tgt || !H)
        return set_error(ACA_ERR_INVALID_ARG, "aca_rect_solve: null tgt or H");
    const Rect R{x0, y0, w, r};
    const cudaStream_t st = as_stream(stream);
    const int threads = 256;
    if (n >= kSmallBatch && ld % 4 == 0 && aligned16(tgt) && aligned16(H)) {
        const int grid = resident_grid(rect_vec4_kernel, threads, 0, ((n + 3) / 4 + threads - 1) / threads);
        launch_after_previous(rect_vec4_kernel, dim3(grid), dim3(threads), 0, st, tgt, R, H, n, ld);
    } else {
        const int grid = resident_grid(rect_scalar_kernel, threads, 0, (n + threads - 1) / threads);
        launch_after_previous(rect_scalar_kernel, dim3(grid), dim3(threads), 0, st, tgt, R, H, n, ld);
    }
    return check_launch("aca_rect_solve");
}
