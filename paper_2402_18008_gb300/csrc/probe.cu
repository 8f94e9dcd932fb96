// FP32 FMA throughput probe: the measured denominator of the FP32-pipe
// rooflines (the RANSAC scoring kernels), beside the one derived from the SM
// count, the 128 FP32 lanes of an SM and the clock.  Each thread runs
// kChains independent FMA chains (enough independent work to cover the FMA
// latency at full occupancy), either as scalar FMAs or as packed f32x2 FMAs,
// the form the scoring kernels issue; the accumulators go to `sink` so that
// no chain is removed.  The operands keep the values bounded (a contraction
// towards a fixed point), so no input leads to overflow or denormals.
#include "common.cuh"

namespace aca {
namespace {

constexpr int kChains = 8;
constexpr int kUnrollSteps = 16;

__device__ __forceinline__ float2 fma2_probe(float2 a, float2 b, float2 c)
{
    float2 d;
    asm volatile("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
                 "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
                 : "=f"(d.x), "=f"(d.y)
                 : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

__global__ void fma_probe_scalar(int32_t steps, float a, float b, float *__restrict__ sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int32_t s = 0; s < steps; s += kUnrollSteps) {
#pragma unroll
        for (int u = 0; u < kUnrollSteps; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float t = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += x[c];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void fma_probe_packed(int32_t steps, float a, float b, float *__restrict__ sink)
{
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int32_t s = 0; s < steps; s += kUnrollSteps) {
#pragma unroll
        for (int u = 0; u < kUnrollSteps; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma2_probe(x[c], a2, b2);
    }
    float t = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += x[c].x + x[c].y;
    sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace
}  // namespace aca

extern "C" int64_t aca_fma_probe_flops(int32_t packed, int32_t blocks, int32_t threads, int32_t steps)
{
    return (int64_t)blocks * threads * steps * aca::kChains * 2 * (packed ? 2 : 1);
}

extern "C" aca_status aca_fma_probe(int32_t packed, int32_t blocks, int32_t threads, int32_t steps, float *sink,
                                    void *stream)
{
    using namespace aca;
    if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0)
        return set_error(ACA_ERR_INVALID_ARG, "aca_fma_probe: blocks >= 1 and threads a multiple of 32 in 32..1024");
    if (steps < kUnrollSteps || steps % kUnrollSteps != 0)
        return set_error(ACA_ERR_INVALID_ARG, "aca_fma_probe: steps must be a positive multiple of %d", kUnrollSteps);
    if (!sink) return set_error(ACA_ERR_INVALID_ARG, "aca_fma_probe: null sink");
    // x -> 0.5 x + 0.25 stays in (0, 1) for starts in [0, 1.1]
    if (packed)
        fma_probe_packed<<<blocks, threads, 0, as_stream(stream)>>>(steps, 0.5f, 0.25f, sink);
    else
        fma_probe_scalar<<<blocks, threads, 0, as_stream(stream)>>>(steps, 0.5f, 0.25f, sink);
    return check_launch("aca_fma_probe");
}
