// Host-side plumbing shared by the C-ABI entry points: status codes, the
// thread-local error message, cached device properties and launch helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <cstdarg>

#include "../../include/aca.h"

namespace aca {

aca_status set_error(aca_status st, const char *fmt, ...);

inline aca_status check_launch(const char *what)
{
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(ACA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return ACA_OK;
}

// SM count of the current device (queried once per device and cached).
int sm_count();

// 32-bit words per hypothesis that a ransac_aca workspace holds for P
// problems (on the one-launch path of small batches one count per point
// slice plus the hypothesis's 9 entries of H, else one count).
size_t ransac_count_slots(int32_t P);

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Below this many sets a stream kernel is latency-bound rather than
// bandwidth-bound: one set per thread (more blocks, a quarter of the serial
// work per thread) beats four sets per thread with 16-byte accesses.
constexpr int64_t kSmallBatch = int64_t(1) << 18;

// Streaming (evict-first) global accesses for data touched exactly once.
__device__ __forceinline__ float4 ld_stream(const float4 *p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(float4 *p, float4 v) { __stcs(p, v); }
__device__ __forceinline__ float ld_stream(const float *p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(float *p, float v) { __stcs(p, v); }

inline float4 *as_f4(float *p) { return reinterpret_cast<float4 *>(p); }
inline const float4 *as_f4(const float *p) { return reinterpret_cast<const float4 *>(p); }

// Resident blocks per SM of a kernel at a launch shape, on the current device
// (queried once per kernel, shape and device, then cached: the query costs
// microseconds, comparable to a small launch).
int blocks_per_sm(const void *kernel, int threads, size_t smem);

// Persistent-grid size: SMs x resident blocks of `kernel` at `threads`
// threads and `smem` dynamic bytes, capped by `work_blocks` (>= 1).
template <typename K>
int resident_grid(K kernel, int threads, size_t smem, int64_t work_blocks)
{
    const int per_sm = blocks_per_sm(reinterpret_cast<const void *>(kernel), threads, smem);
    int64_t g = (int64_t)per_sm * sm_count();
    if (work_blocks < g)
        g = work_blocks;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace aca
