// ransac_aca for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc at all: a plugin whose
// host framework owns every byte of device memory through its own allocator,
// a latency-critical loop where an allocation (which can synchronise the
// device) is not allowed, or a long-running service whose device-memory
// budget is fixed when it starts.  For them, ransac_aca_noalloc runs the
// same RANSAC as ransac_aca, with its scratch (per-problem offsets, work
// counter, per-hypothesis counts) in a fixed array that is part of this
// library's own device image.
//
// That array is a file-scope __device__ variable of ACA_NOALLOC_SCRATCH_BYTES
// bytes.  Every GPU that loads the library holds it until the process exits.
// In host code its name is only a host-side stand-in, not a device address:
// the device address is looked up once per device, with that device current,
// by cudaGetSymbolAddress on the first call made on that device, and cached.
// Under lazy module loading (the CUDA runtime's default), that lookup is also
// what loads this file's module onto the device and reserves the array, so
// the first call on each device may allocate: make it once as a warm-up,
// outside any region that must not allocate and before any stream capture
// (or run with CUDA_MODULE_LOADING=EAGER, which reserves the array when the
// library's context is created).  All calls share the one array and each call re-initialises what
// must start at zero (the work counter, the overflow flag and the counts),
// so calls whose kernels overlap on the GPU (two streams, or two host threads)
// race on it and must be serialised by the caller.  The done counter of the
// one-launch path (at most 8 problems) must be zero before a call and every
// call leaves it zero; the array is zero when the module loads.
#include <mutex>
#include <vector>

#include "common.cuh"

static __device__ __align__(256) unsigned char g_ransac_scratch[ACA_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_scratch_mu;
std::vector<void *> g_scratch_addr;   // device address of g_ransac_scratch, per device

aca_status scratch_for_current_device(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return aca::set_error(ACA_ERR_CUDA, "ransac_aca_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if ((int)g_scratch_addr.size() <= dev)
        g_scratch_addr.resize(dev + 1, nullptr);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_ransac_scratch);
        if (e != cudaSuccess || p == nullptr)
            return aca::set_error(ACA_ERR_CUDA, "ransac_aca_noalloc: cudaGetSymbolAddress: %s",
                                  cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return ACA_OK;
}

}  // namespace

extern "C" aca_status ransac_aca_noalloc(const float *corr, const int64_t *offsets, const int32_t *n_hyp,
                                         int32_t P, int64_t total_hyps, const aca_ransac_params *params,
                                         float *best_H, int32_t *best_count, int32_t *best_hyp,
                                         int32_t *hyp_counts, uint8_t *inlier_mask, void *stream)
{
    if (P < 0 || total_hyps < 0)
        return aca::set_error(ACA_ERR_INVALID_ARG, "ransac_aca_noalloc: P and total_hyps must be >= 0");
    const size_t need = ransac_aca_workspace_size(P, total_hyps);
    if (need > (size_t)ACA_NOALLOC_SCRATCH_BYTES)
        return aca::set_error(ACA_ERR_WORKSPACE,
                              "ransac_aca_noalloc: %d problems with %lld hypotheses need %zu bytes of scratch, "
                              "more than the built-in %zu bytes; use ransac_aca with a caller workspace",
                              (int)P, (long long)total_hyps, need, (size_t)ACA_NOALLOC_SCRATCH_BYTES);
    if (P == 0)
        return ACA_OK;
    void *scratch = nullptr;
    const aca_status st = scratch_for_current_device(&scratch);
    if (st != ACA_OK)
        return st;
    // Only the part of the array that total_hyps accounts for is handed on:
    // the count capacity is then exactly total_hyps, so a device-side sum of
    // n_hyp above it is caught by ransac_aca's overflow check (best_hyp = -2,
    // nothing scored, no write past the caller's hyp_counts) as it is with a
    // caller workspace of the same size.
    const size_t bytes =
        ransac_aca_workspace_size(P, 0) + sizeof(int32_t) * (size_t)total_hyps * aca::ransac_count_slots(P);
    return ransac_aca(corr, offsets, n_hyp, P, params, best_H, best_count, best_hyp, hyp_counts, inlier_mask,
                      scratch, bytes, stream);
}
