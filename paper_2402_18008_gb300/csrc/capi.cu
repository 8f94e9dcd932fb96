// Library-wide C-ABI helpers: error message, version, device properties.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace aca {

static thread_local char g_msg[512] = "";

aca_status set_error(aca_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return st;
}

int sm_count()
{
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 1;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)cache.size() <= dev)
        cache.resize(dev + 1, 0);
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
            v = 1;
        cache[dev] = v;
    }
    return cache[dev];
}

int blocks_per_sm(const void *kernel, int threads, size_t smem)
{
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, size_t, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(kernel, threads, smem, dev);
    {
        std::lock_guard<std::mutex> lock(mu);
        const auto it = cache.find(key);
        if (it != cache.end())
            return it->second;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = per_sm;
    return per_sm;
}

}  // namespace aca

extern "C" const char *aca_last_error(void) { return aca::g_msg; }

extern "C" const char *aca_version(void) { return "aca-gb300 0.1 (sm_103a)"; }
