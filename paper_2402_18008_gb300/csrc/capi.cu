// Library-wide C-ABI helpers: error message, version, device properties.
#include <mutex>
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

}  // namespace aca

extern "C" const char *aca_last_error(void) { return aca::g_msg; }

extern "C" const char *aca_version(void) { return "aca-gb300 0.1 (sm_103a)"; }
