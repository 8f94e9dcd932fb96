// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// launch_after_previous() may be scheduled while its stream predecessor is
// still running, so it must call grid_dependency_wait() before it touches
// anything the predecessor reads or writes; the wait returns once every
// prerequisite grid has completed and its memory operations are visible.
// grid_launch_dependents() lets such a successor be scheduled once every
// block of the current grid has issued it (or exited).  Without the launch
// attribute both are no-ops, so every kernel here can use them either way.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace aca {

__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void grid_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_after_previous(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                  Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace aca
