// Programmatic dependent launch (sm_90 and later): a kernel launched with
// programmatic stream serialization may be scheduled while the previous
// kernel in its stream is still running; it must wait (griddep_wait) before
// touching memory that kernel reads or writes, which here is always its
// first statement.  griddep_launch lets the next such kernel be scheduled as
// soon as every CTA of this one has started.  Memory visibility is unchanged:
// griddepcontrol.wait returns only once the previous grid has completed and
// its writes are visible.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace st {

__device__ __forceinline__ void griddep_wait() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

__device__ __forceinline__ void griddep_launch() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// kernel<<<grid, block, smem, s>>>(args...) with programmatic stream
// serialization allowed (the kernel must start with griddep_wait()).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace st
