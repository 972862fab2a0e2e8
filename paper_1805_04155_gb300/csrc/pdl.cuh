// Programmatic dependent launch for the short kernels of the Krylov iteration.
//
// A kernel launched with launch_pdl may be scheduled while its predecessor in
// the stream is still finishing, so the launch latency of the iteration's
// ~30 short kernels overlaps the previous kernel's tail.  Such a kernel must
// call pdl_wait() before it reads or writes anything: griddepcontrol.wait
// returns once the predecessor grid has completed and its memory operations
// are visible.  pdl_launch_dependents() lets the next kernel of the stream be
// scheduled; it is called right after pdl_wait(), so at most one more grid is
// resident beside the running one (all grids of the iteration fit in one
// resident wave, so the waiting CTAs never displace the running kernel's).
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <utility>

namespace ep {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// pdl_wait() then pdl_launch_dependents(): the first statement of every kernel launched by launch_pdl.
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_launch_dependents();
}

// EP_NO_PDL=1 launches these kernels without the attribute (plain stream order; griddepcontrol.wait
// then returns at once): for kernel profilers that cannot follow programmatic dependencies.
inline bool pdl_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("EP_NO_PDL");
        return !(v && v[0] == '1');
    }();
    return on;
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace ep
