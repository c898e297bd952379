// Programmatic dependent launch: a kernel of the stepping chain may start
// while the previous kernel of its stream finishes.  Each such kernel
//   * triggers its dependents from inside its running CTAs (so a dependent
//     grid is launched only once every CTA of this grid has been scheduled:
//     its waiting CTAs can never keep one of ours from running), and
//   * waits for the previous grid's completion and memory before its first
//     access to data that grid may read or write, doing only setup from
//     host-written data (tables, weights, barriers, TMEM) before that.
// Both instructions are no-ops in a kernel launched without the attribute.
#pragma once
#include <cuda_runtime.h>

namespace starmap {

__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch `kernel` on `stream`, with programmatic stream serialisation if
// `overlap` (else an ordinary launch).
template <class... Params, class... Args>
cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       bool overlap, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = overlap ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

}  // namespace starmap
