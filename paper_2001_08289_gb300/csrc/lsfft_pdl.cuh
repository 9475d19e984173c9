// Programmatic dependent launch for the kernels of one iteration.
//
// A kernel launched by launch_pdl() may be scheduled while the kernel before
// it in the stream is still running (its blocks are placed as soon as every
// block of the previous kernel has executed pdl_trigger() or exited), which
// hides the launch latency between the short passes of small grids.  Every
// such kernel calls pdl_wait() before its first memory access: it returns once
// the previous kernel has completed and its writes are visible, so the passes
// still see each other's results in stream order, and since every kernel in the
// chain waits before it can complete, the ordering is transitive.  A kernel
// launched without the attribute (or with nothing before it) passes pdl_wait()
// at once.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace lsfft {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// `programmatic` = 0 launches in plain stream order (the kernel's pdl_wait() then
// returns at once).  Where a kernel signals its dependents matters: signalled at
// its start (pdl_trigger() right after pdl_wait()), the next pass's blocks are
// placed while it still runs, which hides launch latency on small grids but slowed
// iterations whose passes alternate between kernels of different shapes (256^3:
// 0.928 vs 0.844 ms per iteration with plain launches).  Left to block exit, the
// dependents are released as the blocks finish; measured per iteration of a
// 128-iteration EM solve against signalling at the start: 8192^2 1.015 vs 1.030 ms,
// 512^2 21.5 vs 21.8 us, 256^3 0.837 vs 0.849 ms (plain launches), 128^3 0.106 vs
// 0.110 ms, but 64^2 (FP64) 18.0 vs 17.6 us.  So the passes signal at their start
// only on grids of at most 128^2 voxels (PassArgs::pdl_early) and at exit otherwise.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              int programmatic, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = programmatic ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace lsfft
