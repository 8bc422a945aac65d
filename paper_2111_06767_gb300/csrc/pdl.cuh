// Programmatic dependent launch for the kernels of one smoothing step / V-cycle: a kernel launched
// this way may start (index set-up, static table loads, tensor-memory allocation) while the
// previous kernel on the stream is still running; it calls pdl_wait() before it touches anything
// the previous kernel writes, which returns once that kernel has completed and its memory is
// visible. Every kernel launched with launch_pdl calls pdl_wait() in all threads, so completion
// stays ordered along the stream (kernel k + 2 waits for k + 1, which waited for k).
#pragma once

#include <cuda_runtime.h>

#include <utility>

#include "internal.h"

namespace dg {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Lets the next kernel on the stream begin launching its CTAs (they still wait in pdl_wait()).
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Whether launches use programmatic dependent launch (off unless DG_PDL=1; read once).
bool pdl_enabled();

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  DG_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

}  // namespace dg
