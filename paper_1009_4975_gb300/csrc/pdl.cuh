// Programmatic dependent launch for the kernels of the CG iteration.  A kernel launched with
// launch_pdl may be scheduled while the kernel before it in the stream is still draining, so the
// launch latency and the previous kernel's last wave overlap.  Every kernel launched that way
// begins with pdl_begin(), before it reads or writes any memory: griddepcontrol.wait returns once
// the preceding grid has completed and its writes are visible (at once when there is no
// programmatic dependency), then griddepcontrol.launch_dependents allows the next kernel to be
// scheduled as this grid's CTAs retire.  In a stream capture the dependency becomes a
// programmatic edge of the graph.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace amr {

__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
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

}  // namespace amr
