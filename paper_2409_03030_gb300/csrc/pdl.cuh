// Programmatic dependent launch (sm_90 and later) for the kernels of the CG
// iteration chain.  Each such kernel calls pdl_enter() before it touches
// memory: griddepcontrol.wait returns once the preceding grid in the stream
// has completed and its writes are visible, so the kernel observes exactly
// what plain stream order would give it; it then lets its own successor be
// launched, whose blocks take the SM slots freed by this grid's last wave and
// wait there.  What overlaps is the launch and block-scheduling ramp of each
// kernel, not any computation.  For a launch without the attribute both
// instructions have no effect.
#pragma once
#include <cuda_runtime.h>

namespace jqcd {

__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// kern<<<grid, block, smem, s>>>(args...) with programmatic stream
// serialization allowed; kern must call pdl_enter() first.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace jqcd
