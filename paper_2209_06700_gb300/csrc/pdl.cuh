// Programmatic dependent launch for the chains of short kernels of libirk (sm_90 and later).
//
// Every kernel of the library starts with dev::pdl_enter() and all but the 3D operator kernel are
// launched through launch_pdl(): the next kernel of a stream (or of a captured graph) may then be scheduled while its predecessor
// is still running, so that its launch and setup overlap the predecessor's tail; it waits in
// pdl_enter() until the predecessor has completed and its writes are visible, before it touches
// memory.  A kernel launched without the attribute passes the wait at once.  The operator kernels
// (op3d_kernel, clusters of up to 16 CTAs, one wave of the device) keep plain launches: scheduled
// early, their waiting CTAs held SMs that their predecessor's tail needed (measured 18.4 -> 20.3 ms
// per step at degree 4 on 32^3 cells; 18.1 ms with the operator kernels left out).
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace irk {
namespace dev {

__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

}  // namespace dev

// kern<<<grid, block, smem, st>>>(args...) with programmatic stream serialisation allowed; the
// launch error (if any) is also left for cudaGetLastError().
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
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
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace irk
