// Programmatic dependent launch of the projection's kernel chain.
//
// Each kernel of the step is launched with programmatic stream serialisation:
// it may be scheduled while the kernel before it on the stream is still
// running (its CTAs take the SM slots that the earlier kernel's last wave
// leaves free, and its launch latency overlaps that kernel's tail).  Every such
// kernel begins with pdl_enter(): griddepcontrol.wait blocks until the
// preceding kernel has completed and its memory operations are visible (so no
// global data is read before it), then griddepcontrol.launch_dependents lets
// the next kernel be scheduled in turn.  Because the trigger follows the wait,
// at most one kernel ahead of the running one is ever resident and waiting,
// and a kernel sees everything every earlier kernel wrote (each completed
// after the wait of its successor's predecessor returned).  Launched without
// the attribute, both instructions have no effect.
//
// Launches into a stream that is being captured into a graph take no
// attribute: in the batched graph (independent per-plan branches running side
// by side) the waiting CTAs held slots the other branches could use (64 grids:
// 4.74 -> 4.94 ms per batch with the attribute), and within one plan's
// refinement graph it changed nothing measurable.  On direct launches it saves
// about 1 us per kernel boundary (256^3 step: 1.121 -> 1.105 ms).
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace ppe {

__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// kernel<<<grid, block, smem, st>>>(args...), with programmatic stream
// serialisation unless st is capturing (see above); returns the launch's error.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t ce = cudaStreamIsCapturing(st, &cs);
  if (ce != cudaSuccess) return ce;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = cs == cudaStreamCaptureStatusNone ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace ppe
