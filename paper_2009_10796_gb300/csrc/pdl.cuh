// Programmatic dependent launch between the consecutive kernels of a frame.
// A kernel launched with launch_pdl may be scheduled while the kernel before
// it on the stream is still running: its blocks take the SM resources that
// the earlier kernel's finished blocks give up and wait in pdl_wait() until
// that kernel has completed and its memory is visible, so the launch and
// the ramp of its blocks overlap the earlier kernel's tail.  Every kernel
// launched this way calls pdl_wait() before it touches device memory; the
// kernels call pdl_trigger() right after it, which lets the next kernel's
// blocks be scheduled once all of this kernel's blocks have started.  On a
// kernel launched the ordinary way both are no-ops in effect.  DDGI_NO_PDL=1
// in the environment (read at each launch) makes launch_pdl an ordinary
// launch.
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <utility>

namespace ddgi {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

inline bool pdl_enabled() {
    const char* e = std::getenv("DDGI_NO_PDL");
    return !(e && e[0] == '1');
}

template <typename... K, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              A&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

}  // namespace ddgi
