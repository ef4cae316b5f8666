// Programmatic dependent launch: every kernel of an outer step is launched so that the
// next one may be scheduled while it drains (stream capture turns this into programmatic
// graph edges).  Each kernel waits for its predecessor's completion (and memory) before
// its first read of data the predecessor produced, then lets its own successor launch.
#pragma once
#include <cuda_runtime.h>

namespace helm {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t s, Args... args)
{
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

// Asynchronous global -> shared copies of one complex element (8 or 16 bytes), many in
// flight per thread; a false predicate zero-fills the destination (nothing is read).
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* smem, const void* gmem, bool pred)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int src = pred ? BYTES : 0;
    if constexpr (BYTES == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Every kernel asks for the largest shared-memory carve-out, so consecutive kernels of a
// step never need a different L1 / shared-memory split on an SM.
template <typename... KArgs>
inline cudaError_t max_carveout(void (*kern)(KArgs...))
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

}  // namespace helm
