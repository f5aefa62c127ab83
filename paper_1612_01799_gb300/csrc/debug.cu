// The debug build's bounds-check word (debug.cuh) and its C-ABI accessor.  In the release
// build the accessor reports POISSON_ERR_UNSUPPORTED.
#include <cuda_runtime.h>

#include "../../include/poisson.h"
#include "debug.cuh"

namespace gsp {
#ifdef GSP_DEBUG
__device__ unsigned int gsp_debug_flags = 0;

// The checks on one in-range and two out-of-range cases; only the predicates run, no
// shared or global access is made here.
__global__ void k_debug_selftest(int *ok) {
    extern __shared__ __align__(16) unsigned char sm[];
    const bool inside = dbg_smem_ok(sm + 48, 16);      // the last 16 of 64 bytes
    const bool past = dbg_smem_ok(sm + 64, 4);         // one past the end: fails, sets bit 0
    const bool index = dbg_index_ok(-1, 10);           // fails, sets bit 1
    *ok = inside && !past && !index;
}
#endif
}  // namespace gsp

extern "C" int poisson_debug_flags(unsigned int *flags, void *stream) {
    if (!flags) return POISSON_ERR_ARG;
    *flags = 0;
#ifdef GSP_DEBUG
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int word = 0;
    const unsigned int zero = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&word, gsp::gsp_debug_flags, sizeof word);
    if (e == cudaSuccess && word) e = cudaMemcpyToSymbol(gsp::gsp_debug_flags, &zero, sizeof zero);
    if (e != cudaSuccess) return POISSON_ERR_CUDA;
    *flags = word;
    return POISSON_OK;
#else
    (void)stream;
    return POISSON_ERR_UNSUPPORTED;
#endif
}

extern "C" int poisson_debug_selftest(void *stream) {
#ifdef GSP_DEBUG
    cudaStream_t s = (cudaStream_t)stream;
    int *ok = nullptr, h = 0;
    cudaError_t e = cudaMalloc(&ok, sizeof(int));
    if (e != cudaSuccess) return POISSON_ERR_ALLOC;
    gsp::k_debug_selftest<<<1, 1, 64, s>>>(ok);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ok, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(ok);
    if (e != cudaSuccess) return POISSON_ERR_CUDA;
    return h ? POISSON_OK : POISSON_ERR_NUMERIC;
#else
    (void)stream;
    return POISSON_ERR_UNSUPPORTED;
#endif
}
