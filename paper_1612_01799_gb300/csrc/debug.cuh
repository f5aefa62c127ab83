// Bounds checks of the debug build (compiled with GSP_DEBUG into libgspoisson_debug.so).
// The shared-memory helpers of the pass kernels check every access against the CTA's
// dynamic shared memory, and the runtime-length forms check their computed global row
// indices against their arrays; an access that fails is skipped (a load yields zero) and
// sets a bit of gsp_debug_flags, which poisson_debug_flags reads and clears.  No access
// traps.  In the release build every check is the constant true and compiles to nothing.
#pragma once
#include <cstdint>

namespace gsp {

constexpr unsigned kDebugSmem = 1;    // a shared access outside the CTA's dynamic shared memory
constexpr unsigned kDebugGlobal = 2;  // a computed global index outside its array

#ifdef GSP_DEBUG
extern __device__ unsigned int gsp_debug_flags;

// The start of the CTA's dynamic shared memory (every extern shared array aliases it; the
// pass kernels use no static shared memory).
extern __shared__ __align__(16) unsigned char gsp_dyn_smem[];

__device__ __forceinline__ bool dbg_smem_ok(uint32_t a, uint32_t bytes) {
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(gsp_dyn_smem);
    uint32_t size;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(size));
    if (a >= base && a + bytes <= base + size) return true;
    atomicOr(&gsp_debug_flags, kDebugSmem);
    return false;
}
__device__ __forceinline__ bool dbg_smem_ok(const void *p, uint32_t bytes) {
    return dbg_smem_ok((uint32_t)__cvta_generic_to_shared(p), bytes);
}
__device__ __forceinline__ bool dbg_index_ok(long long i, long long n) {
    if (i >= 0 && i < n) return true;
    atomicOr(&gsp_debug_flags, kDebugGlobal);
    return false;
}
#else
__device__ __forceinline__ constexpr bool dbg_smem_ok(uint32_t, uint32_t) { return true; }
__device__ __forceinline__ constexpr bool dbg_smem_ok(const void *, uint32_t) { return true; }
__device__ __forceinline__ constexpr bool dbg_index_ok(long long, long long) { return true; }
#endif

// Checked shared-memory load and store of a value of type T at p.
template <typename T> __device__ __forceinline__ T sm_ld(const T *p) {
    if (!dbg_smem_ok(p, sizeof(T))) return T{};
    return *p;
}
template <typename T> __device__ __forceinline__ void sm_st(T *p, const T &v) {
    if (dbg_smem_ok(p, sizeof(T))) *p = v;
}

}  // namespace gsp
