// bounds.cuh -- index checks of the debug build.
//
// Built with -DSHK_DEBUG_BOUNDS (build.py --debug-bounds), every global-memory
// access of the kernels goes through checked(base, i, n, site): an index at
// or past its buffer's end records the site (translation unit << 16 | source
// line) of the first such access in a device status word and is replaced by
// index 0, so the access stays inside the buffer and nothing traps.  The
// host reads and clears the word with shk_debug_bounds().  In the normal
// build checked() is plain pointer arithmetic.
#pragma once

#ifndef __CUDACC_RTC__
#include <cstdint>
#include <cuda_runtime.h>
#endif

#ifndef SHK_TU_ID
#define SHK_TU_ID 0
#endif
#define SHK_SITE ((unsigned)((SHK_TU_ID << 16) | (__LINE__ & 0xFFFF)))

namespace shk {

#ifdef SHK_DEBUG_BOUNDS
static __device__ unsigned int g_bounds_site = 0;   // one per translation unit

template <class T>
__device__ __forceinline__ T* checked(T* base, uint64_t i, uint64_t n, unsigned site) {
    if (i >= n) {
        atomicCAS(&g_bounds_site, 0u, site);
        return base;
    }
    return base + i;
}

// The len elements base[i .. i + len) (a bulk copy's source): checked as a
// whole, replaced by the buffer's start when they do not fit.
template <class T>
__device__ __forceinline__ T* checked_range(T* base, uint64_t i, uint64_t len, uint64_t n, unsigned site) {
    if (i + len > n || len > n) {
        atomicCAS(&g_bounds_site, 0u, site);
        return base;
    }
    return base + i;
}

#ifndef __CUDACC_RTC__
// First recorded site of this translation unit (0 = none), cleared.
static inline unsigned take_bounds_site() {
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_site, sizeof v) != cudaSuccess) return 0xFFFFFFFFu;
    cudaMemcpyToSymbol(g_bounds_site, &z, sizeof z);
    return v;
}
#endif
constexpr bool kBoundsChecked = true;
#else
template <class T>
__device__ __forceinline__ T* checked(T* base, uint64_t i, uint64_t, unsigned) {
    return base + i;
}
template <class T>
__device__ __forceinline__ T* checked_range(T* base, uint64_t i, uint64_t, uint64_t, unsigned) {
    return base + i;
}
#ifndef __CUDACC_RTC__
static inline unsigned take_bounds_site() { return 0; }
#endif
constexpr bool kBoundsChecked = false;
#endif

}  // namespace shk
