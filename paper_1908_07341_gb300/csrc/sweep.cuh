// sweep.cuh -- what the half-step sweeps (kernels.cu) and the Section 3
// kernels (sampling.cu) share: the sweep arguments, the neighbour gathers of
// a 32-site block, and the launch-grid helper.
#pragma once

#ifdef __CUDACC_RTC__
#include "device.cuh"
#else
#include <algorithm>
#include <cstdint>

#include "internal.h"
#endif
#include "bounds.cuh"

namespace shk {

struct SweepArgs {
    const void* src;
    void* dst;
    uint32_t L;
    uint32_t Wr;          // blocks per row (aligned layouts)
    uint32_t nblocks;     // ceil(N / 32)
    int64_t N;
    FastDiv div_row;      // division by Wr
    uint32_t hs;
    long long* obs_cur;
    long long* obs_prev;
    long long* zero_slot;
    DrawParams P;
    PhiloxPrefix pre[8];  // round prefixes of the 8 Philox calls of half-step hs
    unsigned int* fault;  // set non-zero by a kernel whose bounded wait gave up (nullable)
};

// Programmatic dependent launch: the kernels are launched so that the next
// kernel in the stream may be scheduled while this one still runs.  Each waits
// here until the kernel before it has completed and its writes are visible
// (nothing is read or written before), then lets the next one be scheduled.
// Both are no-ops for a launch that did not ask for it.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------ neighbour gathers

// Bits of block w of a bit-packed (or bit-converted) plane and of the two field
// neighbours of its sites: HALF 0 -> (x down, x left), HALF 1 -> (x up, x right).
template <int HALF>
__device__ __forceinline__ void words_aligned(const uint32_t* __restrict__ pl, uint32_t w,
                                              uint32_t row, uint32_t col, uint32_t L, uint32_t Wr,
                                              uint32_t nblocks, uint32_t& S, uint32_t& N1,
                                              uint32_t& N2) {
    S = *checked(pl, w, nblocks, SHK_SITE);
    if (HALF == 0) {
        N1 = *checked(pl, row > 0 ? w - Wr : w + nblocks - Wr, nblocks, SHK_SITE);
        const uint32_t prev = *checked(pl, col > 0 ? w - 1 : w + Wr - 1, nblocks, SHK_SITE);
        N2 = (S << 1) | (prev >> 31);
    } else {
        N1 = *checked(pl, row + 1 < L ? w + Wr : w + Wr - nblocks, nblocks, SHK_SITE);
        const uint32_t next = *checked(pl, col + 1 < Wr ? w + 1 : w + 1 - Wr, nblocks, SHK_SITE);
        N2 = (S >> 1) | (next << 31);
    }
}

// Bit of site v of a bit plane of N sites.
__device__ __forceinline__ uint32_t bit_of(const uint32_t* pl, int64_t v, int64_t N) {
    return (*checked(pl, (uint64_t)(v >> 5), (uint64_t)((N + 31) >> 5), SHK_SITE) >> (v & 31)) & 1u;
}

// Generic side length (L % 32 != 0): site-by-site neighbour bits of block w of
// a bit plane with linear site order.
template <int HALF>
__device__ __forceinline__ void words_generic(const uint32_t* pl, uint32_t w, int64_t L, int64_t N,
                                              uint32_t& S, uint32_t& N1, uint32_t& N2,
                                              uint32_t& valid) {
    S = N1 = N2 = valid = 0;
    for (int p = 0; p < 32; ++p) {
        const int64_t u = 32 * (int64_t)w + p;
        if (u >= N) break;
        const int64_t j = u / L, i = u - j * L;
        int64_t a, b;
        if (HALF == 0) {
            a = j > 0 ? u - L : u + N - L;
            b = i > 0 ? u - 1 : u + L - 1;
        } else {
            a = j + 1 < L ? u + L : u + L - N;
            b = i + 1 < L ? u + 1 : u + 1 - L;
        }
        S |= bit_of(pl, u, N) << p;
        N1 |= bit_of(pl, a, N) << p;
        N2 |= bit_of(pl, b, N) << p;
        valid |= 1u << p;
    }
}

// int8 plane, generic L: site-by-site.
template <int HALF>
__device__ __forceinline__ void bytes_generic(const int8_t* __restrict__ pl, uint32_t w, int64_t L,
                                              int64_t N, uint32_t& S, uint32_t& N1, uint32_t& N2,
                                              uint32_t& valid) {
    S = N1 = N2 = valid = 0;
    for (int p = 0; p < 32; ++p) {
        const int64_t u = 32 * (int64_t)w + p;
        if (u >= N) break;
        const int64_t j = u / L, i = u - j * L;
        int64_t a, b;
        if (HALF == 0) {
            a = j > 0 ? u - L : u + N - L;
            b = i > 0 ? u - 1 : u + L - 1;
        } else {
            a = j + 1 < L ? u + L : u + L - N;
            b = i + 1 < L ? u + 1 : u + 1 - L;
        }
        S |= (uint32_t)(*checked(pl, (uint64_t)u, (uint64_t)N, SHK_SITE) > 0) << p;
        N1 |= (uint32_t)(*checked(pl, (uint64_t)a, (uint64_t)N, SHK_SITE) > 0) << p;
        N2 |= (uint32_t)(*checked(pl, (uint64_t)b, (uint64_t)N, SHK_SITE) > 0) << p;
        valid |= 1u << p;
    }
}

// int8 plane with L % 32 == 0: two 16-byte loads per 32 sites.
template <int HALF>
__device__ __forceinline__ void bytes_aligned(const int8_t* __restrict__ pl, uint32_t w, uint32_t row,
                                              uint32_t col, uint32_t L, uint32_t Wr,
                                              uint32_t nblocks, uint32_t& S, uint32_t& N1,
                                              uint32_t& N2) {
    const uint4* q4 = reinterpret_cast<const uint4*>(pl);     // 16-byte chunks, two per block
    const uint64_t n4 = 2 * (uint64_t)nblocks, nbytes = 32 * (uint64_t)nblocks;
    S = pack_up32(__ldg(checked(q4, 2 * (uint64_t)w, n4, SHK_SITE)),
                  __ldg(checked(q4, 2 * (uint64_t)w + 1, n4, SHK_SITE)));
    uint32_t wn;
    if (HALF == 0) wn = row > 0 ? w - Wr : w + nblocks - Wr;
    else wn = row + 1 < L ? w + Wr : w + Wr - nblocks;
    N1 = pack_up32(__ldg(checked(q4, 2 * (uint64_t)wn, n4, SHK_SITE)),
                   __ldg(checked(q4, 2 * (uint64_t)wn + 1, n4, SHK_SITE)));
    if (HALF == 0) {
        const size_t idx = col > 0 ? 32 * (size_t)w - 1 : 32 * (size_t)w + L - 1;
        N2 = (S << 1) | (uint32_t)(__ldg(checked(pl, idx, nbytes, SHK_SITE)) > 0);
    } else {
        const size_t idx = col + 1 < Wr ? 32 * (size_t)w + 32 : 32 * (size_t)w + 32 - L;
        N2 = (S >> 1) | ((uint32_t)(__ldg(checked(pl, idx, nbytes, SHK_SITE)) > 0) << 31);
    }
}

#ifndef __CUDACC_RTC__
// ------------------------------------------------------------ host helpers

int sm_count();
int blocks_per_sm(const void* kernel, int block);
SweepArgs sweep_args(const Geometry& g, const void* src, void* dst, const DrawParams& P,
                     uint32_t hs, long long* oc, long long* op, long long* z);

using SweepKernel = void (*)(SweepArgs);

// Launches kernel(a) with programmatic stream serialization (see pdl_begin):
// its launch overlaps the tail of the kernel before it in the stream.
template <class K>
inline cudaError_t launch_pdl(K kernel, int grid, int block, cudaStream_t st, const SweepArgs& a) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

// Grid of at most `waves` full waves of resident blocks (the kernels stride
// over their work), never more blocks than work items need.  With more than
// one wave the blocks of the later waves start as earlier ones retire, which
// evens out the end of the launch; programmatic dependent launch stays safe,
// because the next kernel launches only once every block of this one has
// started.
template <class K>
inline int grid_for(K kernel, int block, uint64_t work_items, int waves = 1) {
    const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(kernel), block);
    const uint64_t full = (uint64_t)per_sm * sm_count() * (uint64_t)waves;
    const uint64_t need = (work_items + block - 1) / block;
    return (int)std::max<uint64_t>(1, std::min(full, need));
}

#endif  // __CUDACC_RTC__

}  // namespace shk
