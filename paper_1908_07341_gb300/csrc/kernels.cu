// kernels.cu -- sm_103a kernels of the shaken-dynamics hot path and their
// launchers.
//
//   k_sweep_bp<HALF, ...>  one half-step over a bit-packed plane (Eq. leftTrans
//                          for HALF = 0, Eq. rightTrans for HALF = 1) with the
//                          observable reductions fused; launch-shape variants
//   k_sweep_i8a<HALF, ...> the same over an int8 +/-1 plane with L % 32 == 0
//   k_sweep_i8g<HALF>      the same for any L (site-by-site gathers)
//   k_cnn<LAYOUT, AL>      nearest-neighbour sum C_nn of a sigma plane
//   k_init<LAYOUT, AL>     initial states
//   k_run_small<LAYOUT>    a whole run of n steps inside one CTA, both planes
//                          held as bits in shared memory (small lattices)
//
// Each thread owns 32-site blocks (one bit-packed word); a warp walks 32
// consecutive blocks together so that the lazy random-plane loop of
// draw_block() can exit as soon as the whole warp is decided.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>
#include <unordered_map>

#include "internal.h"

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
};

// ------------------------------------------------------------ neighbour gathers

// Bits of block w of a bit-packed (or bit-converted) plane and of the two field
// neighbours of its sites: HALF 0 -> (x down, x left), HALF 1 -> (x up, x right).
template <int HALF>
__device__ __forceinline__ void words_aligned(const uint32_t* __restrict__ pl, uint32_t w,
                                              uint32_t row, uint32_t col, uint32_t L, uint32_t Wr,
                                              uint32_t nblocks, uint32_t& S, uint32_t& N1,
                                              uint32_t& N2) {
    S = pl[w];
    if (HALF == 0) {
        N1 = pl[row > 0 ? w - Wr : w + nblocks - Wr];
        const uint32_t prev = pl[col > 0 ? w - 1 : w + Wr - 1];
        N2 = (S << 1) | (prev >> 31);
    } else {
        N1 = pl[row + 1 < L ? w + Wr : w + Wr - nblocks];
        const uint32_t next = pl[col + 1 < Wr ? w + 1 : w + 1 - Wr];
        N2 = (S >> 1) | (next << 31);
    }
}

__device__ __forceinline__ uint32_t bit_of(const uint32_t* pl, int64_t v) {
    return (pl[v >> 5] >> (v & 31)) & 1u;
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
        S |= bit_of(pl, u) << p;
        N1 |= bit_of(pl, a) << p;
        N2 |= bit_of(pl, b) << p;
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
        S |= (uint32_t)(pl[u] > 0) << p;
        N1 |= (uint32_t)(pl[a] > 0) << p;
        N2 |= (uint32_t)(pl[b] > 0) << p;
        valid |= 1u << p;
    }
}

// int8 plane with L % 32 == 0: two 16-byte loads per 32 sites.
template <int HALF>
__device__ __forceinline__ void bytes_aligned(const int8_t* __restrict__ pl, uint32_t w, uint32_t row,
                                              uint32_t col, uint32_t L, uint32_t Wr,
                                              uint32_t nblocks, uint32_t& S, uint32_t& N1,
                                              uint32_t& N2) {
    const uint4* s4 = reinterpret_cast<const uint4*>(pl + 32 * (size_t)w);
    S = pack_up32(__ldg(s4), __ldg(s4 + 1));
    uint32_t wn;
    if (HALF == 0) wn = row > 0 ? w - Wr : w + nblocks - Wr;
    else wn = row + 1 < L ? w + Wr : w + Wr - nblocks;
    const uint4* n4 = reinterpret_cast<const uint4*>(pl + 32 * (size_t)wn);
    N1 = pack_up32(__ldg(n4), __ldg(n4 + 1));
    if (HALF == 0) {
        const size_t idx = col > 0 ? 32 * (size_t)w - 1 : 32 * (size_t)w + L - 1;
        N2 = (S << 1) | (uint32_t)(__ldg(pl + idx) > 0);
    } else {
        const size_t idx = col + 1 < Wr ? 32 * (size_t)w + 32 : 32 * (size_t)w + 32 - L;
        N2 = (S >> 1) | ((uint32_t)(__ldg(pl + idx) > 0) << 31);
    }
}

// ------------------------------------------------------------ half-step sweeps

template <int HALF>
__device__ __forceinline__ void accumulate_step(int (&acc)[3], uint32_t up, uint32_t S, uint32_t N1,
                                                uint32_t N2, uint32_t valid, bool cnn) {
    const int nv = __popc(valid);
    if (HALF == 0) {
        acc[0] += 2 * __popc(up) - nv;                                              // M_tau
        if (cnn) acc[1] += 2 * nv - 2 * (__popc((S ^ N1) & valid) + __popc((S ^ N2) & valid));
    } else {
        acc[0] += 2 * __popc(up) - nv;                                              // M_sigma
        acc[1] += nv - 2 * __popc((up ^ S) & valid);                                // S_q
        acc[2] += 2 * nv - 2 * (__popc((up ^ N1) & valid) + __popc((up ^ N2) & valid));  // S_J
    }
}

template <int HALF>
__device__ __forceinline__ void finish_step(const int (&acc)[3], const SweepArgs& a) {
    if (HALF == 0) {
        const int v[2] = {acc[0], acc[1]};
        long long* const d[2] = {a.obs_cur ? a.obs_cur + 1 : nullptr,
                                 a.obs_prev ? a.obs_prev + 4 : nullptr};
        block_accumulate<2>(v, d);
    } else {
        const int v[3] = {acc[0], acc[1], acc[2]};
        long long* const d[3] = {a.obs_cur ? a.obs_cur + 0 : nullptr,
                                 a.obs_cur ? a.obs_cur + 2 : nullptr,
                                 a.obs_cur ? a.obs_cur + 3 : nullptr};
        block_accumulate<3>(v, d);
    }
}

// Raw words of one bit-packed block as loaded: the block itself, its row
// neighbour (down for A, up for B) and the adjacent word that supplies the
// wrap-around bit of the left (A) or right (B) neighbour.
struct RawBp {
    uint32_t s, n, x;
};

template <int HALF>
__device__ __forceinline__ RawBp load_bp(const uint32_t* __restrict__ src, uint32_t w,
                                         const SweepArgs& a) {
    const uint32_t row = fdiv(w, a.div_row);
    const uint32_t col = w - row * a.Wr;
    RawBp r;
    r.s = __ldg(src + w);
    if (HALF == 0) {
        r.n = __ldg(src + (row > 0 ? w - a.Wr : w + a.nblocks - a.Wr));
        r.x = __ldg(src + (col > 0 ? w - 1 : w + a.Wr - 1));
    } else {
        r.n = __ldg(src + (row + 1 < a.L ? w + a.Wr : w + a.Wr - a.nblocks));
        r.x = __ldg(src + (col + 1 < a.Wr ? w + 1 : w + 1 - a.Wr));
    }
    return r;
}

template <int HALF>
__device__ __forceinline__ void decode_bp(const RawBp& r, uint32_t& S, uint32_t& N1, uint32_t& N2) {
    S = r.s;
    N1 = r.n;
    N2 = HALF == 0 ? (S << 1) | (r.x >> 31) : (S >> 1) | (r.x << 31);
}

// Bit-packed half-step.  A warp walks groups of 32 * ILP consecutive blocks;
// each thread draws ILP blocks with interleaved Philox chains, and, with
// PREFETCH, issues the loads of its next group before drawing the current one.
template <int HALF, int ILP, bool PREFETCH, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_sweep_bp(const SweepArgs a) {
    const uint32_t* __restrict__ src = static_cast<const uint32_t*>(a.src);
    uint32_t* __restrict__ dst = static_cast<uint32_t*>(a.dst);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t stride = ((gridDim.x * blockDim.x) >> 5) * 32 * ILP;
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[3] = {0, 0, 0};
    // nblocks is a multiple of 32, so a 32-block group is all in or all out and
    // the validity tests below are uniform across the warp.
    uint32_t base = gwarp * 32 * ILP;
    RawBp raw[ILP];
    if (PREFETCH && base < a.nblocks) {
#pragma unroll
        for (int k = 0; k < ILP; ++k)
            if (base + 32 * k < a.nblocks) raw[k] = load_bp<HALF>(src, base + 32 * k + lane, a);
    }
    for (; base < a.nblocks; base += stride) {
        uint32_t S[ILP], N1[ILP], N2[ILP], w[ILP], valid[ILP], up[ILP];
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            w[k] = base + 32 * k + lane;
            const bool in = base + 32 * k < a.nblocks;
            valid[k] = in ? 0xffffffffu : 0u;
            if (!PREFETCH && in) raw[k] = load_bp<HALF>(src, w[k], a);
            if (in) decode_bp<HALF>(raw[k], S[k], N1[k], N2[k]);
            else S[k] = N1[k] = N2[k] = 0;
        }
        if (PREFETCH) {
            const uint32_t nb = base + stride;
#pragma unroll
            for (int k = 0; k < ILP; ++k)
                if (nb + 32 * k < a.nblocks) raw[k] = load_bp<HALF>(src, nb + 32 * k + lane, a);
        }
        draw_blocks<ILP>(S, N1, N2, w, valid, a.hs, a.P, up);
#pragma unroll
        for (int k = 0; k < ILP; ++k) {
            if (valid[k]) {
                dst[w[k]] = up[k];
                accumulate_step<HALF>(acc, up[k], S[k], N1[k], N2[k], 0xffffffffu, cnn);
            }
        }
    }
    finish_step<HALF>(acc, a);
}

// Raw bytes of one int8 block (L % 32 == 0): the 32 sites, the 32 row
// neighbours and the one byte beyond the block that the left/right field needs.
struct RawI8 {
    uint4 s0, s1, n0, n1;
    int x;
};

template <int HALF>
__device__ __forceinline__ RawI8 load_i8(const int8_t* __restrict__ src, uint32_t w, const SweepArgs& a) {
    const uint32_t row = fdiv(w, a.div_row);
    const uint32_t col = w - row * a.Wr;
    RawI8 r;
    const uint4* s4 = reinterpret_cast<const uint4*>(src + 32 * (size_t)w);
    r.s0 = __ldg(s4);
    r.s1 = __ldg(s4 + 1);
    const uint32_t wn = HALF == 0 ? (row > 0 ? w - a.Wr : w + a.nblocks - a.Wr)
                                  : (row + 1 < a.L ? w + a.Wr : w + a.Wr - a.nblocks);
    const uint4* n4 = reinterpret_cast<const uint4*>(src + 32 * (size_t)wn);
    r.n0 = __ldg(n4);
    r.n1 = __ldg(n4 + 1);
    size_t idx;
    if (HALF == 0) idx = col > 0 ? 32 * (size_t)w - 1 : 32 * (size_t)w + a.L - 1;
    else idx = col + 1 < a.Wr ? 32 * (size_t)w + 32 : 32 * (size_t)w + 32 - a.L;
    r.x = __ldg(src + idx);
    return r;
}

template <int HALF>
__device__ __forceinline__ void decode_i8(const RawI8& r, uint32_t& S, uint32_t& N1, uint32_t& N2) {
    S = pack_up32(r.s0, r.s1);
    N1 = pack_up32(r.n0, r.n1);
    N2 = HALF == 0 ? (S << 1) | (uint32_t)(r.x > 0) : (S >> 1) | ((uint32_t)(r.x > 0) << 31);
}

// int8 half-step for L % 32 == 0 (one 32-byte block per thread per step of
// the walk, optionally prefetching the next block's bytes).
template <int HALF, bool PREFETCH, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_sweep_i8a(const SweepArgs a) {
    const int8_t* __restrict__ src = static_cast<const int8_t*>(a.src);
    int8_t* __restrict__ dst = static_cast<int8_t*>(a.dst);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t stride = ((gridDim.x * blockDim.x) >> 5) * 32;
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[3] = {0, 0, 0};
    uint32_t base = gwarp * 32;
    RawI8 raw;
    if (PREFETCH && base < a.nblocks) raw = load_i8<HALF>(src, base + lane, a);
    for (; base < a.nblocks; base += stride) {
        const uint32_t w = base + lane;
        if (!PREFETCH) raw = load_i8<HALF>(src, w, a);
        uint32_t S, N1, N2;
        decode_i8<HALF>(raw, S, N1, N2);
        if (PREFETCH && base + stride < a.nblocks) raw = load_i8<HALF>(src, base + stride + lane, a);
        const uint32_t up = draw_block(S, N1, N2, w, 0xffffffffu, a.hs, a.P);
        uint4 lo, hi;
        unpack32(up, lo, hi);
        uint4* d4 = reinterpret_cast<uint4*>(dst + 32 * (size_t)w);
        d4[0] = lo;
        d4[1] = hi;
        accumulate_step<HALF>(acc, up, S, N1, N2, 0xffffffffu, cnn);
    }
    finish_step<HALF>(acc, a);
}

// ------------------------------------------------------------ two-phase sweeps
//
// Each warp owns a ring of kQueueCap parked blocks in shared memory (structure
// of arrays: block index, undecided mask, decided-up mask and the three input
// words).  Blocks still undecided after Philox calls 0 and 1 wait there; once
// 32 are waiting the warp continues them together from call 2 (draw_rest).

constexpr int kQueueFields = 6;

template <int HALF, int LAYOUT>
__device__ __forceinline__ void finish_block(const SweepArgs& a, uint32_t w, uint32_t up, uint32_t S,
                                             uint32_t N1, uint32_t N2, bool cnn, int (&acc)[3]) {
    if (LAYOUT == kBitpack) {
        static_cast<uint32_t*>(a.dst)[w] = up;
    } else {
        uint4 lo, hi;
        unpack32(up, lo, hi);
        uint4* d4 = reinterpret_cast<uint4*>(static_cast<int8_t*>(a.dst) + 32 * (size_t)w);
        d4[0] = lo;
        d4[1] = hi;
    }
    accumulate_step<HALF>(acc, up, S, N1, N2, 0xffffffffu, cnn);
}

// Continues the `count` (<= 32) oldest parked blocks; all lanes call it.
template <int HALF, int LAYOUT, class PP>
__device__ __forceinline__ void drain_queue(const SweepArgs& a, const PP& P, uint32_t (*q)[kQueueCap],
                                            uint32_t head, int count, bool cnn, int (&acc)[3]) {
    const uint32_t lane = threadIdx.x & 31;
    const bool has = (int)lane < count;
    const uint32_t i = (head + lane) & (kQueueCap - 1);
    uint32_t w = 0, und = 0, up = 0, S = 0, N1 = 0, N2 = 0;
    if (has) {
        w = q[0][i];
        und = q[1][i];
        up = q[2][i];
        S = q[3][i];
        N1 = q[4][i];
        N2 = q[5][i];
    }
    const BlockClass k = block_class(S, N1, N2);
    const uint32_t res = draw_rest(k, w, und, up, a.hs, P);
    if (has) finish_block<HALF, LAYOUT>(a, w, res, S, N1, N2, cnn, acc);
}

template <int HALF, int LAYOUT, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_sweep_q(const SweepArgs a) {
    __shared__ uint32_t qbuf[BLOCK / 32][kQueueFields][kQueueCap];
    const DrawParams& P = a.P;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t stride = ((gridDim.x * blockDim.x) >> 5) * 32;
    uint32_t (*q)[kQueueCap] = qbuf[threadIdx.x >> 5];
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[3] = {0, 0, 0};
    uint32_t head = 0;
    int count = 0;
    const uint32_t below = (1u << lane) - 1u;
    // nblocks is a multiple of 32 for these layouts: every lane is active.
    for (uint32_t base = gwarp * 32; base < a.nblocks; base += stride) {
        const uint32_t w = base + lane;
        uint32_t S, N1, N2;
        if (LAYOUT == kBitpack) {
            const RawBp r = load_bp<HALF>(static_cast<const uint32_t*>(a.src), w, a);
            decode_bp<HALF>(r, S, N1, N2);
        } else {
            const RawI8 r = load_i8<HALF>(static_cast<const int8_t*>(a.src), w, a);
            decode_i8<HALF>(r, S, N1, N2);
        }
        const BlockClass k = block_class(S, N1, N2);
        uint32_t und, up;
        draw_first_two(k, w, 0xffffffffu, a.hs, P, und, up);
        const bool parked = und != 0u;
        const uint32_t mask = __ballot_sync(0xffffffffu, parked);
        if (parked) {
            const uint32_t i = (head + count + __popc(mask & below)) & (kQueueCap - 1);
            q[0][i] = w;
            q[1][i] = und;
            q[2][i] = up;
            q[3][i] = S;
            q[4][i] = N1;
            q[5][i] = N2;
        } else {
            finish_block<HALF, LAYOUT>(a, w, up, S, N1, N2, cnn, acc);
        }
        count += __popc(mask);
        if (count >= 32) {
            __syncwarp();
            drain_queue<HALF, LAYOUT>(a, P, q, head, 32, cnn, acc);
            __syncwarp();
            head = (head + 32) & (kQueueCap - 1);
            count -= 32;
        }
    }
    if (count > 0) {
        __syncwarp();
        drain_queue<HALF, LAYOUT>(a, P, q, head, count, cnn, acc);
    }
    finish_step<HALF>(acc, a);
}

// ------------------------------------------------------------ strip-walk sweep
//
// Planes with L % 1024 == 0 (rows of a multiple of 32 blocks).  A task is a
// strip of 32 consecutive blocks (one per lane) over consecutive rows; every
// warp of the grid gets an equal share of the rows of all strips (at most two
// tasks).  The warp walks the rows
// in the direction that makes the row neighbour the previous row it already
// holds as bits (up for half-step A, which reads x^down; down for B, which
// reads x^up).  The bit beside the block comes from the next lane by a shuffle,
// and from one scalar load at the strip edge.  The next row is prefetched
// while the current one is drawn.  Blocks undecided after two Philox calls go
// through the same warp queue as in k_sweep_q.

// One row of a lane's block as loaded: a word (bit-packed) or 32 bytes (int8).
template <int LAYOUT>
struct RowRaw;
template <>
struct RowRaw<kBitpack> {
    uint32_t v;
};
template <>
struct RowRaw<kInt8> {
    uint4 lo, hi;
};

template <int LAYOUT>
__device__ __forceinline__ RowRaw<LAYOUT> load_row(const void* src, uint32_t w) {
    RowRaw<LAYOUT> r;
    if constexpr (LAYOUT == kBitpack) {
        r.v = __ldg(static_cast<const uint32_t*>(src) + w);
    } else {
        const uint4* p = reinterpret_cast<const uint4*>(static_cast<const int8_t*>(src) + 32 * (size_t)w);
        r.lo = __ldg(p);
        r.hi = __ldg(p + 1);
    }
    return r;
}

template <int LAYOUT>
__device__ __forceinline__ uint32_t row_bits(const RowRaw<LAYOUT>& r) {
    if constexpr (LAYOUT == kBitpack) return r.v;
    else return pack_up32(r.lo, r.hi);
}

// The field-neighbour bit just outside the strip in row `row`: bit 31 of the
// block left of the strip (A) or bit 0 of the block right of it (B).
template <int HALF, int LAYOUT>
__device__ __forceinline__ uint32_t edge_bit(const void* src, uint32_t row, uint32_t edge_block, uint32_t W) {
    const size_t b = (size_t)row * W + edge_block;
    if constexpr (LAYOUT == kBitpack) {
        const uint32_t v = __ldg(static_cast<const uint32_t*>(src) + b);
        return HALF == 0 ? v >> 31 : v & 1u;
    } else {
        const int8_t* p = static_cast<const int8_t*>(src);
        return (uint32_t)(__ldg(p + 32 * b + (HALF == 0 ? 31 : 0)) > 0);
    }
}

template <int HALF, int LAYOUT, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_sweep_strip(const SweepArgs a) {
    __shared__ uint32_t qbuf[BLOCK / 32][kQueueFields][kQueueCap];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    uint32_t (*q)[kQueueCap] = qbuf[threadIdx.x >> 5];
    const DrawParams& P = a.P;
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[3] = {0, 0, 0};
    uint32_t head = 0;
    int count = 0;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t W = a.Wr, L = a.L;
    const uint32_t nstrips = W / 32;
    const bool edge_lane = HALF == 0 ? lane == 0 : lane == 31;
    // Warp g walks the row-strip indices [g T / G, (g+1) T / G) of the
    // strip-major sequence (strip * L + row), T = nstrips * L, G = warps: equal
    // shares, split where a strip ends.
    const uint64_t total = (uint64_t)nstrips * L;
    uint64_t pos = total * gwarp / nwarps;
    const uint64_t end = total * (gwarp + 1) / nwarps;
    while (pos < end) {
        const uint32_t strip = (uint32_t)(pos / L);
        const uint32_t r0 = (uint32_t)(pos - (uint64_t)strip * L);
        const uint64_t left_here = end - pos, left_in_strip = L - r0;
        const uint32_t nrows = (uint32_t)(left_here < left_in_strip ? left_here : left_in_strip);
        pos += nrows;
        const uint32_t col = strip * 32 + lane;
        const uint32_t edge_block = HALF == 0 ? (strip == 0 ? W - 1 : strip * 32 - 1)
                                              : (strip + 1 == nstrips ? 0 : strip * 32 + 32);
        // rows in walk order: A ascends r0..r0+nrows-1, B descends
        auto row_at = [&](uint32_t i) -> uint32_t { return HALF == 0 ? r0 + i : r0 + nrows - 1 - i; };
        const uint32_t first = row_at(0);
        const uint32_t nb_row = HALF == 0 ? (first == 0 ? L - 1 : first - 1) : (first + 1 == L ? 0 : first + 1);
        uint32_t prev = row_bits<LAYOUT>(load_row<LAYOUT>(a.src, nb_row * W + col));
        RowRaw<LAYOUT> cur = load_row<LAYOUT>(a.src, first * W + col);
        uint32_t cur_edge = edge_lane ? edge_bit<HALF, LAYOUT>(a.src, first, edge_block, W) : 0u;
        for (uint32_t i = 0; i < nrows; ++i) {
            const uint32_t row = row_at(i);
            RowRaw<LAYOUT> nxt{};
            uint32_t nxt_edge = 0;
            if (i + 1 < nrows) {                                      // prefetch the next row
                const uint32_t r = row_at(i + 1);
                nxt = load_row<LAYOUT>(a.src, r * W + col);
                if (edge_lane) nxt_edge = edge_bit<HALF, LAYOUT>(a.src, r, edge_block, W);
            }
            const uint32_t S = row_bits<LAYOUT>(cur), N1 = prev;
            uint32_t N2;
            if (HALF == 0) {
                const uint32_t left = __shfl_up_sync(0xffffffffu, S, 1) >> 31;
                N2 = (S << 1) | (lane == 0 ? cur_edge : left);
            } else {
                const uint32_t right = __shfl_down_sync(0xffffffffu, S, 1) & 1u;
                N2 = (S >> 1) | ((lane == 31 ? cur_edge : right) << 31);
            }
            const uint32_t w = row * W + col;
            const BlockClass k = block_class(S, N1, N2);
            uint32_t und, up;
            draw_first_two(k, w, 0xffffffffu, a.hs, a.P, und, up);
            const bool parked = und != 0u;
            const uint32_t mask = __ballot_sync(0xffffffffu, parked);
            if (parked) {
                const uint32_t qi = (head + count + __popc(mask & below)) & (kQueueCap - 1);
                q[0][qi] = w;
                q[1][qi] = und;
                q[2][qi] = up;
                q[3][qi] = S;
                q[4][qi] = N1;
                q[5][qi] = N2;
            } else {
                finish_block<HALF, LAYOUT>(a, w, up, S, N1, N2, cnn, acc);
            }
            count += __popc(mask);
            if (count >= 32) {
                __syncwarp();
                drain_queue<HALF, LAYOUT>(a, P, q, head, 32, cnn, acc);
                __syncwarp();
                head = (head + 32) & (kQueueCap - 1);
                count -= 32;
            }
            prev = S;
            cur = nxt;
            cur_edge = nxt_edge;
        }
    }
    if (count > 0) {
        __syncwarp();
        drain_queue<HALF, LAYOUT>(a, P, q, head, count, cnn, acc);
    }
    finish_step<HALF>(acc, a);
}

// Strip walk with the rows staged DEPTH rows ahead into a per-warp ring in
// shared memory by cp.async (each lane copies its own block's word or 32
// bytes, lane 0 / 31 also the strip-edge word); otherwise as k_sweep_strip.
template <int LAYOUT>
struct RowWords {
    static constexpr int kWords = LAYOUT == kBitpack ? 1 : 8;   // 32-bit words per lane per row
};

template <int HALF, int LAYOUT, int BLOCK, int MINB, int DEPTH>
__global__ void __launch_bounds__(BLOCK, MINB) k_sweep_strip_async(const SweepArgs a) {
    constexpr int NW = RowWords<LAYOUT>::kWords;
    __shared__ uint32_t qbuf[BLOCK / 32][kQueueFields][kQueueCap];
    const DrawParams& P = a.P;
    __shared__ __align__(16) uint32_t ring[BLOCK / 32][DEPTH][32 * NW];
    __shared__ __align__(16) uint32_t ring_edge[BLOCK / 32][DEPTH][4];
    const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    uint32_t (*q)[kQueueCap] = qbuf[wib];
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[3] = {0, 0, 0};
    uint32_t head = 0;
    int count = 0;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t W = a.Wr, L = a.L;
    const uint32_t nstrips = W / 32;
    const bool edge_lane = HALF == 0 ? lane == 0 : lane == 31;
    const uint64_t total = (uint64_t)nstrips * L;
    uint64_t pos = total * gwarp / nwarps;
    const uint64_t end = total * (gwarp + 1) / nwarps;
    while (pos < end) {
        const uint32_t strip = (uint32_t)(pos / L);
        const uint32_t r0 = (uint32_t)(pos - (uint64_t)strip * L);
        const uint64_t left_here = end - pos, left_in_strip = L - r0;
        const uint32_t nrows = (uint32_t)(left_here < left_in_strip ? left_here : left_in_strip);
        pos += nrows;
        const uint32_t col = strip * 32 + lane;
        const uint32_t edge_block = HALF == 0 ? (strip == 0 ? W - 1 : strip * 32 - 1)
                                              : (strip + 1 == nstrips ? 0 : strip * 32 + 32);
        auto row_at = [&](uint32_t i) -> uint32_t { return HALF == 0 ? r0 + i : r0 + nrows - 1 - i; };
        // stage row i of the walk into ring slot i % DEPTH (always commit a group)
        auto stage = [&](uint32_t i) {
            if (i < nrows) {
                const uint32_t r = row_at(i);
                const size_t b = (size_t)r * W + col;
                uint32_t* dst = &ring[wib][i % DEPTH][lane * NW];
                if constexpr (LAYOUT == kBitpack) {
                    cp_async4(dst, static_cast<const uint32_t*>(a.src) + b);
                } else {
                    const int8_t* g = static_cast<const int8_t*>(a.src) + 32 * b;
                    cp_async16(dst, g);
                    cp_async16(dst + 4, g + 16);
                }
                if (edge_lane) {
                    const size_t eb = (size_t)r * W + edge_block;
                    if constexpr (LAYOUT == kBitpack) {
                        cp_async4(&ring_edge[wib][i % DEPTH][0], static_cast<const uint32_t*>(a.src) + eb);
                    } else {
                        // the 4-byte word holding the byte next to the strip
                        const int8_t* g = static_cast<const int8_t*>(a.src) + 32 * eb + (HALF == 0 ? 28 : 0);
                        cp_async4(&ring_edge[wib][i % DEPTH][0], g);
                    }
                }
            }
            cp_async_commit();
        };
        const uint32_t first = row_at(0);
        const uint32_t nb_row = HALF == 0 ? (first == 0 ? L - 1 : first - 1) : (first + 1 == L ? 0 : first + 1);
        uint32_t prev = row_bits<LAYOUT>(load_row<LAYOUT>(a.src, nb_row * W + col));
        __syncwarp();
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) stage(d);
        for (uint32_t i = 0; i < nrows; ++i) {
            const uint32_t row = row_at(i);
            cp_async_wait<DEPTH - 1>();      // row i has landed (this lane's copies)
            __syncwarp();                    // ... and every other lane's
            const uint32_t* slot = &ring[wib][i % DEPTH][lane * NW];
            uint32_t S;
            if constexpr (LAYOUT == kBitpack) {
                S = slot[0];
            } else {
                const uint4 lo = *reinterpret_cast<const uint4*>(slot);
                const uint4 hi = *reinterpret_cast<const uint4*>(slot + 4);
                S = pack_up32(lo, hi);
            }
            uint32_t edge = 0;
            if (edge_lane) {
                const uint32_t e = ring_edge[wib][i % DEPTH][0];
                if constexpr (LAYOUT == kBitpack) edge = HALF == 0 ? e >> 31 : e & 1u;
                else edge = HALF == 0 ? (uint32_t)((int8_t)(e >> 24) > 0) : (uint32_t)((int8_t)(e & 0xFFu) > 0);
            }
            __syncwarp();                    // everyone has read the slot before it is refilled
            stage(i + DEPTH);
            const uint32_t N1 = prev;
            uint32_t N2;
            if (HALF == 0) {
                const uint32_t left = __shfl_up_sync(0xffffffffu, S, 1) >> 31;
                N2 = (S << 1) | (lane == 0 ? edge : left);
            } else {
                const uint32_t right = __shfl_down_sync(0xffffffffu, S, 1) & 1u;
                N2 = (S >> 1) | ((lane == 31 ? edge : right) << 31);
            }
            const uint32_t w = row * W + col;
            const BlockClass k = block_class(S, N1, N2);
            uint32_t und, up;
            draw_first_two(k, w, 0xffffffffu, a.hs, P, und, up);
            const bool parked = und != 0u;
            const uint32_t mask = __ballot_sync(0xffffffffu, parked);
            if (parked) {
                const uint32_t qi = (head + count + __popc(mask & below)) & (kQueueCap - 1);
                q[0][qi] = w;
                q[1][qi] = und;
                q[2][qi] = up;
                q[3][qi] = S;
                q[4][qi] = N1;
                q[5][qi] = N2;
            } else {
                finish_block<HALF, LAYOUT>(a, w, up, S, N1, N2, cnn, acc);
            }
            count += __popc(mask);
            if (count >= 32) {
                __syncwarp();
                drain_queue<HALF, LAYOUT>(a, P, q, head, 32, cnn, acc);
                __syncwarp();
                head = (head + 32) & (kQueueCap - 1);
                count -= 32;
            }
            prev = S;
        }
        cp_async_wait<0>();                  // no copy may still target the ring
        __syncwarp();
    }
    if (count > 0) {
        __syncwarp();
        drain_queue<HALF, LAYOUT>(a, P, q, head, count, cnn, acc);
    }
    finish_step<HALF>(acc, a);
}

// int8 half-step for any L (site-by-site neighbour gathers; partial last block).
template <int HALF>
__global__ void __launch_bounds__(256) k_sweep_i8g(const SweepArgs a) {
    const int8_t* __restrict__ src = static_cast<const int8_t*>(a.src);
    int8_t* __restrict__ dst = static_cast<int8_t*>(a.dst);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[3] = {0, 0, 0};
    for (uint32_t base = gwarp * 32; base < a.nblocks; base += nwarps * 32) {
        const uint32_t w = base + lane;
        const bool active = w < a.nblocks;
        uint32_t S = 0, N1 = 0, N2 = 0, valid = 0;
        if (active) bytes_generic<HALF>(src, w, a.L, a.N, S, N1, N2, valid);
        const uint32_t up = draw_block(S, N1, N2, w, valid, a.hs, a.P);
        if (active) {
            for (int p = 0; p < 32; ++p)
                if ((valid >> p) & 1u) dst[32 * (int64_t)w + p] = ((up >> p) & 1u) ? 1 : -1;
        }
        accumulate_step<HALF>(acc, up, S, N1, N2, valid, cnn);
    }
    finish_step<HALF>(acc, a);
}

// C_nn = sum sigma_x (sigma_{x down} + sigma_{x left}), equal by translation on
// the torus to sum sigma_x (sigma_{x up} + sigma_{x right}); added to obs_cur[4].
template <int LAYOUT, bool ALIGNED>
__global__ void __launch_bounds__(256) k_cnn(const SweepArgs a) {
    int acc = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < a.nblocks; w += stride) {
        uint32_t S, N1, N2, valid = 0xffffffffu;
        if (LAYOUT == kBitpack) {
            const uint32_t row = fdiv(w, a.div_row);
            words_aligned<0>(static_cast<const uint32_t*>(a.src), w, row, w - row * a.Wr, a.L, a.Wr,
                             a.nblocks, S, N1, N2);
        } else if (ALIGNED) {
            const uint32_t row = fdiv(w, a.div_row);
            bytes_aligned<0>(static_cast<const int8_t*>(a.src), w, row, w - row * a.Wr, a.L, a.Wr,
                             a.nblocks, S, N1, N2);
        } else {
            bytes_generic<0>(static_cast<const int8_t*>(a.src), w, a.L, a.N, S, N1, N2, valid);
        }
        const int nv = __popc(valid);
        acc += 2 * nv - 2 * (__popc((S ^ N1) & valid) + __popc((S ^ N2) & valid));
    }
    const int v[1] = {acc};
    long long* const d[1] = {a.obs_cur ? a.obs_cur + 4 : nullptr};
    block_accumulate<1>(v, d);
}

// ------------------------------------------------------------ diagonal correlations

constexpr int kMaxLags = 8;

struct CorrArgs {
    const uint32_t* plane;
    uint32_t L, Wr, nblocks;
    FastDiv div_row;
    int n_lags;
    uint32_t lag[kMaxLags];
    long long* out;      // [0, n_lags): SW-NE sums, [n_lags, 2 n_lags): NW-SE sums
};

// Bits of sites (i + l .. i + l + 31, row) for the block whose first site is
// i = 32 c, read from a bit-packed row with wrap-around.
__device__ __forceinline__ uint32_t shifted_row_word(const uint32_t* row, uint32_t c, uint32_t l, uint32_t Wr) {
    const uint32_t cw = (c + (l >> 5)) % Wr;
    const uint32_t sh = l & 31u;
    const uint32_t lo = row[cw];
    if (sh == 0) return lo;
    const uint32_t hi = row[cw + 1 == Wr ? 0 : cw + 1];
    return (lo >> sh) | (hi << (32u - sh));
}

// sum_x s_x s_{x+(l,l)} and sum_x s_x s_{x+(l,-l)} for every lag (Section
// 3.3: the SW-NE pair (0,0)-(l,l) and the NW-SE pair (0,l)-(l,0), averaged
// over translations of the torus).
__global__ void __launch_bounds__(256) k_diag_corr(const CorrArgs a) {
    int acc[2 * kMaxLags];
#pragma unroll
    for (int k = 0; k < 2 * kMaxLags; ++k) acc[k] = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < a.nblocks; w += stride) {
        const uint32_t j = fdiv(w, a.div_row), c = w - j * a.Wr;
        const uint32_t s = a.plane[w];
#pragma unroll
        for (int k = 0; k < kMaxLags; ++k) {
            if (k < a.n_lags) {
                const uint32_t l = a.lag[k];
                const uint32_t jp = j + l >= a.L ? j + l - a.L : j + l;
                const uint32_t jm = j >= l ? j - l : j + a.L - l;
                const uint32_t p1 = shifted_row_word(a.plane + (size_t)jp * a.Wr, c, l, a.Wr);
                const uint32_t p2 = shifted_row_word(a.plane + (size_t)jm * a.Wr, c, l, a.Wr);
                acc[k] += 32 - 2 * __popc(s ^ p1);
                acc[kMaxLags + k] += 32 - 2 * __popc(s ^ p2);
            }
        }
    }
    __shared__ long long red[2 * kMaxLags][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 2 * kMaxLags; ++k) {
        const int v = warp_sum(acc[k]);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2 * kMaxLags) {
        const int k = threadIdx.x;
        const int lk = k < kMaxLags ? k : k - kMaxLags;
        if (lk < a.n_lags) {
            long long t = 0;
            for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += red[k][i];
            const int idx = k < kMaxLags ? lk : a.n_lags + lk;
            atomicAdd(reinterpret_cast<unsigned long long*>(a.out + idx), (unsigned long long)t);
        }
    }
}

// ------------------------------------------------------------ checkerboard heat bath

// The square-lattice comparison dynamics of Section 3.2: the sites with
// (i + j) % 2 == parity are redrawn in place, P(+1) = e^h / (2 cosh h) with
// h = J (2n - 4), n the number of + among the four neighbours (all of the
// other parity, so unchanged while the parity is redrawn).  With the
// complement rule the five thresholds fold onto the three-class draw: sites
// with n < 2 compare their complemented uniform, and the class is
// n' = max(n, 4 - n) - 2 with thresholds (T[2], T[3], T[4]).  Returns the
// classes of block w (row, col) of a bit-packed plane and sets pm to the mask
// of its sites of the given parity.
__device__ __forceinline__ BlockClass checkerboard_class(const uint32_t* pl, uint32_t w, uint32_t row,
                                                         uint32_t col, uint32_t L, uint32_t Wr,
                                                         uint32_t nblocks, uint32_t parity, uint32_t& pm) {
    const uint32_t S = pl[w];
    const uint32_t U = pl[row + 1 < L ? w + Wr : w + Wr - nblocks];
    const uint32_t D = pl[row > 0 ? w - Wr : w + nblocks - Wr];
    const uint32_t prev = pl[col > 0 ? w - 1 : w + Wr - 1];
    const uint32_t next = pl[col + 1 < Wr ? w + 1 : w + 1 - Wr];
    const uint32_t Lf = (S << 1) | (prev >> 31);
    const uint32_t Rt = (S >> 1) | (next << 31);
    // n = U + D + Lf + Rt per site, as bits b0 + 2 b1 + 4 b2
    const uint32_t ab_s = U ^ D, ab_c = U & D, cd_s = Lf ^ Rt, cd_c = Lf & Rt;
    const uint32_t b0 = ab_s ^ cd_s, c0 = ab_s & cd_s;
    const uint32_t b1 = ab_c ^ cd_c ^ c0;
    const uint32_t b2 = (ab_c & cd_c) | ((ab_c ^ cd_c) & c0);
    const uint32_t extreme = b2 | ~(b0 | b1 | b2);       // n == 4 or n == 0
    pm = ((row & 1u) == parity) ? 0x55555555u : 0xAAAAAAAAu;
    BlockClass k;
    k.F = ~(b1 | b2);                                   // n < 2
    k.C2 = extreme;
    k.Cg = b0 | extreme;                                // n odd or extreme
    return k;
}

template <int PARITY>
__global__ void __launch_bounds__(256) k_checkerboard(const SweepArgs a) {
    uint32_t* pl = static_cast<uint32_t*>(a.dst);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t base = gwarp * 32; base < a.nblocks; base += nwarps * 32) {
        const uint32_t w = base + lane;
        const uint32_t row = fdiv(w, a.div_row);
        uint32_t pm;
        const BlockClass k = checkerboard_class(pl, w, row, w - row * a.Wr, a.L, a.Wr, a.nblocks, PARITY, pm);
        const uint32_t S = pl[w];
        const uint32_t up = draw_block_class(k, w, pm, a.hs, a.P);
        pl[w] = (S & ~pm) | (up & pm);
    }
}

// ------------------------------------------------------------ coalescence and coupling from the past

struct CoalescePair {
    uint32_t L, Wr, nblocks;
    uint32_t pad;
    DrawParams P;
};

struct CoalesceArgs {
    const CoalescePair* pairs;
    uint32_t n_pairs;
    unsigned long long max_steps;
    unsigned long long* T;      // per pair: first n with sigma_top == sigma_bottom, or max_steps + 1
};

struct CftpArgs {
    const CoalescePair* pairs;
    uint32_t n_pairs;
    int k_max;
    uint32_t* samples;          // per pair: sample_words words (the sigma plane at time 0)
    uint32_t sample_words;
    int* k_out;                 // per pair: k of the successful attempt, or -1
};

// Bits of block w and of its two field neighbours in a bit-packed shared-
// memory plane (rows of Wr words, L rows, wrapping).
template <int HALF>
__device__ __forceinline__ void smem_fields(const uint32_t* pl, uint32_t w, uint32_t Wr, uint32_t L,
                                            uint32_t nblocks, uint32_t& S, uint32_t& N1, uint32_t& N2) {
    const uint32_t row = w / Wr, col = w - row * Wr;
    words_aligned<HALF>(pl, w, row, col, L, Wr, nblocks, S, N1, N2);
}

// Four bit-packed planes of one CTA: sigma and tau of the chain started from
// all + (top) and of the one started from all - (bottom).
struct PairPlanes {
    uint32_t *st, *tt, *sb, *tb;
    uint32_t nb, nbp, Wr, L;
};

__device__ __forceinline__ PairPlanes pair_planes(uint32_t* smem, const CoalescePair& cp) {
    PairPlanes p;
    p.nb = cp.nblocks;
    p.nbp = (cp.nblocks + 31u) & ~31u;
    p.Wr = cp.Wr;
    p.L = cp.L;
    p.st = smem;
    p.tt = smem + p.nbp;
    p.sb = smem + 2 * p.nbp;
    p.tb = smem + 3 * p.nbp;
    return p;
}

__device__ __forceinline__ void pair_reset(const PairPlanes& p) {
    for (uint32_t w = threadIdx.x; w < p.nbp; w += blockDim.x) {
        p.st[w] = w < p.nb ? 0xffffffffu : 0u;
        p.sb[w] = 0u;
        p.tt[w] = p.tb[w] = 0u;
    }
    __syncthreads();
}

// One full step with index t of both chains, driven by the same uniforms
// (shaken: half-steps A and B; checkerboard: even then odd sites of sigma).
template <int DYN>
__device__ __forceinline__ void pair_step(const PairPlanes& p, unsigned long long t, const DrawParams& P) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t hs = (uint32_t)(2 * t);
    for (int half = 0; half < 2; ++half) {
        for (uint32_t base = warp * 32; base < p.nbp; base += nwarps * 32) {
            const uint32_t w = base + lane;
            const bool in = w < p.nb;
            if (DYN == kDynShaken) {
                uint32_t S0 = 0, A0 = 0, B0 = 0, S1 = 0, A1 = 0, B1 = 0;
                if (in) {
                    if (half == 0) {
                        smem_fields<0>(p.st, w, p.Wr, p.L, p.nb, S0, A0, B0);
                        smem_fields<0>(p.sb, w, p.Wr, p.L, p.nb, S1, A1, B1);
                    } else {
                        smem_fields<1>(p.tt, w, p.Wr, p.L, p.nb, S0, A0, B0);
                        smem_fields<1>(p.tb, w, p.Wr, p.L, p.nb, S1, A1, B1);
                    }
                }
                const uint32_t S[2] = {S0, S1}, A[2] = {A0, A1}, B[2] = {B0, B1}, ww[2] = {w, w};
                const uint32_t v[2] = {in ? 0xffffffffu : 0u, in ? 0xffffffffu : 0u};
                uint32_t up[2];
                draw_blocks<2>(S, A, B, ww, v, hs + (uint32_t)half, P, up);
                if (in) {
                    if (half == 0) {
                        p.tt[w] = up[0];
                        p.tb[w] = up[1];
                    } else {
                        p.st[w] = up[0];
                        p.sb[w] = up[1];
                    }
                }
            } else {
                // in place: the words read for the neighbour counts keep the
                // bits of the other parity, which no lane changes now
                uint32_t* planes2[2] = {p.st, p.sb};
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    uint32_t* pl = planes2[c];
                    BlockClass k = {0u, 0u, 0u};
                    uint32_t pm = 0u, S = 0u;
                    if (in) {
                        const uint32_t row = w / p.Wr;
                        k = checkerboard_class(pl, w, row, w - row * p.Wr, p.L, p.Wr, p.nb, (uint32_t)half, pm);
                        S = pl[w];
                    }
                    const uint32_t up = draw_block_class(k, w, pm, hs + (uint32_t)half, P);
                    if (in) pl[w] = (S & ~pm) | (up & pm);
                }
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ bool pair_equal(const PairPlanes& p) {
    uint32_t diff = 0;
    for (uint32_t w = threadIdx.x; w < p.nb; w += blockDim.x) diff |= p.st[w] ^ p.sb[w];
    return !__syncthreads_or(diff != 0u);
}

// Section 3.2: two copies of the chain, from all + (top) and all - (bottom),
// driven by the same random numbers (the same seed, lattice id and steps).
// The order is preserved, and once the sigma planes agree they agree forever;
// T is the first step count n with sigma_top(n) == sigma_bottom(n).  One CTA
// per pair, all four planes in shared memory.
template <int DYN>
__global__ void __launch_bounds__(256) k_coalesce(const CoalesceArgs a) {
    extern __shared__ uint32_t planes[];
    const uint32_t pi = blockIdx.x;
    if (pi >= a.n_pairs) return;
    const CoalescePair& cp = a.pairs[pi];
    const PairPlanes p = pair_planes(planes, cp);
    pair_reset(p);
    unsigned long long T = a.max_steps + 1;
    for (unsigned long long t = 0; t < a.max_steps; ++t) {
        pair_step<DYN>(p, t, cp.P);
        if (pair_equal(p)) {
            T = t + 1;
            break;
        }
    }
    if (threadIdx.x == 0) a.T[pi] = T;
}

// Propp-Wilson coupling from the past (Section 3.2).  The step from time -s
// to -s + 1 always uses forward step index s - 1, so every attempt reuses the
// randomness of the times it shares with the previous one.  Attempt k runs
// both chains from -2^k to 0; the first one after which their sigma planes
// agree gives the sample (its sigma at time 0) and k.  One CTA per pair.
template <int DYN>
__global__ void __launch_bounds__(256) k_cftp(const CftpArgs a) {
    extern __shared__ uint32_t planes[];
    const uint32_t pi = blockIdx.x;
    if (pi >= a.n_pairs) return;
    const CoalescePair& cp = a.pairs[pi];
    const PairPlanes p = pair_planes(planes, cp);
    int result = -1;
    for (int k = 0; k <= a.k_max; ++k) {
        pair_reset(p);
        for (unsigned long long s = 1ull << k; s >= 1; --s) pair_step<DYN>(p, s - 1, cp.P);
        if (pair_equal(p)) {
            result = k;
            break;
        }
    }
    uint32_t* out = a.samples + (size_t)pi * a.sample_words;
    for (uint32_t w = threadIdx.x; w < a.sample_words; w += blockDim.x)
        out[w] = (result >= 0 && w < p.nb) ? p.st[w] : 0u;
    if (threadIdx.x == 0) a.k_out[pi] = result;
}

// Magnetisation and C_nn = sum_x s_x (s_{x down} + s_{x left}) (equal by
// translation to the up/right form) of a bit-packed plane, added to out[0..1].
__global__ void __launch_bounds__(256) k_sq_obs(const SweepArgs a) {
    int m = 0, c = 0;
    const uint32_t* pl = static_cast<const uint32_t*>(a.src);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < a.nblocks; w += stride) {
        const uint32_t row = fdiv(w, a.div_row);
        uint32_t S, N1, N2;
        words_aligned<0>(pl, w, row, w - row * a.Wr, a.L, a.Wr, a.nblocks, S, N1, N2);
        m += 2 * __popc(S) - 32;
        c += 64 - 2 * (__popc(S ^ N1) + __popc(S ^ N2));
    }
    const int v[2] = {m, c};
    long long* const d[2] = {a.obs_cur, a.obs_cur ? a.obs_cur + 1 : nullptr};
    block_accumulate<2>(v, d);
}

// ------------------------------------------------------------ initial states

struct InitArgs {
    void* plane;
    uint32_t L;
    uint32_t nblocks;
    int64_t N;
    int kind;
    uint32_t plane_index;
    DrawParams P;   // only the round keys, lattice id and c3_base are used
};

template <int LAYOUT>
__global__ void __launch_bounds__(256) k_init(const InitArgs a) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < a.nblocks; w += stride) {
        uint32_t bits;
        if (a.kind == 0) {
            bits = 0xffffffffu;
        } else if (a.kind == 1) {
            bits = 0u;
        } else {
            // r(u) < 2^31 iff the most significant bit of r(u) is 0, i.e. bit
            // p of the first Philox word of the block is 0.
            uint32_t x0 = a.plane_index, x1 = w, x2 = a.P.lattice_id, x3 = a.P.c3_base;
            philox10(x0, x1, x2, x3, a.P);
            bits = ~x0;
        }
        const int64_t rem = a.N - 32 * (int64_t)w;
        const uint32_t valid = rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
        bits &= valid;
        if (LAYOUT == kBitpack) {
            static_cast<uint32_t*>(a.plane)[w] = bits;
        } else if (valid == 0xffffffffu && ((a.L & 31u) == 0u)) {
            uint4 lo, hi;
            unpack32(bits, lo, hi);
            uint4* d4 = reinterpret_cast<uint4*>(static_cast<int8_t*>(a.plane) + 32 * (size_t)w);
            d4[0] = lo;
            d4[1] = hi;
        } else {
            int8_t* d = static_cast<int8_t*>(a.plane);
            for (int p = 0; p < 32; ++p)
                if ((valid >> p) & 1u) d[32 * (int64_t)w + p] = ((bits >> p) & 1u) ? 1 : -1;
        }
    }
}

// ------------------------------------------------------------ small lattices

struct SmallArgs {
    void* sigma;
    void* tau;
    uint32_t L;
    uint32_t Wr;
    uint32_t nblocks;
    uint32_t nbp;       // nblocks rounded up to a multiple of 32
    int64_t N;
    int aligned;
    FastDiv div_row;
    uint64_t t0;
    uint32_t n;
    long long* obs;     // n rows of five sums, nullable
    long long* last;    // last row, nullable
    DrawParams P;
};

template <int HALF>
__device__ __forceinline__ void small_fields(const uint32_t* pl, uint32_t w, const SmallArgs& a,
                                             uint32_t& S, uint32_t& N1, uint32_t& N2,
                                             uint32_t& valid) {
    if (w >= a.nblocks) {
        S = N1 = N2 = valid = 0;
    } else if (a.aligned) {
        const uint32_t row = fdiv(w, a.div_row);
        words_aligned<HALF>(pl, w, row, w - row * a.Wr, a.L, a.Wr, a.nblocks, S, N1, N2);
        valid = 0xffffffffu;
    } else {
        words_generic<HALF>(pl, w, a.L, a.N, S, N1, N2, valid);
    }
}

template <int LAYOUT>
__global__ void __launch_bounds__(1024) k_run_small(const SmallArgs a) {
    extern __shared__ uint32_t sm_planes[];
    uint32_t* sg = sm_planes;
    uint32_t* tu = sm_planes + a.nbp;
    __shared__ long long red[kNumObs][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;

    // load both planes as bits
    for (uint32_t w = threadIdx.x; w < a.nbp; w += blockDim.x) {
        uint32_t bs = 0, bt = 0;
        if (w < a.nblocks) {
            if (LAYOUT == kBitpack) {
                bs = static_cast<const uint32_t*>(a.sigma)[w];
                bt = static_cast<const uint32_t*>(a.tau)[w];
            } else {
                const int8_t* s8 = static_cast<const int8_t*>(a.sigma);
                const int8_t* t8 = static_cast<const int8_t*>(a.tau);
                for (int p = 0; p < 32; ++p) {
                    const int64_t u = 32 * (int64_t)w + p;
                    if (u >= a.N) break;
                    bs |= (uint32_t)(s8[u] > 0) << p;
                    bt |= (uint32_t)(t8[u] > 0) << p;
                }
            }
        }
        sg[w] = bs;
        tu[w] = bt;
    }
    __syncthreads();

    for (uint32_t s = 0; s < a.n; ++s) {
        const uint64_t t = a.t0 + s;
        const uint32_t hs = (uint32_t)(2 * t);
        for (uint32_t base = warp * 32; base < a.nbp; base += nwarps * 32) {
            const uint32_t w = base + lane;
            uint32_t S, N1, N2, valid;
            small_fields<0>(sg, w, a, S, N1, N2, valid);
            const uint32_t up = draw_block(S, N1, N2, w, valid, hs, a.P);
            if (w < a.nblocks) tu[w] = up;
        }
        __syncthreads();
        for (uint32_t base = warp * 32; base < a.nbp; base += nwarps * 32) {
            const uint32_t w = base + lane;
            uint32_t S, N1, N2, valid;
            small_fields<1>(tu, w, a, S, N1, N2, valid);
            const uint32_t up = draw_block(S, N1, N2, w, valid, hs + 1, a.P);
            if (w < a.nblocks) sg[w] = up;
        }
        __syncthreads();
        if (a.obs == nullptr && s + 1 < a.n) continue;
        // observables of (sigma_t, tau_t)
        int v[kNumObs] = {0, 0, 0, 0, 0};
        for (uint32_t w = threadIdx.x; w < a.nblocks; w += blockDim.x) {
            uint32_t Sg, SgU, SgR, Tu, TuU, TuR, valid;
            small_fields<1>(sg, w, a, Sg, SgU, SgR, valid);
            small_fields<1>(tu, w, a, Tu, TuU, TuR, valid);
            const int nv = __popc(valid);
            v[0] += 2 * __popc(Sg) - nv;
            v[1] += 2 * __popc(Tu) - nv;
            v[2] += nv - 2 * __popc((Sg ^ Tu) & valid);
            v[3] += 2 * nv - 2 * (__popc((Sg ^ TuU) & valid) + __popc((Sg ^ TuR) & valid));
            v[4] += 2 * nv - 2 * (__popc((Sg ^ SgU) & valid) + __popc((Sg ^ SgR) & valid));
        }
#pragma unroll
        for (int i = 0; i < kNumObs; ++i) {
            const int r = warp_sum(v[i]);
            if (lane == 0) red[i][warp] = r;
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int i = 0; i < kNumObs; ++i) {
                long long r = lane < nwarps ? red[i][lane] : 0;
                r = warp_sum64(r);
                if (lane == 0) {
                    if (a.obs) a.obs[(size_t)s * kNumObs + i] = r;
                    if (s + 1 == a.n && a.last) a.last[i] = r;
                }
            }
        }
        __syncthreads();
    }

    // store both planes back
    for (uint32_t w = threadIdx.x; w < a.nblocks; w += blockDim.x) {
        if (LAYOUT == kBitpack) {
            static_cast<uint32_t*>(a.sigma)[w] = sg[w];
            static_cast<uint32_t*>(a.tau)[w] = tu[w];
        } else {
            int8_t* s8 = static_cast<int8_t*>(a.sigma);
            int8_t* t8 = static_cast<int8_t*>(a.tau);
            for (int p = 0; p < 32; ++p) {
                const int64_t u = 32 * (int64_t)w + p;
                if (u >= a.N) break;
                s8[u] = ((sg[w] >> p) & 1u) ? 1 : -1;
                t8[u] = ((tu[w] >> p) & 1u) ? 1 : -1;
            }
        }
    }
}

// ------------------------------------------------------------ host side

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Resident blocks per SM of a kernel at a block size, queried once per kernel.
static int blocks_per_sm(const void* kernel, int block) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(kernel);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
    if (per_sm <= 0) per_sm = 1;
    cache.emplace(kernel, per_sm);
    return per_sm;
}

// Grid of at most one full wave of resident blocks (the kernels stride over
// their work), never more blocks than work items need.
template <class K>
static int grid_for(K kernel, int block, uint64_t work_items) {
    const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(kernel), block);
    const uint64_t full = (uint64_t)per_sm * sm_count();
    const uint64_t need = (work_items + block - 1) / block;
    return (int)std::max<uint64_t>(1, std::min(full, need));
}

static SweepArgs sweep_args(const Geometry& g, const void* src, void* dst, const DrawParams& P,
                            uint32_t hs, long long* oc, long long* op, long long* z) {
    SweepArgs a;
    a.src = src;
    a.dst = dst;
    a.L = (uint32_t)g.L;
    a.Wr = g.Wr;
    a.nblocks = g.nblocks;
    a.N = g.N;
    a.div_row = make_fastdiv(g.Wr > 0 ? g.Wr : 1);
    a.hs = hs;
    a.obs_cur = oc;
    a.obs_prev = op;
    a.zero_slot = z;
    a.P = P;
    return a;
}

// ------------------------------------------------------------ sweep variants
//
// Launch shapes of the half-step sweeps, chosen per layout at run time
// (shk_set_sweep_variant; the autotuner times them and picks one).

using SweepKernel = void (*)(SweepArgs);

struct SweepVariant {
    SweepKernel k[2];   // half A, half B
    int block;
    bool strip;         // needs rows of a multiple of 32 blocks (L % 1024 == 0)
    const char* name;
};

// The first entry of each table is the default (the fastest measured at
// L = 16384 on GB300); the autotuner may pick another per size.
static const SweepVariant kBpVariants[] = {
    {{k_sweep_q<0, kBitpack, 256, 3>, k_sweep_q<1, kBitpack, 256, 3>}, 256, false, "queue-256x3"},
    {{k_sweep_strip_async<0, kBitpack, 256, 3, 4>, k_sweep_strip_async<1, kBitpack, 256, 3, 4>}, 256, true,
     "strip-async4-256x3"},
    {{k_sweep_strip<0, kBitpack, 256, 3>, k_sweep_strip<1, kBitpack, 256, 3>}, 256, true, "strip-256x3"},
    {{k_sweep_q<0, kBitpack, 128, 6>, k_sweep_q<1, kBitpack, 128, 6>}, 128, false, "queue-128x6"},
    {{k_sweep_q<0, kBitpack, 256, 4>, k_sweep_q<1, kBitpack, 256, 4>}, 256, false, "queue-256x4"},
    {{k_sweep_bp<0, 1, false, 256, 1>, k_sweep_bp<1, 1, false, 256, 1>}, 256, false, "plain-256"},
};

static const SweepVariant kI8Variants[] = {
    {{k_sweep_strip_async<0, kInt8, 256, 3, 2>, k_sweep_strip_async<1, kInt8, 256, 3, 2>}, 256, true,
     "strip-async2-256x3"},
    {{k_sweep_strip<0, kInt8, 256, 3>, k_sweep_strip<1, kInt8, 256, 3>}, 256, true, "strip-256x3"},
    {{k_sweep_q<0, kInt8, 256, 3>, k_sweep_q<1, kInt8, 256, 3>}, 256, false, "queue-256x3"},
    {{k_sweep_q<0, kInt8, 256, 4>, k_sweep_q<1, kInt8, 256, 4>}, 256, false, "queue-256x4"},
    {{k_sweep_i8a<0, false, 256, 1>, k_sweep_i8a<1, false, 256, 1>}, 256, false, "plain-256"},
};

constexpr int kNumBpVariants = sizeof(kBpVariants) / sizeof(kBpVariants[0]);
constexpr int kNumI8Variants = sizeof(kI8Variants) / sizeof(kI8Variants[0]);
constexpr int kBpRowFallback = 0;   // non-strip variant used when rows are too short
constexpr int kI8RowFallback = 2;

static std::atomic<int> g_bp_variant{0};
static std::atomic<int> g_i8_variant{0};

int sweep_variant_count(int layout) {
    return layout == kBitpack ? kNumBpVariants : layout == kInt8 ? kNumI8Variants : 0;
}

const char* sweep_variant_name(int layout, int v) {
    if (v < 0 || v >= sweep_variant_count(layout)) return nullptr;
    return layout == kBitpack ? kBpVariants[v].name : kI8Variants[v].name;
}

int get_sweep_variant(int layout) {
    return layout == kBitpack ? g_bp_variant.load() : g_i8_variant.load();
}

bool set_sweep_variant(int layout, int v) {
    if (v < 0 || v >= sweep_variant_count(layout)) return false;
    (layout == kBitpack ? g_bp_variant : g_i8_variant).store(v);
    return true;
}

cudaError_t launch_halfstep(const Geometry& g, int half, const void* src, void* dst,
                            const DrawParams& P, uint32_t hs, long long* obs_cur,
                            long long* obs_prev, long long* zero_slot, cudaStream_t st) {
    SweepArgs a = sweep_args(g, src, dst, P, hs, obs_cur, half == 0 ? obs_prev : nullptr, zero_slot);
    if (g.layout == kBitpack || g.aligned) {
        const SweepVariant* table = g.layout == kBitpack ? kBpVariants : kI8Variants;
        int vi = g.layout == kBitpack ? g_bp_variant.load() : g_i8_variant.load();
        // strip-walk variants need rows of a multiple of 32 blocks (L % 1024 == 0)
        if (table[vi].strip && (g.Wr % 32) != 0) vi = g.layout == kBitpack ? kBpRowFallback : kI8RowFallback;
        const SweepVariant& v = table[vi];
        SweepKernel k = v.k[half];
        const int grid = grid_for(k, v.block, g.nblocks);
        k<<<grid, v.block, 0, st>>>(a);
    } else {
        const int block = 256;
        if (half == 0) {
            k_sweep_i8g<0><<<grid_for(k_sweep_i8g<0>, block, g.nblocks), block, 0, st>>>(a);
        } else {
            k_sweep_i8g<1><<<grid_for(k_sweep_i8g<1>, block, g.nblocks), block, 0, st>>>(a);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_cnn(const Geometry& g, const void* sigma, long long* obs, cudaStream_t st) {
    DrawParams P{};
    const SweepArgs a = sweep_args(g, sigma, nullptr, P, 0, obs, nullptr, nullptr);
    const int block = 256;
    if (g.layout == kBitpack) {
        k_cnn<kBitpack, true><<<grid_for(k_cnn<kBitpack, true>, block, g.nblocks), block, 0, st>>>(a);
    } else if (g.aligned) {
        k_cnn<kInt8, true><<<grid_for(k_cnn<kInt8, true>, block, g.nblocks), block, 0, st>>>(a);
    } else {
        k_cnn<kInt8, false><<<grid_for(k_cnn<kInt8, false>, block, g.nblocks), block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_init(const Geometry& g, void* plane, int kind, uint64_t init_seed,
                        uint32_t lattice_id, uint32_t plane_index, cudaStream_t st) {
    InitArgs a;
    a.plane = plane;
    a.L = (uint32_t)g.L;
    a.nblocks = g.nblocks;
    a.N = g.N;
    a.kind = kind;
    a.plane_index = plane_index;
    const uint32_t dummyT[6] = {0x80000000u, 0x80000000u, 0x80000000u,
                                0x80000000u, 0x80000000u, 0x80000000u};
    make_draw_params(init_seed, lattice_id, dummyT, 1u, &a.P);
    const int block = 256;
    if (g.layout == kBitpack) {
        k_init<kBitpack><<<grid_for(k_init<kBitpack>, block, g.nblocks), block, 0, st>>>(a);
    } else {
        k_init<kInt8><<<grid_for(k_init<kInt8>, block, g.nblocks), block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_diag_corr(const Geometry& g, const void* plane, const int* lags, int n_lags, long long* out,
                             cudaStream_t st) {
    CorrArgs a;
    a.plane = static_cast<const uint32_t*>(plane);
    a.L = (uint32_t)g.L;
    a.Wr = g.Wr;
    a.nblocks = g.nblocks;
    a.div_row = make_fastdiv(g.Wr);
    a.n_lags = n_lags;
    for (int k = 0; k < kMaxLags; ++k) a.lag[k] = k < n_lags ? (uint32_t)lags[k] : 0u;
    a.out = out;
    k_diag_corr<<<grid_for(k_diag_corr, 256, g.nblocks), 256, 0, st>>>(a);
    return cudaGetLastError();
}

size_t coalesce_smem_bytes(int L) { return 4 * (size_t)(((L * L / 32) + 31) & ~31) * 4; }

template <class K>
static cudaError_t allow_smem(K kernel, size_t smem) {
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

cudaError_t launch_coalesce(int dyn, const void* pairs, uint32_t n_pairs, int max_L, uint64_t max_steps,
                            unsigned long long* T, cudaStream_t st) {
    CoalesceArgs a;
    a.pairs = static_cast<const CoalescePair*>(pairs);
    a.n_pairs = n_pairs;
    a.max_steps = max_steps;
    a.T = T;
    const size_t smem = coalesce_smem_bytes(max_L);
    cudaError_t e;
    if (dyn == kDynShaken) {
        e = allow_smem(k_coalesce<kDynShaken>, smem);
        if (e == cudaSuccess) k_coalesce<kDynShaken><<<n_pairs, 256, smem, st>>>(a);
    } else {
        e = allow_smem(k_coalesce<kDynCheckerboard>, smem);
        if (e == cudaSuccess) k_coalesce<kDynCheckerboard><<<n_pairs, 256, smem, st>>>(a);
    }
    return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t launch_cftp(int dyn, const void* pairs, uint32_t n_pairs, int max_L, int k_max, uint32_t* samples,
                        uint32_t sample_words, int* k_out, cudaStream_t st) {
    CftpArgs a;
    a.pairs = static_cast<const CoalescePair*>(pairs);
    a.n_pairs = n_pairs;
    a.k_max = k_max;
    a.samples = samples;
    a.sample_words = sample_words;
    a.k_out = k_out;
    const size_t smem = coalesce_smem_bytes(max_L);
    cudaError_t e;
    if (dyn == kDynShaken) {
        e = allow_smem(k_cftp<kDynShaken>, smem);
        if (e == cudaSuccess) k_cftp<kDynShaken><<<n_pairs, 256, smem, st>>>(a);
    } else {
        e = allow_smem(k_cftp<kDynCheckerboard>, smem);
        if (e == cudaSuccess) k_cftp<kDynCheckerboard><<<n_pairs, 256, smem, st>>>(a);
    }
    return e == cudaSuccess ? cudaGetLastError() : e;
}

size_t coalesce_pair_bytes() { return sizeof(CoalescePair); }

void fill_coalesce_pair(void* dst, int L, const DrawParams& P) {
    CoalescePair* c = static_cast<CoalescePair*>(dst);
    c->L = (uint32_t)L;
    c->Wr = (uint32_t)L / 32;
    c->nblocks = (uint32_t)((int64_t)L * L / 32);
    c->pad = 0;
    c->P = P;
}

cudaError_t launch_checkerboard(const Geometry& g, void* plane, const DrawParams& P, uint32_t hs, int parity,
                                long long* obs, cudaStream_t st) {
    SweepArgs a = sweep_args(g, plane, plane, P, hs, obs, nullptr, nullptr);
    const int block = 256;
    if (parity == 0) {
        k_checkerboard<0><<<grid_for(k_checkerboard<0>, block, g.nblocks), block, 0, st>>>(a);
    } else {
        k_checkerboard<1><<<grid_for(k_checkerboard<1>, block, g.nblocks), block, 0, st>>>(a);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && obs != nullptr && parity == 1)
        k_sq_obs<<<grid_for(k_sq_obs, block, g.nblocks), block, 0, st>>>(a);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

static uint32_t small_block_threads(const Geometry& g) {
    const uint32_t nbp = (g.nblocks + 31u) & ~31u;
    return std::min<uint32_t>(1024u, std::max<uint32_t>(32u, nbp));
}

bool small_path_fits(const Geometry& g) {
    // Lattices up to 2^16 sites per plane (L <= 256) run faster inside one CTA
    // than as a sequence of grid-wide launches.
    return g.N <= 65536;
}

cudaError_t launch_run_small(const Geometry& g, void* sigma, void* tau, const DrawParams& P,
                             uint64_t t0, uint64_t n, long long* obs, long long* last,
                             cudaStream_t st) {
    SmallArgs a;
    a.sigma = sigma;
    a.tau = tau;
    a.L = (uint32_t)g.L;
    a.Wr = g.Wr;
    a.nblocks = g.nblocks;
    a.nbp = (g.nblocks + 31u) & ~31u;
    a.N = g.N;
    a.aligned = g.aligned ? 1 : 0;
    a.div_row = make_fastdiv(g.Wr > 0 ? g.Wr : 1);
    a.t0 = t0;
    a.n = (uint32_t)n;
    a.obs = obs;
    a.last = last;
    a.P = P;
    const uint32_t threads = small_block_threads(g);
    const size_t smem = 2 * (size_t)a.nbp * sizeof(uint32_t);
    if (g.layout == kBitpack) {
        k_run_small<kBitpack><<<1, threads, smem, st>>>(a);
    } else {
        k_run_small<kInt8><<<1, threads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace shk
