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
//   k_sweep_q, k_sweep_strip[_async]  the two-phase and strip-walk forms of
//                          the half-step (the launch-shape variants)
//
// The Section 3 kernels (correlations, coalescence, coupling from the past,
// the checkerboard chain) live in sampling.cu.
//
// Each thread owns 32-site blocks (one bit-packed word); a warp walks 32
// consecutive blocks together so that the lazy random-plane loop of
// draw_block() can exit as soon as the whole warp is decided.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>
#include <unordered_map>

#define SHK_TU_ID 1
#include "internal.h"
#include "sweep.cuh"

namespace shk {

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
    r.s = __ldg(checked(src, w, a.nblocks, SHK_SITE));
    if (HALF == 0) {
        r.n = __ldg(checked(src, row > 0 ? w - a.Wr : w + a.nblocks - a.Wr, a.nblocks, SHK_SITE));
        r.x = __ldg(checked(src, col > 0 ? w - 1 : w + a.Wr - 1, a.nblocks, SHK_SITE));
    } else {
        r.n = __ldg(checked(src, row + 1 < a.L ? w + a.Wr : w + a.Wr - a.nblocks, a.nblocks, SHK_SITE));
        r.x = __ldg(checked(src, col + 1 < a.Wr ? w + 1 : w + 1 - a.Wr, a.nblocks, SHK_SITE));
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
                *checked(dst, w[k], a.nblocks, SHK_SITE) = up[k];
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
    const uint4* q4 = reinterpret_cast<const uint4*>(src);      // 16-byte chunks, two per block
    const uint64_t n4 = 2 * (uint64_t)a.nblocks;
    r.s0 = __ldg(checked(q4, 2 * (uint64_t)w, n4, SHK_SITE));
    r.s1 = __ldg(checked(q4, 2 * (uint64_t)w + 1, n4, SHK_SITE));
    const uint32_t wn = HALF == 0 ? (row > 0 ? w - a.Wr : w + a.nblocks - a.Wr)
                                  : (row + 1 < a.L ? w + a.Wr : w + a.Wr - a.nblocks);
    r.n0 = __ldg(checked(q4, 2 * (uint64_t)wn, n4, SHK_SITE));
    r.n1 = __ldg(checked(q4, 2 * (uint64_t)wn + 1, n4, SHK_SITE));
    size_t idx;
    if (HALF == 0) idx = col > 0 ? 32 * (size_t)w - 1 : 32 * (size_t)w + a.L - 1;
    else idx = col + 1 < a.Wr ? 32 * (size_t)w + 32 : 32 * (size_t)w + 32 - a.L;
    r.x = __ldg(checked(src, idx, 32 * (uint64_t)a.nblocks, SHK_SITE));
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
        uint4* q4 = reinterpret_cast<uint4*>(dst);
        *checked(q4, 2 * (uint64_t)w, 2 * (uint64_t)a.nblocks, SHK_SITE) = lo;
        *checked(q4, 2 * (uint64_t)w + 1, 2 * (uint64_t)a.nblocks, SHK_SITE) = hi;
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
        *checked(static_cast<uint32_t*>(a.dst), w, a.nblocks, SHK_SITE) = up;
    } else {
        uint4 lo, hi;
        unpack32(up, lo, hi);
        uint4* q4 = reinterpret_cast<uint4*>(a.dst);
        *checked(q4, 2 * (uint64_t)w, 2 * (uint64_t)a.nblocks, SHK_SITE) = lo;
        *checked(q4, 2 * (uint64_t)w + 1, 2 * (uint64_t)a.nblocks, SHK_SITE) = hi;
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
    const uint32_t res = draw_rest_pre(k, w, und, up, a.pre, P);
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
        draw_first_two_pre(k, w, 0xffffffffu, a.pre, P, und, up);
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
__device__ __forceinline__ RowRaw<LAYOUT> load_row(const void* src, uint32_t w, uint32_t nblocks) {
    RowRaw<LAYOUT> r;
    if constexpr (LAYOUT == kBitpack) {
        r.v = __ldg(checked(static_cast<const uint32_t*>(src), w, nblocks, SHK_SITE));
    } else {
        const uint4* q4 = reinterpret_cast<const uint4*>(src);
        r.lo = __ldg(checked(q4, 2 * (uint64_t)w, 2 * (uint64_t)nblocks, SHK_SITE));
        r.hi = __ldg(checked(q4, 2 * (uint64_t)w + 1, 2 * (uint64_t)nblocks, SHK_SITE));
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
__device__ __forceinline__ uint32_t edge_bit(const void* src, uint32_t row, uint32_t edge_block, uint32_t W,
                                             uint32_t nblocks) {
    const size_t b = (size_t)row * W + edge_block;
    if constexpr (LAYOUT == kBitpack) {
        const uint32_t v = __ldg(checked(static_cast<const uint32_t*>(src), b, nblocks, SHK_SITE));
        return HALF == 0 ? v >> 31 : v & 1u;
    } else {
        const int8_t* p = static_cast<const int8_t*>(src);
        return (uint32_t)(__ldg(checked(p, 32 * b + (HALF == 0 ? 31 : 0), 32 * (uint64_t)nblocks, SHK_SITE)) > 0);
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
        uint32_t prev = row_bits<LAYOUT>(load_row<LAYOUT>(a.src, nb_row * W + col, a.nblocks));
        RowRaw<LAYOUT> cur = load_row<LAYOUT>(a.src, first * W + col, a.nblocks);
        uint32_t cur_edge = edge_lane ? edge_bit<HALF, LAYOUT>(a.src, first, edge_block, W, a.nblocks) : 0u;
        for (uint32_t i = 0; i < nrows; ++i) {
            const uint32_t row = row_at(i);
            RowRaw<LAYOUT> nxt{};
            uint32_t nxt_edge = 0;
            if (i + 1 < nrows) {                                      // prefetch the next row
                const uint32_t r = row_at(i + 1);
                nxt = load_row<LAYOUT>(a.src, r * W + col, a.nblocks);
                if (edge_lane) nxt_edge = edge_bit<HALF, LAYOUT>(a.src, r, edge_block, W, a.nblocks);
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
            draw_first_two_pre(k, w, 0xffffffffu, a.pre, a.P, und, up);
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
                    cp_async4(dst, checked(static_cast<const uint32_t*>(a.src), b, a.nblocks, SHK_SITE));
                } else {
                    const uint4* q4 = reinterpret_cast<const uint4*>(a.src);
                    cp_async16(dst, checked(q4, 2 * b, 2 * (uint64_t)a.nblocks, SHK_SITE));
                    cp_async16(dst + 4, checked(q4, 2 * b + 1, 2 * (uint64_t)a.nblocks, SHK_SITE));
                }
                if (edge_lane) {
                    const size_t eb = (size_t)r * W + edge_block;
                    if constexpr (LAYOUT == kBitpack) {
                        cp_async4(&ring_edge[wib][i % DEPTH][0],
                                  checked(static_cast<const uint32_t*>(a.src), eb, a.nblocks, SHK_SITE));
                    } else {
                        // the 4-byte word holding the byte next to the strip
                        const uint32_t* q1 = reinterpret_cast<const uint32_t*>(a.src);
                        cp_async4(&ring_edge[wib][i % DEPTH][0],
                                  checked(q1, 8 * eb + (HALF == 0 ? 7 : 0), 8 * (uint64_t)a.nblocks, SHK_SITE));
                    }
                }
            }
            cp_async_commit();
        };
        const uint32_t first = row_at(0);
        const uint32_t nb_row = HALF == 0 ? (first == 0 ? L - 1 : first - 1) : (first + 1 == L ? 0 : first + 1);
        uint32_t prev = row_bits<LAYOUT>(load_row<LAYOUT>(a.src, nb_row * W + col, a.nblocks));
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
            draw_first_two_pre(k, w, 0xffffffffu, a.pre, P, und, up);
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
                if ((valid >> p) & 1u)
                    *checked(dst, 32 * (uint64_t)w + p, (uint64_t)a.N, SHK_SITE) = ((up >> p) & 1u) ? 1 : -1;
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
            *checked(static_cast<uint32_t*>(a.plane), w, a.nblocks, SHK_SITE) = bits;
        } else if (valid == 0xffffffffu && ((a.L & 31u) == 0u)) {
            uint4 lo, hi;
            unpack32(bits, lo, hi);
            uint4* q4 = reinterpret_cast<uint4*>(a.plane);
            *checked(q4, 2 * (uint64_t)w, 2 * (uint64_t)a.nblocks, SHK_SITE) = lo;
            *checked(q4, 2 * (uint64_t)w + 1, 2 * (uint64_t)a.nblocks, SHK_SITE) = hi;
        } else {
            int8_t* d = static_cast<int8_t*>(a.plane);
            for (int p = 0; p < 32; ++p)
                if ((valid >> p) & 1u)
                    *checked(d, 32 * (uint64_t)w + p, (uint64_t)a.N, SHK_SITE) = ((bits >> p) & 1u) ? 1 : -1;
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
                bs = *checked(static_cast<const uint32_t*>(a.sigma), w, a.nblocks, SHK_SITE);
                bt = *checked(static_cast<const uint32_t*>(a.tau), w, a.nblocks, SHK_SITE);
            } else {
                const int8_t* s8 = static_cast<const int8_t*>(a.sigma);
                const int8_t* t8 = static_cast<const int8_t*>(a.tau);
                for (int p = 0; p < 32; ++p) {
                    const int64_t u = 32 * (int64_t)w + p;
                    if (u >= a.N) break;
                    bs |= (uint32_t)(*checked(s8, (uint64_t)u, (uint64_t)a.N, SHK_SITE) > 0) << p;
                    bt |= (uint32_t)(*checked(t8, (uint64_t)u, (uint64_t)a.N, SHK_SITE) > 0) << p;
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
            *checked(static_cast<uint32_t*>(a.sigma), w, a.nblocks, SHK_SITE) = sg[w];
            *checked(static_cast<uint32_t*>(a.tau), w, a.nblocks, SHK_SITE) = tu[w];
        } else {
            int8_t* s8 = static_cast<int8_t*>(a.sigma);
            int8_t* t8 = static_cast<int8_t*>(a.tau);
            for (int p = 0; p < 32; ++p) {
                const int64_t u = 32 * (int64_t)w + p;
                if (u >= a.N) break;
                *checked(s8, (uint64_t)u, (uint64_t)a.N, SHK_SITE) = ((sg[w] >> p) & 1u) ? 1 : -1;
                *checked(t8, (uint64_t)u, (uint64_t)a.N, SHK_SITE) = ((tu[w] >> p) & 1u) ? 1 : -1;
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
int blocks_per_sm(const void* kernel, int block) {
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

// Host side of PhiloxPrefix: the uniform words of rounds 1 to 3 of call c.
static PhiloxPrefix philox_prefix(const DrawParams& P, uint32_t hs, int c) {
    const uint64_t p0 = (uint64_t)kPhiloxM0 * hs, p1 = (uint64_t)kPhiloxM1 * P.lattice_id;
    const uint32_t c1 = (uint32_t)p1, c3 = (uint32_t)p0;
    const uint32_t c2 = (uint32_t)(p0 >> 32) ^ (P.c3_base + (uint32_t)c) ^ P.rk1[0];
    const uint64_t q1 = (uint64_t)kPhiloxM1 * c2;
    const uint32_t B = (uint32_t)(q1 >> 32) ^ c1 ^ P.rk0[1];
    const uint64_t q0 = (uint64_t)kPhiloxM0 * B;
    PhiloxPrefix u;
    u.A = (uint32_t)(p1 >> 32) ^ P.rk0[0];
    u.K2 = c3 ^ P.rk1[1];
    u.K3 = (uint32_t)q1 ^ P.rk0[2];
    u.H3 = (uint32_t)(q0 >> 32) ^ P.rk1[2];
    u.D = (uint32_t)q0;
    return u;
}

SweepArgs sweep_args(const Geometry& g, const void* src, void* dst, const DrawParams& P,
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
    for (int c = 0; c < 8; ++c) a.pre[c] = philox_prefix(P, hs, c);
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

unsigned bounds_site_kernels() { return take_bounds_site(); }

}  // namespace shk
