// sweep_kernels.cuh -- the half-step sweep kernels (Eqs. leftTrans /
// rightTrans over a whole plane, the fused observable sums) and their device
// helpers: the per-block ILP sweeps (k_sweep_bp, k_sweep_i8a), the two-phase
// sweep with the warp queue (k_sweep_q) and its vector-load form
// (k_sweep_qv), the strip walks (k_sweep_strip,
// k_sweep_strip_async), the generic-L int8 sweep (k_sweep_i8g) and the C_nn
// tail pass (k_cnn).  Device code only: kernels.cu instantiates them for the
// launch-shape tables, and jit.cu compiles the same text at run time for one
// threshold table.
#pragma once

#include "sweep.cuh"

namespace shk {

// ------------------------------------------------------------ half-step sweeps

// Per-thread sums of a half-step, kept as raw counts and turned into the
// signed sums once per thread (finish_step): acc[0] = up sites drawn,
// acc[1] and acc[2] = disagreeing pairs (A: sigma with its down and left
// neighbours, for C_nn; B: sigma with tau, for S_q, and sigma with tau's up
// and right neighbours, for S_J), acc[3] = sites drawn.  With a full valid
// mask the masking and the site count fold to constants.
template <int HALF>
__device__ __forceinline__ void accumulate_step(int (&acc)[4], uint32_t up, uint32_t S, uint32_t N1,
                                                uint32_t N2, uint32_t valid, bool cnn) {
    acc[3] += __popc(valid);
    acc[0] += __popc(up);
    if (HALF == 0) {
        if (cnn) acc[1] += __popc((S ^ N1) & valid) + __popc((S ^ N2) & valid);
    } else {
        acc[1] += __popc((up ^ S) & valid);
        acc[2] += __popc((up ^ N1) & valid) + __popc((up ^ N2) & valid);
    }
}

// A: M_tau = 2 up - n, C_nn = 2 n - 2 disagreeing; B: M_sigma, S_q = n - 2
// disagreeing, S_J = 2 n - 2 disagreeing.  Each is added to the step's row.
template <int HALF>
__device__ __forceinline__ void finish_step(const int (&acc)[4], const SweepArgs& a) {
    const int n = acc[3];
    if (HALF == 0) {
        const int v[2] = {2 * acc[0] - n, 2 * n - 2 * acc[1]};
        long long* const d[2] = {a.obs_cur ? a.obs_cur + 1 : nullptr,
                                 a.obs_prev ? a.obs_prev + 4 : nullptr};
        block_accumulate<2>(v, d);
    } else {
        const int v[3] = {2 * acc[0] - n, n - 2 * acc[1], 2 * n - 2 * acc[2]};
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
    pdl_begin();
    const uint32_t* __restrict__ src = static_cast<const uint32_t*>(a.src);
    uint32_t* __restrict__ dst = static_cast<uint32_t*>(a.dst);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t stride = ((gridDim.x * blockDim.x) >> 5) * 32 * ILP;
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[4] = {0, 0, 0, 0};
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
    pdl_begin();
    const int8_t* __restrict__ src = static_cast<const int8_t*>(a.src);
    int8_t* __restrict__ dst = static_cast<int8_t*>(a.dst);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t stride = ((gridDim.x * blockDim.x) >> 5) * 32;
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[4] = {0, 0, 0, 0};
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
// Each warp owns a ring of kQueueCap parked blocks in shared memory.  Blocks
// still undecided after Philox calls 0 and 1 wait there; once 32 are waiting
// the warp continues them together from call 2 (draw_rest).

// One parked block, 32 bytes: block index, undecided mask, decided-up mask and
// source word in one 16-byte store, the two field-neighbour words in an 8-byte
// one (two shared-memory instructions per parking warp instead of six).
struct QueueEntry {
    uint4 a;   // w, und, up, S
    uint2 b;   // N1, N2
    uint2 pad;
};

__device__ __forceinline__ void queue_put(QueueEntry& e, uint32_t w, uint32_t und, uint32_t up, uint32_t S,
                                          uint32_t N1, uint32_t N2) {
    e.a = make_uint4(w, und, up, S);
    e.b = make_uint2(N1, N2);
}

// The four int8 spins of every 4-bit group of a result word (unpack4 of
// 0..15), one table per CTA: the int8 sweeps that store through finish_block
// fill it at entry (unpack_table_init) and expand a word with 8 lookups.
__shared__ uint32_t g_unpack_table[16];

template <int LAYOUT>
__device__ __forceinline__ void unpack_table_init() {
    if constexpr (LAYOUT == kInt8) {
        if (threadIdx.x < 16) g_unpack_table[threadIdx.x] = unpack4(threadIdx.x);
        __syncthreads();
    }
}

__device__ __forceinline__ void unpack32_table(uint32_t bits, uint4& lo, uint4& hi) {
    lo.x = g_unpack_table[bits & 0xFu];
    lo.y = g_unpack_table[(bits >> 4) & 0xFu];
    lo.z = g_unpack_table[(bits >> 8) & 0xFu];
    lo.w = g_unpack_table[(bits >> 12) & 0xFu];
    hi.x = g_unpack_table[(bits >> 16) & 0xFu];
    hi.y = g_unpack_table[(bits >> 20) & 0xFu];
    hi.z = g_unpack_table[(bits >> 24) & 0xFu];
    hi.w = g_unpack_table[bits >> 28];
}

template <int HALF, int LAYOUT>
__device__ __forceinline__ void finish_block(const SweepArgs& a, uint32_t w, uint32_t up, uint32_t S,
                                             uint32_t N1, uint32_t N2, bool cnn, int (&acc)[4]) {
    if (LAYOUT == kBitpack) {
        *checked(static_cast<uint32_t*>(a.dst), w, a.nblocks, SHK_SITE) = up;
    } else {
        uint4 lo, hi;
        unpack32_table(up, lo, hi);
        uint4* q4 = reinterpret_cast<uint4*>(a.dst);
        *checked(q4, 2 * (uint64_t)w, 2 * (uint64_t)a.nblocks, SHK_SITE) = lo;
        *checked(q4, 2 * (uint64_t)w + 1, 2 * (uint64_t)a.nblocks, SHK_SITE) = hi;
    }
    accumulate_step<HALF>(acc, up, S, N1, N2, 0xffffffffu, cnn);
}

// Continues the `count` (<= 32) oldest parked blocks; all lanes call it.
template <int HALF, int LAYOUT, class PP>
__device__ __forceinline__ void drain_queue(const SweepArgs& a, const PP& P, QueueEntry* q,
                                            uint32_t head, int count, bool cnn, int (&acc)[4]) {
    const uint32_t lane = threadIdx.x & 31;
    const bool has = (int)lane < count;
    const uint32_t i = (head + lane) & (kQueueCap - 1);
    uint32_t w = 0, und = 0, up = 0, S = 0, N1 = 0, N2 = 0;
    if (has) {
        const uint4 x = q[i].a;
        const uint2 y = q[i].b;
        w = x.x;
        und = x.y;
        up = x.z;
        S = x.w;
        N1 = y.x;
        N2 = y.y;
    }
    const BlockClass k = block_class(S, N1, N2);
    const uint32_t res = draw_rest_pre(k, w, und, up, a.pre, P);
    if (has) finish_block<HALF, LAYOUT>(a, w, res, S, N1, N2, cnn, acc);
}

template <int HALF, int LAYOUT, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_sweep_q(const SweepArgs a) {
    pdl_begin();
    unpack_table_init<LAYOUT>();
    __shared__ QueueEntry qbuf[BLOCK / 32][kQueueCap];
    const DrawParams& P = a.P;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t stride = ((gridDim.x * blockDim.x) >> 5) * 32;
    QueueEntry* q = qbuf[threadIdx.x >> 5];
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[4] = {0, 0, 0, 0};
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
            queue_put(q[i], w, und, up, S, N1, N2);
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

// V consecutive words of a bit plane, vector index i of n (16- or 8-byte load).
template <int V>
__device__ __forceinline__ void load_words(const uint32_t* __restrict__ pl, uint32_t i, uint32_t n,
                                           uint32_t (&o)[V]) {
    static_assert(V == 2 || V == 4, "vector of 2 or 4 words");
    if constexpr (V == 4) {
        const uint4 t = __ldg(checked(reinterpret_cast<const uint4*>(pl), i, n, SHK_SITE));
        o[0] = t.x;
        o[1] = t.y;
        o[2] = t.z;
        o[3] = t.w;
    } else {
        const uint2 t = __ldg(checked(reinterpret_cast<const uint2*>(pl), i, n, SHK_SITE));
        o[0] = t.x;
        o[1] = t.y;
    }
}

// Bit-packed half-step with V consecutive blocks per thread: the blocks and
// their row neighbours come in one vector load each and the wrap-around bit
// in one scalar load, so the index arithmetic and the loads are shared by V
// blocks.  Each block then takes the two-phase draw with the warp queue
// exactly as in k_sweep_q (the blocks of a thread one after the other).
// Needs rows of a multiple of V blocks (L % (32 V) == 0), which also makes
// the number of vectors a multiple of 32: every lane is active.
template <int HALF, int V, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_sweep_qv(const SweepArgs a) {
    pdl_begin();
    __shared__ QueueEntry qbuf[BLOCK / 32][kQueueCap];
    const DrawParams& P = a.P;
    const uint32_t* __restrict__ src = static_cast<const uint32_t*>(a.src);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t stride = ((gridDim.x * blockDim.x) >> 5) * 32;
    QueueEntry* q = qbuf[threadIdx.x >> 5];
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[4] = {0, 0, 0, 0};
    uint32_t head = 0;
    int count = 0;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t nvec = a.nblocks / V, Wv = a.Wr / V;
    for (uint32_t base = gwarp * 32; base < nvec; base += stride) {
        const uint32_t v = base + lane;
        const uint32_t w0 = v * V;
        const uint32_t row = fdiv(w0, a.div_row);
        const uint32_t col = w0 - row * a.Wr;
        uint32_t S[V], N1[V];
        load_words<V>(src, v, nvec, S);
        if (HALF == 0) {
            load_words<V>(src, row > 0 ? v - Wv : v + nvec - Wv, nvec, N1);
        } else {
            load_words<V>(src, row + 1 < a.L ? v + Wv : v + Wv - nvec, nvec, N1);
        }
        // the word left of the first block (A) or right of the last one (B)
        const uint32_t x = HALF == 0 ? __ldg(checked(src, col > 0 ? w0 - 1 : w0 + a.Wr - 1, a.nblocks, SHK_SITE))
                                     : __ldg(checked(src, col + V < a.Wr ? w0 + V : w0 + V - a.Wr, a.nblocks,
                                                     SHK_SITE));
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const uint32_t w = w0 + k;
            const uint32_t N2 = HALF == 0 ? (S[k] << 1) | ((k == 0 ? x : S[k - 1]) >> 31)
                                          : (S[k] >> 1) | ((k == V - 1 ? x : S[k + 1]) << 31);
            const BlockClass c = block_class(S[k], N1[k], N2);
            uint32_t und, up;
            draw_first_two_pre(c, w, 0xffffffffu, a.pre, P, und, up);
            const bool parked = und != 0u;
            const uint32_t mask = __ballot_sync(0xffffffffu, parked);
            if (parked) {
                const uint32_t i = (head + count + __popc(mask & below)) & (kQueueCap - 1);
                queue_put(q[i], w, und, up, S[k], N1[k], N2);
            } else {
                finish_block<HALF, kBitpack>(a, w, up, S[k], N1[k], N2, cnn, acc);
            }
            count += __popc(mask);
            if (count >= 32) {
                __syncwarp();
                drain_queue<HALF, kBitpack>(a, P, q, head, 32, cnn, acc);
                __syncwarp();
                head = (head + 32) & (kQueueCap - 1);
                count -= 32;
            }
        }
    }
    if (count > 0) {
        __syncwarp();
        drain_queue<HALF, kBitpack>(a, P, q, head, count, cnn, acc);
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
    pdl_begin();
    unpack_table_init<LAYOUT>();
    __shared__ QueueEntry qbuf[BLOCK / 32][kQueueCap];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    QueueEntry* q = qbuf[threadIdx.x >> 5];
    const DrawParams& P = a.P;
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[4] = {0, 0, 0, 0};
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
                queue_put(q[qi], w, und, up, S, N1, N2);
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
    pdl_begin();
    unpack_table_init<LAYOUT>();
    constexpr int NW = RowWords<LAYOUT>::kWords;
    __shared__ QueueEntry qbuf[BLOCK / 32][kQueueCap];
    const DrawParams& P = a.P;
    __shared__ __align__(16) uint32_t ring[BLOCK / 32][DEPTH][32 * NW];
    __shared__ __align__(16) uint32_t ring_edge[BLOCK / 32][DEPTH][4];
    const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    QueueEntry* q = qbuf[wib];
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[4] = {0, 0, 0, 0};
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
                queue_put(q[qi], w, und, up, S, N1, N2);
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

// int8 strip walk with the rows moved by bulk asynchronous copies: a strip's
// row is 32 blocks of 32 bytes, 1024 contiguous bytes, so lane 0 stages the
// whole row with one cp.async.bulk (plus one 16-byte copy of the aligned
// chunk that holds the strip-edge byte), DEPTH rows ahead, into a per-warp
// ring whose slots complete on their own mbarrier.  The lanes wait for the
// slot's phase, unpack their 32 bytes and continue as k_sweep_strip_async.
// A wait that gives up (kCopyWaitCycles) sets *a.fault, waits (bounded) for
// the warp's copies still in flight and skips the rest of the warp's rows;
// the launch still completes, and the host reports the fault.
template <int HALF, int BLOCK, int MINB, int DEPTH>
__global__ void __launch_bounds__(BLOCK, MINB) k_sweep_strip_bulk(const SweepArgs a) {
    pdl_begin();
    unpack_table_init<kInt8>();
    __shared__ QueueEntry qbuf[BLOCK / 32][kQueueCap];
    __shared__ __align__(128) uint32_t ring[BLOCK / 32][DEPTH][256];       // 1024 bytes per row
    __shared__ uint32_t ring_edge[BLOCK / 32][DEPTH];                      // the word holding the edge byte
    __shared__ __align__(8) uint64_t bar[BLOCK / 32][DEPTH];
    const DrawParams& P = a.P;
    const uint32_t lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    QueueEntry* q = qbuf[wib];
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[4] = {0, 0, 0, 0};
    uint32_t head = 0;
    int count = 0;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t W = a.Wr, L = a.L;
    const uint32_t nstrips = W / 32;
    const bool edge_lane = HALF == 0 ? lane == 0 : lane == 31;
    const unsigned char* src8 = static_cast<const unsigned char*>(a.src);
    if (lane == 0) {
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) mbar_init(&bar[wib][d], 1);
        mbar_fence_init();
    }
    __syncwarp();
    uint32_t seq = 0;          // rows staged by this warp before the current task (slot = seq % DEPTH)
    bool failed = false;
    const uint64_t total = (uint64_t)nstrips * L;
    uint64_t pos = total * gwarp / nwarps;
    const uint64_t end = total * (gwarp + 1) / nwarps;
    while (pos < end && !failed) {
        const uint32_t strip = (uint32_t)(pos / L);
        const uint32_t r0 = (uint32_t)(pos - (uint64_t)strip * L);
        const uint64_t left_here = end - pos, left_in_strip = L - r0;
        const uint32_t nrows = (uint32_t)(left_here < left_in_strip ? left_here : left_in_strip);
        pos += nrows;
        const uint32_t col = strip * 32 + lane;
        const uint32_t edge_block = HALF == 0 ? (strip == 0 ? W - 1 : strip * 32 - 1)
                                              : (strip + 1 == nstrips ? 0 : strip * 32 + 32);
        auto row_at = [&](uint32_t i) -> uint32_t { return HALF == 0 ? r0 + i : r0 + nrows - 1 - i; };
        // row i of the walk goes to slot (seq + i) % DEPTH: lane 0 stages the
        // strip's 1024 bytes with one bulk copy, the edge lane the 4-byte word
        // holding the byte next to the strip with cp.async (one group per
        // lane and row, committed by every lane)
        auto stage = [&](uint32_t i) {
            if (i < nrows) {
                const uint32_t r = row_at(i), sl = (seq + i) % DEPTH;
                if (lane == 0) {
                    const size_t row_byte = (size_t)r * L;
                    // the lanes' reads of this slot (generic proxy) come
                    // before the copy engine's writes to it
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive_expect_tx(&bar[wib][sl], 1024u);
                    bulk_g2s(&ring[wib][sl][0],
                             checked_range(src8, row_byte + (size_t)strip * 1024, 1024, 32 * (uint64_t)a.nblocks,
                                           SHK_SITE),
                             1024u, &bar[wib][sl]);
                }
                if (edge_lane) {
                    const size_t eb = (size_t)r * W + edge_block;
                    const uint32_t* q1 = reinterpret_cast<const uint32_t*>(a.src);
                    cp_async4(&ring_edge[wib][sl],
                              checked(q1, 8 * eb + (HALF == 0 ? 7 : 0), 8 * (uint64_t)a.nblocks, SHK_SITE));
                }
            }
            cp_async_commit();
        };
        const uint32_t first = row_at(0);
        const uint32_t nb_row = HALF == 0 ? (first == 0 ? L - 1 : first - 1) : (first + 1 == L ? 0 : first + 1);
        uint32_t prev = row_bits<kInt8>(load_row<kInt8>(a.src, nb_row * W + col, a.nblocks));
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) stage(d);
        uint32_t i = 0;
        for (; i < nrows; ++i) {
            const uint32_t row = row_at(i), sl = (seq + i) % DEPTH, par = ((seq + i) / DEPTH) & 1u;
            const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[wib][sl], par, kCopyWaitCycles));
            if (!ok) {
                failed = true;
                break;
            }
            cp_async_wait<DEPTH - 1>();      // the edge lane's word of row i has landed
            const uint32_t* slot = &ring[wib][sl][lane * 8];
            const uint4 lo = *reinterpret_cast<const uint4*>(slot);
            const uint4 hi = *reinterpret_cast<const uint4*>(slot + 4);
            const uint32_t S = pack_up32(lo, hi);
            uint32_t edge = 0;
            if (edge_lane) {
                const uint32_t e = ring_edge[wib][sl];
                edge = HALF == 0 ? (uint32_t)((int8_t)(e >> 24) > 0) : (uint32_t)((int8_t)(e & 0xFFu) > 0);
            }
            __syncwarp();                    // every lane has read the slot before it is refilled
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
                queue_put(q[qi], w, und, up, S, N1, N2);
            } else {
                finish_block<HALF, kInt8>(a, w, up, S, N1, N2, cnn, acc);
            }
            count += __popc(mask);
            if (count >= 32) {
                __syncwarp();
                drain_queue<HALF, kInt8>(a, P, q, head, 32, cnn, acc);
                __syncwarp();
                head = (head + 32) & (kQueueCap - 1);
                count -= 32;
            }
            prev = S;
        }
        if (failed) {
            // the rows staged but not consumed: wait (bounded) for their copies,
            // so that none still writes to the ring when the block exits
            for (uint32_t j = i; j < nrows && j < i + DEPTH; ++j)
                (void)mbar_wait_bounded(&bar[wib][(seq + j) % DEPTH], ((seq + j) / DEPTH) & 1u, kCopyWaitCycles);
            if (lane == 0 && a.fault != nullptr) atomicOr(a.fault, 1u);
        }
        cp_async_wait<0>();                  // no edge copy may still target the ring
        __syncwarp();
        seq += nrows;
    }
    if (count > 0) {
        __syncwarp();
        drain_queue<HALF, kInt8>(a, P, q, head, count, cnn, acc);
    }
    finish_step<HALF>(acc, a);
}

// int8 half-step for any L (site-by-site neighbour gathers; partial last block).
template <int HALF>
__global__ void __launch_bounds__(256) k_sweep_i8g(const SweepArgs a) {
    pdl_begin();
    const int8_t* __restrict__ src = static_cast<const int8_t*>(a.src);
    int8_t* __restrict__ dst = static_cast<int8_t*>(a.dst);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    if (a.zero_slot != nullptr && blockIdx.x == 0 && threadIdx.x < kNumObs) a.zero_slot[threadIdx.x] = 0;
    const bool cnn = HALF == 0 && a.obs_prev != nullptr;
    int acc[4] = {0, 0, 0, 0};
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
    pdl_begin();
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

}  // namespace shk
