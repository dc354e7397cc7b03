// checkerboard.cuh -- the checkerboard heat bath of the square-lattice Ising
// model (the comparison dynamics of Section 3.2): the kernel that redraws the
// sites of one parity in place, with the magnetisation and C_nn fused into the
// odd half.  Device code only: sampling.cu launches it, and jit.cu compiles the
// same text at run time with the thresholds of one J as constants.
#pragma once

#include "sweep.cuh"

namespace shk {

// ------------------------------------------------------------ checkerboard heat bath
//
// The square-lattice comparison dynamics of Section 3.2: the sites with
// (i + j) % 2 == parity are redrawn in place, P(+1) = e^h / (2 cosh h) with
// h = J (2n - 4), n the number of + among the four neighbours (all of the
// other parity, so unchanged while the parity is redrawn).
//
// Only the redrawn sites consume uniforms: numbered row by row,
// a = j (L/2) + floor(i/2), they fill draw blocks of 32, and draw block d
// (uniforms of counter word d) covers exactly the active sites of plane words
// 2d and 2d + 1 (16 each, in order).  A thread gathers those 32 sites and
// their neighbours into 32-bit words by bit compaction, draws them with the
// half-steps' machinery, and spreads the result back.
//
// With the complement rule the five thresholds fold onto the three-class
// draw: sites with n < 2 compare their complemented uniform, and the class
// is max(n, 4 - n) - 2 with thresholds (T[2], T[3], T[4]).

// The 16 bits of x at even positions 0, 2, .., 30, compacted to bits 0..15.
__device__ __forceinline__ uint32_t even_bits(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
    return x;
}

// Inverse of even_bits: bits 0..15 of x to positions 0, 2, .., 30.
__device__ __forceinline__ uint32_t spread_even(uint32_t x) {
    x &= 0x0000FFFFu;
    x = (x | (x << 8)) & 0x00FF00FFu;
    x = (x | (x << 4)) & 0x0F0F0F0Fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}

// The four neighbour bits (up, down, left, right) of the 16 active sites of
// plane word w, compacted, and the word's active offset o (active sites at
// bit positions o, o + 2, ..).
struct CbWord {
    uint32_t U, D, Lf, Rt, o;
};

__device__ __forceinline__ CbWord cb_word(const uint32_t* pl, uint32_t w, uint32_t row, uint32_t col, uint32_t L,
                                          uint32_t Wr, uint32_t nblocks, uint32_t parity) {
    CbWord r;
    r.o = (row + parity) & 1u;
    const uint32_t S = *checked(pl, w, nblocks, SHK_SITE);
    const uint32_t U = *checked(pl, row + 1 < L ? w + Wr : w + Wr - nblocks, nblocks, SHK_SITE);
    const uint32_t D = *checked(pl, row > 0 ? w - Wr : w + nblocks - Wr, nblocks, SHK_SITE);
    r.U = even_bits(U >> r.o);
    r.D = even_bits(D >> r.o);
    if (r.o == 0) {   // active at even positions: left and right neighbours are the odd bits
        const uint32_t prev = *checked(pl, col > 0 ? w - 1 : w + Wr - 1, nblocks, SHK_SITE);
        const uint32_t odd = even_bits(S >> 1);
        r.Rt = odd;
        r.Lf = ((odd << 1) | (prev >> 31)) & 0xFFFFu;
    } else {          // active at odd positions: neighbours are the even bits
        const uint32_t next = *checked(pl, col + 1 < Wr ? w + 1 : w + 1 - Wr, nblocks, SHK_SITE);
        const uint32_t even = even_bits(S);
        r.Lf = even;
        r.Rt = (even >> 1) | ((next & 1u) << 15);
    }
    return r;
}

// Class masks of draw block d (plane words 2d and 2d + 1) and the compacted
// neighbour words (for the fused C_nn).
struct CbBlock {
    BlockClass k;
    uint32_t U, D, Lf, Rt;
    uint32_t o0, o1;
};

__device__ __forceinline__ CbBlock cb_block(const uint32_t* pl, uint32_t d, uint32_t r0, uint32_t r1, uint32_t L,
                                            uint32_t Wr, uint32_t nblocks, uint32_t parity) {
    const uint32_t w0 = 2 * d, w1 = w0 + 1;
    const CbWord a = cb_word(pl, w0, r0, w0 - r0 * Wr, L, Wr, nblocks, parity);
    const CbWord b = cb_word(pl, w1, r1, w1 - r1 * Wr, L, Wr, nblocks, parity);
    CbBlock c;
    c.U = a.U | (b.U << 16);
    c.D = a.D | (b.D << 16);
    c.Lf = a.Lf | (b.Lf << 16);
    c.Rt = a.Rt | (b.Rt << 16);
    c.o0 = a.o;
    c.o1 = b.o;
    // n = U + D + Lf + Rt per site, as bits b0 + 2 b1 + 4 b2
    const uint32_t ab_s = c.U ^ c.D, ab_c = c.U & c.D, cd_s = c.Lf ^ c.Rt, cd_c = c.Lf & c.Rt;
    const uint32_t b0 = ab_s ^ cd_s, c0 = ab_s & cd_s;
    const uint32_t b1 = ab_c ^ cd_c ^ c0;
    const uint32_t b2 = (ab_c & cd_c) | ((ab_c ^ cd_c) & c0);
    const uint32_t extreme = b2 | ~(b0 | b1 | b2);       // n == 4 or n == 0
    c.k.F = ~(b1 | b2);                                 // n < 2
    c.k.C2 = extreme;
    c.k.Cg = b0 | extreme;                              // n odd or extreme
    return c;
}

// Writes the 32 drawn spins of draw block d back into plane words 2d, 2d + 1
// (their other bits are unchanged); returns the new words.
__device__ __forceinline__ uint2 cb_store(uint32_t* pl, uint32_t d, uint32_t up, uint32_t o0, uint32_t o1,
                                          uint32_t nblocks) {
    uint32_t* p0 = checked(pl, 2 * (uint64_t)d, nblocks, SHK_SITE);
    uint32_t* p1 = checked(pl, 2 * (uint64_t)d + 1, nblocks, SHK_SITE);
    const uint32_t m0 = 0x55555555u << o0, m1 = 0x55555555u << o1;
    const uint32_t v0 = (*p0 & ~m0) | (spread_even(up) << o0);
    const uint32_t v1 = (*p1 & ~m1) | (spread_even(up >> 16) << o1);
    *p0 = v0;
    *p1 = v1;
    return make_uint2(v0, v1);
}

// Adds the fused sums of a finished draw block: the magnetisation of its two
// words and, for the odd half (every bond has exactly one odd end), the bonds
// of its 32 redrawn sites.
__device__ __forceinline__ void cb_accumulate(int (&acc)[2], uint2 v, uint32_t up, uint32_t U, uint32_t D,
                                              uint32_t Lf, uint32_t Rt) {
    acc[0] += 2 * (__popc(v.x) + __popc(v.y)) - 64;
    acc[1] += 128 - 2 * (__popc(up ^ U) + __popc(up ^ D) + __popc(up ^ Lf) + __popc(up ^ Rt));
}

// Queue fields of a parked draw block: d, und, up, F, Cg, C2 (the neighbour
// words for the sums are gathered again when it is finished).
template <int PARITY>
__device__ __forceinline__ void cb_finish(const SweepArgs& a, uint32_t* pl, uint32_t d, uint32_t up, uint32_t o0,
                                          uint32_t o1, int (&acc)[2], const CbBlock* known) {
    const uint2 v = cb_store(pl, d, up, o0, o1, a.nblocks);
    if (PARITY == 1 && a.obs_cur != nullptr) {
        if (known != nullptr) {
            cb_accumulate(acc, v, up, known->U, known->D, known->Lf, known->Rt);
        } else {
            const CbBlock c = cb_block(pl, d, fdiv(2 * d, a.div_row), fdiv(2 * d + 1, a.div_row), a.L, a.Wr,
                                       a.nblocks, PARITY);
            cb_accumulate(acc, v, up, c.U, c.D, c.Lf, c.Rt);
        }
    }
}

// Continues the `take` (<= 32) oldest parked draw blocks from Philox call 2;
// all lanes call it.
template <int PARITY>
__device__ __forceinline__ void cb_drain(const SweepArgs& a, uint32_t* pl, uint32_t (*q)[kQueueCap], uint32_t head,
                                         int take, int (&acc)[2]) {
    const uint32_t lane = threadIdx.x & 31;
    const bool has = (int)lane < take;
    const uint32_t i = (head + lane) & (kQueueCap - 1);
    BlockClass k = {0u, 0u, 0u};
    uint32_t d = 0, und = 0, up = 0;
    if (has) {
        d = q[0][i];
        und = q[1][i];
        up = q[2][i];
        k.F = q[3][i];
        k.Cg = q[4][i];
        k.C2 = q[5][i];
    }
    const uint32_t res = draw_rest_pre(k, d, und, up, a.pre, a.P);
    if (has) {
        const uint32_t r0 = fdiv(2 * d, a.div_row), r1 = fdiv(2 * d + 1, a.div_row);
        cb_finish<PARITY>(a, pl, d, res, (r0 + PARITY) & 1u, (r1 + PARITY) & 1u, acc, nullptr);
    }
}

template <int PARITY>
__global__ void __launch_bounds__(256, 3) k_checkerboard(const SweepArgs a) {
    pdl_begin();
    __shared__ uint32_t qbuf[8][6][kQueueCap];
    uint32_t* pl = static_cast<uint32_t*>(a.dst);
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t stride = ((gridDim.x * blockDim.x) >> 5) * 32;
    uint32_t (*q)[kQueueCap] = qbuf[threadIdx.x >> 5];
    const uint32_t nd = a.nblocks / 2;
    const uint32_t below = (1u << lane) - 1u;
    int acc[2] = {0, 0};
    uint32_t head = 0;
    int count = 0;
    for (uint32_t base = gwarp * 32; base < nd; base += stride) {
        const uint32_t d = base + lane;
        const bool in = d < nd;
        CbBlock c;
        c.k = {0u, 0u, 0u};
        c.o0 = c.o1 = 0u;
        if (in) c = cb_block(pl, d, fdiv(2 * d, a.div_row), fdiv(2 * d + 1, a.div_row), a.L, a.Wr, a.nblocks, PARITY);
        uint32_t und, up;
        draw_first_two_pre(c.k, d, in ? 0xffffffffu : 0u, a.pre, a.P, und, up);
        const bool parked = und != 0u;
        const uint32_t mask = __ballot_sync(0xffffffffu, parked);
        if (parked) {
            const uint32_t i = (head + count + __popc(mask & below)) & (kQueueCap - 1);
            q[0][i] = d;
            q[1][i] = und;
            q[2][i] = up;
            q[3][i] = c.k.F;
            q[4][i] = c.k.Cg;
            q[5][i] = c.k.C2;
        } else if (in) {
            cb_finish<PARITY>(a, pl, d, up, c.o0, c.o1, acc, &c);
        }
        count += __popc(mask);
        if (count >= 32) {
            __syncwarp();
            cb_drain<PARITY>(a, pl, q, head, 32, acc);
            __syncwarp();
            head = (head + 32) & (kQueueCap - 1);
            count -= 32;
        }
    }
    if (count > 0) {
        __syncwarp();
        cb_drain<PARITY>(a, pl, q, head, count, acc);
    }
    if (PARITY == 1) {
        const int v[2] = {acc[0], acc[1]};
        long long* const dst[2] = {a.obs_cur, a.obs_cur ? a.obs_cur + 1 : nullptr};
        block_accumulate<2>(v, dst);
    }
}

}  // namespace shk
