// device.cuh -- device building blocks of the shaken-dynamics half-step.
//
// A half-step (Eqs. leftTrans / rightTrans of arXiv:1908.07341) redraws every
// spin of one sublattice independently, +1 with probability
// e^h / (2 cosh h), h the left or right local field (Eq. urdl).  The library
// realises the draw as "r < T[k]" with a 32-bit site uniform r and the integer
// threshold T[k] of the site's field class k = 3*[s = +1] + n (s the site's
// own spin, n the number of +1 neighbours in the field).
//
// GB300 design: spins are processed 32 at a time as bit-sliced words.  The 32
// uniforms of a 32-site block are the columns of the 32 x 32 bit matrix whose
// rows are the block's 32 Philox4x32-10 output words, most significant bit
// first.  Comparing 32 uniforms with 32 thresholds is then a bit-serial
// comparison from the most significant bit down: plane b of the random matrix
// is one Philox word, and each plane settles every still-undecided site with
// probability 1/2.  Planes (and the Philox calls that produce them, four per
// call) are generated only while some site of the warp is still undecided:
// about 13 of the 32 planes on average, so 3.2 instead of 8 Philox calls per
// block, with results identical bit for bit to the full comparison.
#pragma once

#ifdef __CUDACC_RTC__
// runtime compilation (jit.cu): the integer types without the host headers
typedef unsigned char uint8_t;
typedef signed char int8_t;
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned long long uint64_t;
typedef long long int64_t;
#else
#include <cstdint>
#include <cuda_runtime.h>
#endif

namespace shk {

// Plane layouts.
constexpr int kBitpack = 1;
constexpr int kInt8 = 2;

// Philox4x32 round multipliers and Weyl key increments (Salmon et al., 2011).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;

constexpr int kNumObs = 5;

// Everything a half-step needs besides the spins: the ten Philox round keys of
// the seed and, per random plane b = 0..31 (bit 31-b of the thresholds), the
// bit masks that select the threshold bit of each field class.  With the
// complement rule T[k] + T[5-k] = 2^32 only the three thresholds of a + site,
// U[n'] = T[3 + n'], are needed: a - site with n up-neighbours compares the
// complemented uniform against U[2 - n] and takes the complemented result.
// n' counts the neighbours that agree with the site.
struct DrawParams {
    uint32_t rk0[10];     // seed_lo + r * W0
    uint32_t rk1[10];     // seed_hi + r * W1
    uint32_t m0[32];      // all ones iff bit (31-b) of U[0] is set
    uint32_t d01[32];     // m0 ^ m1
    uint32_t d12[32];     // m1 ^ m2
    uint32_t lattice_id;  // third counter word
    uint32_t c3_base;     // fourth counter word of call 0 (256 * domain)
};

// Philox4x32-10 on the counter (c0, c1, c2, c3) with precomputed round keys.
// The caller puts the per-thread block index in c1: the first round's two
// products then involve only block-uniform words.  (The compiler's own
// lowering of the low/high product pair measured faster than an explicit
// mul.wide.u32.)
template <class PP>
__device__ __forceinline__ void philox10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                         const PP& P) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = kPhiloxM0 * c0;
        const uint32_t hi0 = __umulhi(kPhiloxM0, c0);
        const uint32_t lo1 = kPhiloxM1 * c2;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c2);
        const uint32_t n0 = hi1 ^ c1 ^ P.rk0[r];
        const uint32_t n2 = hi0 ^ c3 ^ P.rk1[r];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
}

// Draws the 32 spins of each of K blocks w[k] (sites 32w .. 32w+31), with the
// K Philox chains interleaved for instruction-level parallelism.
//   S      bits of the sites themselves in the source plane (1 = +1)
//   A, B   bits of the two field neighbours of each site
//   valid  sites that exist (bits beyond the plane are 0 and never delay exit)
//   hs     half-step index (first counter word)
// All 32 lanes of the warp must call this together: the loop over random
// planes stops when no lane has an undecided valid site in any of its blocks.
template <int K, class PP>
__device__ __forceinline__ void draw_blocks(const uint32_t (&S)[K], const uint32_t (&A)[K],
                                            const uint32_t (&B)[K], const uint32_t (&w)[K],
                                            const uint32_t (&valid)[K], uint32_t hs, const PP& P,
                                            uint32_t (&up)[K]) {
    uint32_t F[K], C2[K], Cg[K], und[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        F[k] = ~S[k];                       // sites that are -1
        const uint32_t a1 = ~(A[k] ^ S[k]); // neighbour A agrees with the site
        const uint32_t a2 = ~(B[k] ^ S[k]);
        C2[k] = a1 & a2;                    // both neighbours agree
        Cg[k] = a1 | a2;                    // at least one agrees
        und[k] = valid[k];                  // not yet decided
        up[k] = 0;                          // decided +1
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint32_t R[K][4];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            uint32_t x0 = hs, x1 = w[k], x2 = P.lattice_id, x3 = P.c3_base + (uint32_t)c;
            philox10(x0, x1, x2, x3, P);
            R[k][0] = x0;
            R[k][1] = x1;
            R[k][2] = x2;
            R[k][3] = x3;
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int b = 4 * c + m;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const uint32_t x = R[k][m];
                // g: the raw random bit value that would decide the site as +1,
                // i.e. the class threshold bit, complemented for - sites.
                const uint32_t g = F[k] ^ P.m0[b] ^ (Cg[k] & P.d01[b]) ^ (C2[k] & P.d12[b]);
                up[k] |= und[k] & ~x & g;
                und[k] &= ~(x ^ g);
            }
        }
        if (c < 7) {
            uint32_t any = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) any |= und[k];
            if (!__any_sync(0xffffffffu, any != 0u)) break;
        }
    }
    // A uniform equal to its threshold is not below it.  A + site therefore
    // stays -1; a - site compares its complemented uniform, so it comes out +1.
#pragma unroll
    for (int k = 0; k < K; ++k) up[k] |= und[k] & F[k];
}

// ---------------------------------------------------------------- two-phase draw
//
// Two Philox calls (8 planes) settle a 32-site block with probability
// (1 - 2^-8)^32 = 0.88, but a warp that runs the lazy loop to the end waits
// for the slowest of its 32 blocks and so needs 3.2 calls per block on
// average.  The two-phase form runs calls 0 and 1 unconditionally (two
// independent Philox chains), parks the blocks that still have undecided
// sites in a warp-private queue, and continues 32 parked blocks at a time
// from call 2 with the lazy early exit.  The result is the same comparison,
// bit for bit.

// Capacity of a warp's ring of parked blocks: a power of two; at most 31 + 32
// entries are held (a drain starts as soon as 32 are waiting).
constexpr int kQueueCap = 64;

// Class masks of a block (see draw_blocks).
struct BlockClass {
    uint32_t F, Cg, C2;
};

__device__ __forceinline__ BlockClass block_class(uint32_t S, uint32_t A, uint32_t B) {
    const uint32_t a1 = ~(A ^ S), a2 = ~(B ^ S);
    return {~S, a1 | a2, a1 & a2};
}

// Philox call c of block w in half-step hs: random planes 4c .. 4c+3.
template <class PP>
__device__ __forceinline__ uint4 philox_call(uint32_t w, uint32_t hs, int c, const PP& P) {
    uint32_t x0 = hs, x1 = w, x2 = P.lattice_id, x3 = P.c3_base + (uint32_t)c;
    philox10(x0, x1, x2, x3, P);
    return make_uint4(x0, x1, x2, x3);
}

// The warp-uniform part of the first three Philox rounds of one call.  In a
// half-step the counter (hs, w, lattice_id, c3) varies across threads only in
// the block index w, and w enters round 1 only through an XOR.  Folding the
// uniform words into constants leaves one varying product in round 2, one in
// round 3 and two in each of rounds 4 to 10 (round function as in philox10):
//   after round 1: c = (A ^ w, u1, u2, u3)            (u1..u3 uniform)
//   after round 2: c = (u4, u5, hi(M0 x1) ^ K2, lo(M0 x1)),  x1 = A ^ w
//   after round 3: c = (hi(M1 x2) ^ K3, lo(M1 x2), H3 ^ lo(M0 x1), D),
//                  x2 = hi(M0 x1) ^ K2
// The host computes (A, K2, K3, H3, D) per call and half-step.
struct PhiloxPrefix {
    uint32_t A, K2, K3, H3, D;
};

//
// The call index c enters round 1 only through an XOR into the third word,
// which round 2 multiplies by a constant; so A and K2 are the same for all
// calls of a half-step, and the two varying products of rounds 2 and 3
// (M0 x1 and M1 x2) depend on the block only.  A block computes them once
// (PhiloxBlock) and shares them among its calls.
struct PhiloxBlock {
    uint32_t h1, l1, l0;   // hi(M1 x2), lo(M1 x2), lo(M0 x1)
};

__device__ __forceinline__ PhiloxBlock philox_block(uint32_t w, const PhiloxPrefix& u) {
    const uint32_t x1 = u.A ^ w;
    const uint32_t x2 = __umulhi(kPhiloxM0, x1) ^ u.K2;
    return {__umulhi(kPhiloxM1, x2), kPhiloxM1 * x2, kPhiloxM0 * x1};
}

// Rounds 4 to 10 of one call from the block's shared products and the call's
// own uniform words (K3, H3, D).
template <class PP>
__device__ __forceinline__ uint4 philox_call_blk(const PhiloxBlock& b, const PhiloxPrefix& u, const PP& P) {
    uint32_t c0 = b.h1 ^ u.K3;
    uint32_t c1 = b.l1;
    uint32_t c2 = u.H3 ^ b.l0;
    uint32_t c3 = u.D;
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        const uint32_t lo0 = kPhiloxM0 * c0;
        const uint32_t hi0 = __umulhi(kPhiloxM0, c0);
        const uint32_t lo1 = kPhiloxM1 * c2;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c2);
        const uint32_t n0 = hi1 ^ c1 ^ P.rk0[r];
        const uint32_t n2 = hi0 ^ c3 ^ P.rk1[r];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

template <class PP>
__device__ __forceinline__ uint4 philox_call_pre(uint32_t w, const PhiloxPrefix& u, const PP& P) {
    return philox_call_blk(philox_block(w, u), u, P);
}

// Threshold bit masks of random plane b: all ones where bit 31-b of the
// class-0 threshold is set (m0), and the changes from class 0 to 1 (d01) and
// 1 to 2 (d12).  Read from the draw parameters; a kernel compiled at run time
// for one threshold table (jit.cu) gets the three thresholds as constants
// instead, so that each plane's mask folds into the logic.
#ifdef SHK_JIT_U0
__device__ __forceinline__ uint32_t jit_plane_bit(uint32_t u, int b) {
    return ((u >> (31 - b)) & 1u) ? 0xffffffffu : 0u;
}
#define SHK_PLANE_M0(P, b) jit_plane_bit(SHK_JIT_U0, (b))
#define SHK_PLANE_D01(P, b) (jit_plane_bit(SHK_JIT_U0, (b)) ^ jit_plane_bit(SHK_JIT_U1, (b)))
#define SHK_PLANE_D12(P, b) (jit_plane_bit(SHK_JIT_U1, (b)) ^ jit_plane_bit(SHK_JIT_U2, (b)))
#else
#define SHK_PLANE_M0(P, b) ((P).m0[b])
#define SHK_PLANE_D01(P, b) ((P).d01[b])
#define SHK_PLANE_D12(P, b) ((P).d12[b])
#endif

// Applies the four planes of call c to the state (und, v) of one block.
// g is the raw random bit that would decide a site as +1.  A site is decided
// at the first plane whose random bit differs from g, and its result is then
// that plane's g.  v takes g at every plane while the site is undecided and
// keeps it from then on (a bitwise select); und clears at the deciding
// plane.  Two three-input logic operations per plane.  The result of the
// block is draw_result(und, v, F) after the last plane (v alone once und is
// 0).
template <class PP>
__device__ __forceinline__ void apply_planes(const uint4& R, int c, const BlockClass& k, uint32_t& und,
                                             uint32_t& v, const PP& P) {
    const uint32_t x[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int b = 4 * c + m;
        const uint32_t g = k.F ^ SHK_PLANE_M0(P, b) ^ (k.Cg & SHK_PLANE_D01(P, b)) ^ (k.C2 & SHK_PLANE_D12(P, b));
        v = (und & g) | (~und & v);
        und &= ~(x[m] ^ g);
    }
}

// Result of a block whose undecided sites (und) tied their thresholds in all
// 32 planes: a uniform equal to its threshold is not below it, so a + site
// stays -1, and a - site (which compares its complemented uniform) comes out
// +1, i.e. the tie result is F.  Decided sites take v.
__device__ __forceinline__ uint32_t draw_result(uint32_t und, uint32_t v, uint32_t F) {
    return (und & F) | (~und & v);
}

// Phase 1: calls 0 and 1 for one block.
template <class PP>
__device__ __forceinline__ void draw_first_two(const BlockClass& k, uint32_t w, uint32_t valid,
                                               uint32_t hs, const PP& P, uint32_t& und,
                                               uint32_t& up) {
    const uint4 R0 = philox_call(w, hs, 0, P);
    const uint4 R1 = philox_call(w, hs, 1, P);
    und = valid;
    up = 0;
    apply_planes(R0, 0, k, und, up, P);
    apply_planes(R1, 1, k, und, up, P);
}

// Phase 1 with the host-computed round prefixes of the half-step (pre[c] for
// call c); the same draw as draw_first_two.  The two calls share the block's
// products of rounds 2 and 3.
template <class PP>
__device__ __forceinline__ void draw_first_two_pre(const BlockClass& k, uint32_t w, uint32_t valid,
                                                   const PhiloxPrefix (&pre)[8], const PP& P, uint32_t& und,
                                                   uint32_t& up) {
    const PhiloxBlock pb = philox_block(w, pre[0]);
    const uint4 R0 = philox_call_blk(pb, pre[0], P);
    const uint4 R1 = philox_call_blk(pb, pre[1], P);
    und = valid;
    up = 0;
    apply_planes(R0, 0, k, und, up, P);
    apply_planes(R1, 1, k, und, up, P);
}

// Phase 2 with the round prefixes; the same draw as draw_rest.
template <class PP>
__device__ __forceinline__ uint32_t draw_rest_pre(const BlockClass& k, uint32_t w, uint32_t und, uint32_t up,
                                                  const PhiloxPrefix (&pre)[8], const PP& P) {
    const PhiloxBlock pb = philox_block(w, pre[0]);
#pragma unroll
    for (int c = 2; c < 8; ++c) {
        if (!__any_sync(0xffffffffu, und != 0u)) break;
        const uint4 R = philox_call_blk(pb, pre[c], P);
        apply_planes(R, c, k, und, up, P);
    }
    return draw_result(und, up, k.F);
}

// Phase 2: calls 2..7 with the lazy exit; all 32 lanes call it together.
template <class PP>
__device__ __forceinline__ uint32_t draw_rest(const BlockClass& k, uint32_t w, uint32_t und,
                                              uint32_t up, uint32_t hs, const PP& P) {
#pragma unroll
    for (int c = 2; c < 8; ++c) {
        if (!__any_sync(0xffffffffu, und != 0u)) break;
        const uint4 R = philox_call(w, hs, c, P);
        apply_planes(R, c, k, und, up, P);
    }
    return draw_result(und, up, k.F);
}

// One block with precomputed class masks (lazy loop to the end; all lanes of
// the warp call it together).
template <class PP>
__device__ __forceinline__ uint32_t draw_block_class(const BlockClass& k, uint32_t w, uint32_t valid,
                                                     uint32_t hs, const PP& P) {
    uint32_t und = valid, up = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint4 R = philox_call(w, hs, c, P);
        apply_planes(R, c, k, und, up, P);
        if (c < 7 && !__any_sync(0xffffffffu, und != 0u)) break;
    }
    return draw_result(und, up, k.F);
}

// One block (the common case).
template <class PP>
__device__ __forceinline__ uint32_t draw_block(uint32_t S, uint32_t A, uint32_t B, uint32_t w,
                                               uint32_t valid, uint32_t hs, const PP& P) {
    const uint32_t s1[1] = {S}, a1[1] = {A}, b1[1] = {B}, w1[1] = {w}, v1[1] = {valid};
    uint32_t up[1];
    draw_blocks<1>(s1, a1, b1, w1, v1, hs, P, up);
    return up[0];
}

// ---------------------------------------------------------------- int8 <-> bits

// Up-bits of the four int8 spins (+1 = 0x01, -1 = 0xFF) of one 32-bit word:
// bit k of the result is 1 iff byte k is +1 (its sign bit is clear).
__device__ __forceinline__ uint32_t pack_up4(uint32_t x) {
    return (((~x) & 0x80808080u) * 0x00204081u) >> 28;
}

// Up-bits of 32 int8 spins (bytes of lo, then hi): the four flags of each
// word land in bits 28..31 of its product, and a funnel shift appends them to
// the result, last word first, so that word m ends in bits 4m..4m+3.
__device__ __forceinline__ uint32_t pack_up32(const uint4& lo, const uint4& hi) {
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
    uint32_t acc = 0;
#pragma unroll
    for (int m = 7; m >= 0; --m) acc = __funnelshift_l(((~w[m]) & 0x80808080u) * 0x00204081u, acc, 4);
    return acc;
}

// Four int8 spins from the low four bits of nib (bit k -> byte k): the
// product puts bit k on the sign bit of byte k (nib < 16, so the partial
// products do not overlap there), prmt replicates each byte's sign bit over
// the byte, and the complement with bit 0 set gives +1 = 0x01, -1 = 0xFF.
__device__ __forceinline__ uint32_t unpack4(uint32_t nib) {
    const uint32_t s = nib * 0x10204080u;
    uint32_t r;
    asm("prmt.b32 %0, %1, 0, 0xBA98;" : "=r"(r) : "r"(s));
    return ~r | 0x01010101u;
}

__device__ __forceinline__ void unpack32(uint32_t bits, uint4& lo, uint4& hi) {
    lo.x = unpack4(bits & 0xFu);
    lo.y = unpack4((bits >> 4) & 0xFu);
    lo.z = unpack4((bits >> 8) & 0xFu);
    lo.w = unpack4((bits >> 12) & 0xFu);
    hi.x = unpack4((bits >> 16) & 0xFu);
    hi.y = unpack4((bits >> 20) & 0xFu);
    hi.z = unpack4((bits >> 24) & 0xFu);
    hi.w = unpack4(bits >> 28);
}

// ---------------------------------------------------------------- async copies

// Asynchronous global -> shared copies (cp.async, sm_80 and later): the copy
// holds no registers and completes in the background; cp.async.wait_group N
// returns once at most N committed groups of this thread are still pending.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------- bulk copies
//
// Blackwell bulk asynchronous copies (cp.async.bulk, the tensor memory
// accelerator's untiled form): one thread moves a contiguous range of global
// memory (16-byte aligned, a multiple of 16 bytes) into shared memory, and
// the transfer signals completion on an mbarrier in shared memory by its byte
// count.  Waiting threads poll the barrier's phase; every wait here is
// bounded.

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the asynchronous copy engine.
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The calling thread's arrival, announcing `bytes` more to be transferred in
// the barrier's current phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(smem_dst)), "l"(gsrc), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.b32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(smem_addr(bar)), "r"(parity), "r"(1000u) : "memory");
    return done != 0u;
}

// Non-blocking check of the same phase.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.b32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return done != 0u;
}

// Waits until the barrier's phase with the given parity has completed, for at
// most limit_cycles SM clock cycles (and 2^24 polls): false if it gave up.
// A phase that has already completed (the common case, copies being staged
// rows ahead) is seen by one non-blocking test.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit_cycles) {
    if (mbar_test_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t n = 0; n < (1u << 24); ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > limit_cycles) return false;
    }
    return false;
}

// Poll limit of the sweeps' waits on their own copies: about two seconds at
// the maximum SM clock, far beyond any transfer that is still making progress.
constexpr long long kCopyWaitCycles = 4000000000LL;

// ---------------------------------------------------------------- division

// Division by a fixed divisor d >= 1 for n < 2^31: q = (umulhi(n, m) + n) >> s
// with s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
    uint32_t d, m, s;
};

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
    return (__umulhi(n, f.m) + n) >> f.s;
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long warp_sum64(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Adds per-thread values v[0..NV) of the whole block into dst[idx[i]] with one
// 64-bit atomic per value per block.  All threads of the block must call it.
template <int NV>
__device__ __forceinline__ void block_accumulate(const int (&v)[NV], long long* const (&dst)[NV]) {
    __shared__ long long red[NV][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const int s = warp_sum(v[i]);
        if (lane == 0) red[i][warp] = s;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            long long s = lane < nwarps ? red[i][lane] : 0;
            s = warp_sum64(s);
            if (lane == 0 && dst[i] != nullptr)
                atomicAdd(reinterpret_cast<unsigned long long*>(dst[i]),
                          static_cast<unsigned long long>(s));
        }
    }
}

}  // namespace shk
