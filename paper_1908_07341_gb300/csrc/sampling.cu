// sampling.cu -- the Section 3 kernels on bit-packed planes and their
// launchers:
//   k_diag_corr          SW-NE / NW-SE spin-spin sums at up to eight lags
//                        (Section 3.3, Table 1)
//   k_checkerboard<P>    the square-lattice heat bath on the sites of one
//                        parity (the comparison dynamics of Section 3.2), with
//                        the magnetisation and C_nn fused into the odd half
//                        (device code in checkerboard.cuh)
//   k_coalesce<DYN>      coalescence times of the all + / all - coupling
//   k_cftp<DYN>          Propp-Wilson coupling from the past
// The draw machinery (Philox, lazy bit-serial comparison) is the half-steps'
// own (device.cuh).
#include <algorithm>

#define SHK_TU_ID 3
#include "internal.h"
#include "sweep.cuh"
#include "checkerboard.cuh"

namespace shk {

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
    uint32_t cw = c + (l >> 5);     // c < Wr and l < L, so below 2 Wr
    if (cw >= Wr) cw -= Wr;
    const uint32_t sh = l & 31u;
    const uint32_t lo = *checked(row, cw, Wr, SHK_SITE);
    if (sh == 0) return lo;
    const uint32_t hi = *checked(row, cw + 1 == Wr ? 0 : cw + 1, Wr, SHK_SITE);
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
        const uint32_t s = *checked(a.plane, w, a.nblocks, SHK_SITE);
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

// ------------------------------------------------------------ coalescence and coupling from the past

struct CoalescePair {
    uint32_t L, Wr, nblocks;
    uint32_t pad;
    FastDiv div_wr;     // division by Wr
    uint32_t pad2;
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
__device__ __forceinline__ void smem_fields(const uint32_t* pl, uint32_t w, uint32_t Wr, const FastDiv& dw,
                                            uint32_t L, uint32_t nblocks, uint32_t& S, uint32_t& N1,
                                            uint32_t& N2) {
    const uint32_t row = fdiv(w, dw), col = w - row * Wr;
    words_aligned<HALF>(pl, w, row, col, L, Wr, nblocks, S, N1, N2);
}

// Four bit-packed planes of one CTA: sigma and tau of the chain started from
// all + (top) and of the one started from all - (bottom).
struct PairPlanes {
    uint32_t *st, *tt, *sb, *tb;
    uint32_t nb, nbp, Wr, L;
    FastDiv dw;
};

__device__ __forceinline__ PairPlanes pair_planes(uint32_t* smem, const CoalescePair& cp) {
    PairPlanes p;
    p.nb = cp.nblocks;
    p.nbp = (cp.nblocks + 31u) & ~31u;
    p.Wr = cp.Wr;
    p.L = cp.L;
    p.dw = cp.div_wr;
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

// The four planes of call c for one chain of a coupled pair, accumulating
// the decided-up sites directly (up |= und & ~x & g); the same comparison as
// apply_planes, in the form that measured faster for the two-chain draw.
__device__ __forceinline__ void apply_planes_up(const uint4& R, int c, const BlockClass& k, uint32_t& und,
                                                uint32_t& up, const DrawParams& P) {
    const uint32_t x[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int b = 4 * c + m;
        const uint32_t g = k.F ^ SHK_PLANE_M0(P, b) ^ (k.Cg & SHK_PLANE_D01(P, b)) ^ (k.C2 & SHK_PLANE_D12(P, b));
        up |= und & ~x[m] & g;
        und &= ~(x[m] ^ g);
    }
}

// Draws block w of both coupled chains from one set of uniforms: each Philox
// call (four planes) serves the two chains, and the lazy loop ends when
// neither has an undecided site in the warp.  All 32 lanes call it together.
__device__ __forceinline__ void draw_coupled(const BlockClass (&k)[2], uint32_t w, uint32_t valid, uint32_t hs,
                                             const DrawParams& P, uint32_t (&up)[2]) {
    uint32_t und[2] = {valid, valid};
    up[0] = up[1] = 0u;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint4 R = philox_call(w, hs, c, P);
        apply_planes_up(R, c, k[0], und[0], up[0], P);
        apply_planes_up(R, c, k[1], und[1], up[1], P);
        if (c < 7 && !__any_sync(0xffffffffu, (und[0] | und[1]) != 0u)) break;
    }
    // ties through all 32 planes: a + site stays -1, a - site comes out +1
    up[0] |= und[0] & k[0].F;
    up[1] |= und[1] & k[1].F;
}

// One full step with index t of both chains, driven by the same uniforms
// (shaken: half-steps A and B over the plane words; checkerboard: even then
// odd sites of sigma over the draw blocks of two words each).
template <int DYN>
__device__ __forceinline__ void pair_step(const PairPlanes& p, unsigned long long t, const DrawParams& P) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t hs = (uint32_t)(2 * t);
    for (int half = 0; half < 2; ++half) {
        if (DYN == kDynShaken) {
            for (uint32_t base = warp * 32; base < p.nbp; base += nwarps * 32) {
                const uint32_t w = base + lane;
                const bool in = w < p.nb;
                BlockClass k[2] = {{0u, 0u, 0u}, {0u, 0u, 0u}};
                if (in) {
                    uint32_t S0, A0, B0, S1, A1, B1;
                    if (half == 0) {
                        smem_fields<0>(p.st, w, p.Wr, p.dw, p.L, p.nb, S0, A0, B0);
                        smem_fields<0>(p.sb, w, p.Wr, p.dw, p.L, p.nb, S1, A1, B1);
                    } else {
                        smem_fields<1>(p.tt, w, p.Wr, p.dw, p.L, p.nb, S0, A0, B0);
                        smem_fields<1>(p.tb, w, p.Wr, p.dw, p.L, p.nb, S1, A1, B1);
                    }
                    k[0] = block_class(S0, A0, B0);
                    k[1] = block_class(S1, A1, B1);
                }
                uint32_t up[2];
                draw_coupled(k, w, in ? 0xffffffffu : 0u, hs + (uint32_t)half, P, up);
                if (in) {
                    uint32_t* d0 = half == 0 ? p.tt : p.st;
                    uint32_t* d1 = half == 0 ? p.tb : p.sb;
                    d0[w] = up[0];
                    d1[w] = up[1];
                }
            }
        } else {
            // in place: the words read for the neighbours keep the bits of the
            // other parity, which no lane changes now
            const uint32_t nd = p.nb / 2;
            for (uint32_t base = warp * 32; base < nd; base += nwarps * 32) {
                const uint32_t d = base + lane;
                const bool in = d < nd;
                CbBlock c0, c1;
                c0.k = c1.k = {0u, 0u, 0u};
                c0.o0 = c0.o1 = 0u;
                if (in) {
                    const uint32_t r0 = fdiv(2 * d, p.dw), r1 = fdiv(2 * d + 1, p.dw);
                    c0 = cb_block(p.st, d, r0, r1, p.L, p.Wr, p.nb, (uint32_t)half);
                    c1 = cb_block(p.sb, d, r0, r1, p.L, p.Wr, p.nb, (uint32_t)half);
                }
                const BlockClass k[2] = {c0.k, c1.k};
                uint32_t up[2];
                draw_coupled(k, d, in ? 0xffffffffu : 0u, hs + (uint32_t)half, P, up);
                if (in) {
                    cb_store(p.st, d, up[0], c0.o0, c0.o1, p.nb);
                    cb_store(p.sb, d, up[1], c0.o0, c0.o1, p.nb);
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

// ------------------------------------------------------------ host side

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

// One warp per 32 words of the largest plane, at most 256 threads: a 32 x 32
// pair runs as a single-warp CTA, so an SM holds many pairs at once.
static int pair_threads(int max_L) {
    const int words = (max_L * max_L / 32 + 31) & ~31;
    return std::min(256, std::max(32, words));
}

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
        if (e == cudaSuccess) k_coalesce<kDynShaken><<<n_pairs, pair_threads(max_L), smem, st>>>(a);
    } else {
        e = allow_smem(k_coalesce<kDynCheckerboard>, smem);
        if (e == cudaSuccess) k_coalesce<kDynCheckerboard><<<n_pairs, pair_threads(max_L), smem, st>>>(a);
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
        if (e == cudaSuccess) k_cftp<kDynShaken><<<n_pairs, pair_threads(max_L), smem, st>>>(a);
    } else {
        e = allow_smem(k_cftp<kDynCheckerboard>, smem);
        if (e == cudaSuccess) k_cftp<kDynCheckerboard><<<n_pairs, pair_threads(max_L), smem, st>>>(a);
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
    c->div_wr = make_fastdiv(c->Wr);
    c->pad2 = 0;
    c->P = P;
}

cudaError_t launch_checkerboard(const Geometry& g, void* plane, const DrawParams& P, uint32_t hs, int parity,
                                long long* obs, cudaStream_t st) {
    SweepArgs a = sweep_args(g, plane, plane, P, hs, obs, nullptr, nullptr);
    const int block = 256;
    const uint64_t draw_blocks = g.nblocks / 2;   // 32 redrawn sites each
    cudaError_t e = cudaSuccess;
    if (jit_launch("shk::k_checkerboard<0>", "shk::k_checkerboard<1>", block, parity, (uint32_t)draw_blocks, a, st, &e))
        return e;
    SweepKernel k = parity == 0 ? k_checkerboard<0> : k_checkerboard<1>;
    return launch_pdl(k, grid_for(k, block, draw_blocks), block, st, a);
}

unsigned bounds_site_sampling() { return take_bounds_site(); }

}  // namespace shk
