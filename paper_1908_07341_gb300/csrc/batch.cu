// batch.cu -- many independent lattices in one persistent launch.
//
// The paper's phase-diagram runs give every (q, J) point its own lattice and
// thread (Section 4, multicore implementation).  Here a batch of bit-packed
// lattices of uneven side L is advanced by one persistent kernel.  Every
// lattice is cut into tiles of whole rows; a work item is one tile.  A launch
// advances every tile by k full steps: the CTA loads the tile's sigma rows
// together with k rows below and k + 1 rows above (wrapping around the torus)
// into shared memory and runs k steps there.  Each full step narrows the
// valid rows by one at each end (half-step A reads x^down, B reads x^up), so
// after k steps sigma is exact on the tile plus one row above and tau on the
// tile plus two rows above: enough for the observables of every step.  The
// halo rows are recomputed rather than exchanged; the counter-based random
// numbers make the recomputation exact.
// A lattice small enough to be one tile keeps its whole torus in shared memory
// with the rows wrapping, and needs no halo.
//
// sigma is double-buffered across launches (a tile reads the halo rows that
// neighbouring tiles overwrite); tau is written but never read.  The five
// observable sums of every step are added per tile into per-lattice partials;
// the last tile of a lattice to finish (ticket counter) folds them into exact
// int64 statistics; the last CTA of the launch advances the device-side step
// counter and resets the work counter.  No CTA ever waits for another, so a
// whole run is one CUDA graph launch: a while node whose body is one launch of
// the kernel, the last CTA of each launch counting the run's launches down and
// ending the loop after the last.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "shaken.h"
#define SHK_TU_ID 2
#include "internal.h"
#include "bounds.cuh"
#include "prefix.cuh"

namespace shk {

constexpr int kMaxStepsPerLaunch = 32;
constexpr int kStatFields = SHK_NSTATS;
static_assert(SHK_NSTATS == 11, "statistics layout");
// A parked block: w, und, up, S | N1, N2, local index (two 16-byte stores)
struct BatchQueueEntry {
    uint4 a, b;
};

struct BatchLattice {
    uint32_t L, Wr;             // side, words per row
    unsigned long long sigma_off[2];   // byte offsets of the two sigma buffers
    unsigned long long tau_off;
    unsigned long long scratch_off;    // partials [kMaxStepsPerLaunch][5] int64, then the ticket
    unsigned long long t;              // next step of this lattice (advanced on the device)
    unsigned long long remaining;      // steps still to run (decreased on the device)
    unsigned long long burn_in;        // steps t < burn_in are not added to the statistics
    uint32_t parity;                   // sigma buffer holding the current state (flipped on the device)
    uint32_t pad;
    FastDiv div_wr;                    // division by Wr
    uint32_t pad2;
    DrawParams P;
};

// One tile: rows [r0, r0 + nrows) of a lattice cut into ntiles tiles in this
// launch (ntiles == 1: the whole torus, rows wrapping).
struct BatchItem {
    uint32_t lattice, r0, nrows, ntiles;
};

struct BatchState {
    unsigned long long launches;   // launches completed
    unsigned int next;             // work counter of the running launch
    unsigned int done;             // CTAs finished in the running launch
    unsigned int launches_left;    // launches still to run in a graph loop (see loop)
};

struct BatchArgs {
    unsigned char* arena;
    BatchLattice* lat;             // per-lattice t, parity and remaining advance on the device
    const BatchItem* items;
    uint32_t n_items;
    uint32_t k;                    // full steps per launch (a lattice runs min(k, remaining))
    BatchState* state;
    long long* stats;              // n_lattices x kStatFields
    long long* last_obs;           // n_lattices x 5
    // Inside the body of a graph's while node: the launch's last CTA counts
    // launches_left down (never below zero) and keeps the loop running while
    // it is positive.  Outside a graph loop, loop = 0 and cond is unused.
    cudaGraphConditionalHandle cond;
    int loop;
};

// Global row of local row rho of a tile whose first row is r_base: r_base is
// at least -32 (the halo below row 0) and r_base + rho stays below 2L, so one
// wrap each way is enough.
__device__ __forceinline__ uint32_t global_row(int32_t r_base, uint32_t rho, uint32_t L) {
    int32_t g = r_base + (int32_t)rho;
    if (g < 0) g += (int32_t)L;
    else if (g >= (int32_t)L) g -= (int32_t)L;
    return (uint32_t)g;
}

// Geometry of one tile in shared memory: R local rows of Wr words (rows
// wrapping when the tile is the whole torus), local row 0 at global row
// r_base, and the tile's own rows [own_lo, own_lo + Hloc).
struct TileGeom {
    uint32_t R;
    bool wrap;
    uint32_t Wr;
    FastDiv dw;
    uint32_t L;
    int32_t r_base;
    uint32_t own_lo, Hloc;
};

// Draws rows [rlo, rhi) of dst (local row index) from src in shared memory.
// HALF 0 reads the row below (rho - 1), HALF 1 the row above (rho + 1); the
// left/right neighbour wraps within the row.  Random numbers use the global
// block index (global row g = (r_base + rho) mod L).
// ROWS: the lattice's rows are whole multiples of 32 words (L a multiple of
// 1024), so the 32 lanes of a warp always cover 32 consecutive words of one
// row: the row, its neighbour row and its global row are the same for the
// whole warp and advance by a fixed stride, with no per-word division and
// every lane holding a valid block.  Otherwise a warp's 32 words may span
// rows and the tile's end.
template <int HALF, int BLOCK, bool ROWS>
__device__ __forceinline__ void tile_sweep(const uint32_t* src, uint32_t* dst, uint32_t rlo, uint32_t rhi,
                                           const TileGeom& g, const DrawParams& P, const PhiloxPrefix (&pre)[8],
                                           BatchQueueEntry* q) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t Wr = g.Wr, R = g.R;
    uint32_t head = 0;
    int count = 0;
    auto drain = [&](int n) {
        const bool has = (int)lane < n;
        const uint32_t e = (head + lane) & (kQueueCap - 1);
        uint32_t w = 0, und = 0, up = 0, S = 0, N1 = 0, N2 = 0, i = 0;
        if (has) {
            const uint4 x = q[e].a, y = q[e].b;
            w = x.x; und = x.y; up = x.z; S = x.w; N1 = y.x; N2 = y.y; i = y.z;
        }
        const uint32_t res = draw_rest_pre(block_class(S, N1, N2), w, und, up, pre, P);
        if (has) dst[i] = res;
    };
    // phase 1 of the warp's 32 blocks (block i of lane: local word i, Philox
    // block w); blocks with undecided sites wait in the queue
    auto visit = [&](uint32_t i, uint32_t S, uint32_t N1, uint32_t N2, uint32_t w, uint32_t valid) {
        const BlockClass k = block_class(S, N1, N2);
        uint32_t und, up;
        draw_first_two_pre(k, w, valid, pre, P, und, up);
        const bool parked = und != 0u;
        const uint32_t mask = __ballot_sync(0xffffffffu, parked);
        if (parked) {
            const uint32_t e = (head + count + __popc(mask & below)) & (kQueueCap - 1);
            q[e].a = make_uint4(w, und, up, S);
            q[e].b = make_uint4(N1, N2, i, 0u);
        } else if (valid != 0u) {
            dst[i] = up;
        }
        count += __popc(mask);
        if (count >= 32) {
            __syncwarp();
            drain(32);
            __syncwarp();
            head = (head + 32) & (kQueueCap - 1);
            count -= 32;
        }
    };
    if constexpr (ROWS) {
        // this warp's first word (rlo, 0) + 32 warp and the stride of BLOCK words
        const uint32_t f = warp * 32u, dr = fdiv((uint32_t)BLOCK, g.dw), dc = (uint32_t)BLOCK - dr * Wr;
        uint32_t rho = rlo + fdiv(f, g.dw);
        uint32_t c0 = f - (rho - rlo) * Wr;
        while (rho < rhi) {
            // The lattice's draw parameters stay in shared memory, read where
            // used: held in registers across iterations they would cost a
            // third of the CTAs an SM can hold.
            asm volatile("" ::: "memory");
            const uint32_t c = c0 + lane, row = rho * Wr, i = row + c;
            const uint32_t S = src[i];
            uint32_t N1, N2;
            if (HALF == 0) {
                N1 = src[(rho == 0 && g.wrap ? (R - 1) * Wr : row - Wr) + c];
                const uint32_t prev = src[row + (c == 0 ? Wr - 1 : c - 1)];
                N2 = (S << 1) | (prev >> 31);
            } else {
                N1 = src[(rho + 1 == R && g.wrap ? 0 : row + Wr) + c];
                const uint32_t next = src[row + (c + 1 == Wr ? 0 : c + 1)];
                N2 = (S >> 1) | (next << 31);
            }
            visit(i, S, N1, N2, global_row(g.r_base, rho, g.L) * Wr + c, 0xffffffffu);
            c0 += dc;
            rho += dr;
            if (c0 >= Wr) {
                c0 -= Wr;
                ++rho;
            }
        }
    } else {
        const uint32_t lo = rlo * Wr, hi = rhi * Wr;
        for (uint32_t base = lo + warp * 32; base < hi; base += BLOCK) {
            const uint32_t i = base + lane;
            const bool in = i < hi;
            uint32_t S = 0, N1 = 0, N2 = 0, w = 0;
            if (in) {
                const uint32_t rho = fdiv(i, g.dw);
                const uint32_t c = i - rho * Wr;
                S = src[i];
                if (HALF == 0) {
                    N1 = src[(rho == 0 && g.wrap ? R - 1 : rho - 1) * Wr + c];
                    const uint32_t prev = src[rho * Wr + (c == 0 ? Wr - 1 : c - 1)];
                    N2 = (S << 1) | (prev >> 31);
                } else {
                    N1 = src[(rho + 1 == R && g.wrap ? 0 : rho + 1) * Wr + c];
                    const uint32_t next = src[rho * Wr + (c + 1 == Wr ? 0 : c + 1)];
                    N2 = (S >> 1) | (next << 31);
                }
                w = global_row(g.r_base, rho, g.L) * Wr + c;
            }
            visit(i, S, N1, N2, w, in ? 0xffffffffu : 0u);
        }
    }
    if (count > 0) {
        __syncwarp();
        drain(count);
    }
}

// Raw counts of one step over the tile's own rows (sigma in sg, tau in tu,
// both after the step): v[0] = up sites of sigma, v[1] = up sites of tau,
// v[2] = sites where sigma and tau disagree, v[3] = sigma sites that
// disagree with tau's up and right neighbours, v[4] = sigma sites that
// disagree with sigma's up and right neighbours.  ROWS as in tile_sweep: a
// warp reads 32 words of one row at a time.
template <int BLOCK, bool ROWS>
__device__ __forceinline__ void tile_counts(const uint32_t* sg, const uint32_t* tu, const TileGeom& g,
                                            int (&v)[kNumObs]) {
    const uint32_t Wr = g.Wr;
    auto add = [&](uint32_t x, uint32_t xu, uint32_t xr) {
        const uint32_t s = sg[x], t = tu[x];
        const uint32_t sU = sg[xu], tU = tu[xu];
        const uint32_t sR = (s >> 1) | (sg[xr] << 31), tR = (t >> 1) | (tu[xr] << 31);
        v[0] += __popc(s);
        v[1] += __popc(t);
        v[2] += __popc(s ^ t);
        v[3] += __popc(s ^ tU) + __popc(s ^ tR);
        v[4] += __popc(s ^ sU) + __popc(s ^ sR);
    };
    const uint32_t rlo = g.own_lo, rhi = g.own_lo + g.Hloc;
    if constexpr (ROWS) {
        const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const uint32_t f = warp * 32u, dr = fdiv((uint32_t)BLOCK, g.dw), dc = (uint32_t)BLOCK - dr * Wr;
        uint32_t rho = rlo + fdiv(f, g.dw);
        uint32_t c0 = f - (rho - rlo) * Wr;
        while (rho < rhi) {
            const uint32_t c = c0 + lane, row = rho * Wr;
            add(row + c, (rho + 1 == g.R && g.wrap ? 0 : row + Wr) + c, row + (c + 1 == Wr ? 0 : c + 1));
            c0 += dc;
            rho += dr;
            if (c0 >= Wr) {
                c0 -= Wr;
                ++rho;
            }
        }
    } else {
        for (uint32_t x = rlo * Wr + threadIdx.x; x < rhi * Wr; x += BLOCK) {
            const uint32_t rho = fdiv(x, g.dw), c = x - rho * Wr;
            add(x, (rho + 1 == g.R && g.wrap ? 0 : rho + 1) * Wr + c, rho * Wr + (c + 1 == Wr ? 0 : c + 1));
        }
    }
}

// Adds the block's per-thread values v[f] into red and, from warp 0, the
// signed sums off[f] + mul[f] * (sum of v[f]) into dst[f] (nullptr: skipped).
template <int BLOCK, int NV>
__device__ __forceinline__ void tile_reduce(const int (&v)[NV], long long (*red)[BLOCK / 32],
                                            const long long (&off)[NV], const int (&mul)[NV],
                                            long long* const (&dst)[NV]) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int f = 0; f < NV; ++f) {
        const int r = warp_sum(v[f]);
        if (lane == 0) red[f][warp] = r;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int f = 0; f < NV; ++f) {
            long long r = lane < BLOCK / 32 ? red[f][lane] : 0;
            r = warp_sum64(r);
            if (lane == 0 && dst[f] != nullptr)
                atomicAdd(reinterpret_cast<unsigned long long*>(dst[f]), (unsigned long long)(off[f] + mul[f] * r));
        }
    }
    __syncthreads();
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_batch(const __grid_constant__ BatchArgs a) {
    extern __shared__ uint32_t tile_mem[];
    __shared__ DrawParams P;
    __shared__ PhiloxPrefix pre[2][8];     // half-steps A and B of the current step
    __shared__ BatchQueueEntry qbuf[BLOCK / 32][kQueueCap];
    __shared__ long long red[kNumObs][BLOCK / 32];
    __shared__ uint32_t item_sh;
    __shared__ unsigned long long t0_sh, burn_sh;
    __shared__ uint32_t par_sh, k_sh;
    const uint32_t tid = threadIdx.x, warp = tid >> 5;
    BatchQueueEntry* q = qbuf[warp];

    for (;;) {
        if (tid == 0) item_sh = atomicAdd(&a.state->next, 1u);
        __syncthreads();
        const uint32_t ii = item_sh;
        if (ii >= a.n_items) break;
        const BatchItem it = a.items[ii];
        BatchLattice* B = a.lat + it.lattice;
        // The lattice's counters change only when its last tile of this launch
        // folds, after every tile of it (this one included) has read them.
        if (tid == 0) {
            const volatile BatchLattice* vb = B;
            t0_sh = vb->t;
            burn_sh = vb->burn_in;
            par_sh = vb->parity;
            const unsigned long long rem = vb->remaining;
            k_sh = (uint32_t)(rem < a.k ? rem : a.k);
        }
        __syncthreads();
        const unsigned long long t0 = t0_sh;
        const uint32_t par = par_sh, k = k_sh;
        if (k == 0) {              // the lattice has finished: nothing to do
            __syncthreads();
            continue;
        }
        const uint32_t L = B->L, Wr = B->Wr;
        const uint32_t r0 = it.r0;
        const uint32_t Hloc = it.nrows;
        // A lattice that is a single tile keeps its whole torus, rows wrapping;
        // otherwise the tile carries rows r0-k .. r0+Hloc+k (k below, k+1 above).
        const bool wrap = it.ntiles == 1;
        const uint32_t R = wrap ? L : Hloc + 2 * k + 1;
        const int32_t r_base = wrap ? 0 : (int32_t)r0 - (int32_t)k;
        const FastDiv dw = B->div_wr;
        const uint32_t own_lo = wrap ? 0 : k;           // local rows of the tile itself
        {
            const uint32_t* src = reinterpret_cast<const uint32_t*>(&B->P);
            uint32_t* dstp = reinterpret_cast<uint32_t*>(&P);
            for (uint32_t x = tid; x < sizeof(DrawParams) / 4; x += BLOCK) dstp[x] = src[x];
        }
        uint32_t* sg = tile_mem;
        uint32_t* tu = tile_mem + R * Wr;
        const uint32_t* sig_in = reinterpret_cast<const uint32_t*>(a.arena + B->sigma_off[par]);
        for (uint32_t x = tid; x < R * Wr; x += BLOCK) {
            const uint32_t rho = fdiv(x, dw), c = x - rho * Wr;
            sg[x] = *checked(sig_in, (uint64_t)global_row(r_base, rho, L) * Wr + c, (uint64_t)L * Wr, SHK_SITE);
        }
        __syncthreads();
        long long* partial = reinterpret_cast<long long*>(a.arena + B->scratch_off);
        const TileGeom g{R, wrap, Wr, dw, L, r_base, own_lo, Hloc};
        const long long n_own = (long long)Hloc * Wr * 32;   // sites in the tile's own rows
        for (uint32_t j = 0; j < k; ++j) {
            const uint32_t hs = (uint32_t)(2 * (t0 + j));
            fill_prefixes(pre[0], P, hs);
            if (tid >= 8 && tid < 16) pre[1][tid - 8] = philox_prefix_dev(P, hs + 1, (int)(tid - 8));
            __syncthreads();
            // Rows that later steps and the outputs still need: tau of step j
            // on [j + 1, R - j), sigma on [j + 1, R - 1 - j) (all rows when
            // the tile is the whole torus).
            const uint32_t lo = wrap ? 0 : j + 1, hiA = wrap ? R : R - j, hiB = wrap ? R : R - 1 - j;
            if (Wr % 32u == 0u) {
                tile_sweep<0, BLOCK, true>(sg, tu, lo, hiA, g, P, pre[0], q);
                __syncthreads();
                tile_sweep<1, BLOCK, true>(tu, sg, lo, hiB, g, P, pre[1], q);
            } else {
                tile_sweep<0, BLOCK, false>(sg, tu, lo, hiA, g, P, pre[0], q);
                __syncthreads();
                tile_sweep<1, BLOCK, false>(tu, sg, lo, hiB, g, P, pre[1], q);
            }
            __syncthreads();
            // The step's sums enter the statistics from the burn-in on, and the
            // launch's last step gives the last observables; the sums of other
            // burn-in steps are never read, so they are not formed.
            if (t0 + j < burn_sh && j + 1 < k) continue;
            int v[kNumObs] = {0, 0, 0, 0, 0};
            if (Wr % 32u == 0u) tile_counts<BLOCK, true>(sg, tu, g, v);
            else tile_counts<BLOCK, false>(sg, tu, g, v);
            // M = 2 up - n, M_tau = 2 up - n, S_q = n - 2 disagreeing,
            // S_J = 2 n - 2 disagreeing, C_nn = 2 n - 2 disagreeing
            long long* const pj = partial + j * kNumObs;
            const long long off[kNumObs] = {-n_own, -n_own, n_own, 2 * n_own, 2 * n_own};
            const int mul[kNumObs] = {2, 2, -2, -2, -2};
            long long* const dst[kNumObs] = {pj, pj + 1, pj + 2, pj + 3, pj + 4};
            tile_reduce<BLOCK, kNumObs>(v, red, off, mul, dst);
        }
        // write the tile's rows of sigma (other buffer) and tau
        uint32_t* sig_out = reinterpret_cast<uint32_t*>(a.arena + B->sigma_off[par ^ 1u]);
        uint32_t* tau_out = reinterpret_cast<uint32_t*>(a.arena + B->tau_off);
        for (uint32_t x = tid; x < Hloc * Wr; x += BLOCK) {
            const uint32_t lx = x + own_lo * Wr;
            const size_t gx = (size_t)r0 * Wr + x;
            *checked(sig_out, gx, (uint64_t)L * Wr, SHK_SITE) = sg[lx];
            *checked(tau_out, gx, (uint64_t)L * Wr, SHK_SITE) = tu[lx];
        }
        // the last tile of this lattice folds the k steps into the statistics
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            unsigned int* ticket = reinterpret_cast<unsigned int*>(partial + kMaxStepsPerLaunch * kNumObs);
            const unsigned int tk = atomicAdd(ticket, 1u);
            if (tk + 1 == it.ntiles) {
                __threadfence();
                long long* st = a.stats + (size_t)it.lattice * kStatFields;
                for (uint32_t j = 0; j < k; ++j) {
                    volatile long long* pj = partial + j * kNumObs;
                    const long long M = pj[0], Mt = pj[1], Sq = pj[2], SJ = pj[3], C = pj[4];
                    if (t0 + j >= burn_sh) {
                        st[0] += M;
                        st[1] += M * M;
                        st[2] += M < 0 ? -M : M;
                        st[3] += SJ;
                        st[4] += Sq;
                        st[5] += SJ * SJ;
                        st[6] += Sq * Sq;
                        st[7] += SJ * Sq;
                        st[8] += C;
                        st[9] += C * C;
                        st[10] += 1;
                    }
                    if (j + 1 == k) {
                        long long* lo = a.last_obs + (size_t)it.lattice * kNumObs;
                        lo[0] = M; lo[1] = Mt; lo[2] = Sq; lo[3] = SJ; lo[4] = C;
                    }
                    for (int f = 0; f < kNumObs; ++f) pj[f] = 0;
                }
                *ticket = 0u;
                volatile BatchLattice* vb = B;
                vb->t = t0 + k;
                vb->parity = par ^ 1u;
                vb->remaining = vb->remaining - k;
                __threadfence();
            }
        }
        __syncthreads();
    }
    // the last CTA of the launch prepares the next one
    if (tid == 0) {
        __threadfence();
        const unsigned int d = atomicAdd(&a.state->done, 1u);
        if (d + 1 == gridDim.x) {
            a.state->next = 0u;
            a.state->done = 0u;
            a.state->launches += 1ull;
            if (a.loop) {
                const unsigned int left = a.state->launches_left;
                const unsigned int now = left > 0u ? left - 1u : 0u;
                a.state->launches_left = now;
                cudaGraphSetConditional(a.cond, now > 0u ? 1u : 0u);
            }
            __threadfence();
        }
    }
}

// Launch count of the next graph run (one thread).
__global__ void k_batch_set_launches(BatchState* state, unsigned int launches) { state->launches_left = launches; }

}  // namespace shk

namespace shk {
unsigned bounds_site_batch() { return take_bounds_site(); }
}  // namespace shk

using namespace shk;

struct shk_batch {
    int n = 0;
    unsigned char* dev = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    std::vector<int> L;
    std::vector<BatchLattice> lat;
    std::vector<double> q, J;
    std::vector<uint64_t> seed;
    std::vector<uint32_t> lattice_id;
    // device-side pieces (offsets into dev)
    size_t off_state = 0, off_lat = 0, off_items = 0, off_stats = 0, off_last = 0;
    size_t items_capacity = 0;
    uint32_t n_items = 0;
    // host mirror of the per-lattice counters (all lattices advance together)
    uint64_t step = 0;
    uint32_t parity = 0;
    uint64_t burn_in = 0;
    // configuration
    int k = 8;
    int block = 256;
    int tile_sites = 1 << 18;
    size_t smem_bytes = 0;
    // graph of a whole run: a while node whose body is one launch
    cudaGraphExec_t graph = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_batch_err;

int bfail(shk_batch* b, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_batch_err = buf;
    set_thread_error(buf);
    return code;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr size_t kScratchPerLattice = 256 * ((kMaxStepsPerLaunch * kNumObs * 8 + 8 + 255) / 256);

bool batch_layout(int n, const int* L, std::vector<size_t>* lat_offsets, size_t* total, size_t* off_state,
                  size_t* off_lat, size_t* off_items, size_t* off_stats, size_t* off_last,
                  size_t* items_capacity) {
    size_t off = 0;
    *off_state = off;
    off += 256;
    *off_lat = off;
    off = align256(off + (size_t)n * sizeof(BatchLattice));
    size_t cap = 0;
    for (int i = 0; i < n; ++i) cap += (size_t)L[i];   // at most one tile per row
    *items_capacity = cap;
    *off_items = off;
    off = align256(off + cap * sizeof(BatchItem));
    *off_stats = off;
    off = align256(off + (size_t)n * kStatFields * 8);
    *off_last = off;
    off = align256(off + (size_t)n * kNumObs * 8);
    lat_offsets->resize(n);
    for (int i = 0; i < n; ++i) {
        Geometry g;
        if (!make_geometry(L[i], kBitpack, &g)) return false;
        (*lat_offsets)[i] = off;
        off += 3 * g.plane_bytes + kScratchPerLattice;
    }
    *total = off;
    return true;
}

// Rows per tile of a lattice of side L for a target of tile_sites sites.
uint32_t tile_rows_for(uint32_t L, int64_t tile_sites) {
    return (uint32_t)std::max<int64_t>(1, std::min<int64_t>(L, tile_sites / (int64_t)L));
}

// Appends the tiles of lattice i (rows per tile H) and returns the shared
// memory words its largest tile needs for k steps per launch.
size_t add_tiles(std::vector<BatchItem>* items, uint32_t i, uint32_t L, uint32_t Wr, uint32_t H, uint32_t k) {
    const uint32_t nt = (L + H - 1) / H;
    for (uint32_t t = 0; t < nt; ++t) items->push_back({i, t * H, std::min(H, L - t * H), nt});
    const uint32_t rows = nt == 1 ? L : H + 2 * k + 1;
    return 2 * (size_t)rows * Wr;
}

void sort_items(std::vector<BatchItem>* items, const std::vector<BatchLattice>& lat) {
    std::stable_sort(items->begin(), items->end(), [&](const BatchItem& x, const BatchItem& y) {
        return (uint64_t)x.nrows * lat[x.lattice].L > (uint64_t)y.nrows * lat[y.lattice].L;
    });
}

// Builds the work items (largest tiles first) and the shared memory a tile needs.
void build_items(shk_batch* b, std::vector<BatchItem>* items) {
    items->clear();
    size_t smem_words = 0;
    for (int i = 0; i < b->n; ++i) {
        const BatchLattice& B = b->lat[i];
        smem_words = std::max(smem_words, add_tiles(items, (uint32_t)i, B.L, B.Wr,
                                                    tile_rows_for(B.L, b->tile_sites), (uint32_t)b->k));
    }
    sort_items(items, b->lat);
    b->smem_bytes = smem_words * 4;
}

// Shared-memory attribute and grid size (kept out of stream capture).
template <int BLOCK>
cudaError_t prepare_block(shk_batch* b, int* grid) {
    cudaError_t e = cudaFuncSetAttribute(k_batch<BLOCK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)b->smem_bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<BLOCK>, BLOCK, b->smem_bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid = (int)std::min<uint64_t>((uint64_t)per_sm * sm_count(), std::max<uint32_t>(1, b->n_items));
    return cudaSuccess;
}

cudaError_t prepare_batch(shk_batch* b, int* grid) {
    switch (b->block) {
        case 128: return prepare_block<128>(b, grid);
        case 512: return prepare_block<512>(b, grid);
        default: return prepare_block<256>(b, grid);
    }
}

cudaError_t launch_batch(shk_batch* b, int grid, cudaStream_t st, bool loop = false,
                         cudaGraphConditionalHandle cond = 0) {
    BatchArgs args;
    args.cond = cond;
    args.loop = loop ? 1 : 0;
    args.arena = b->dev;
    args.lat = reinterpret_cast<BatchLattice*>(b->dev + b->off_lat);
    args.items = reinterpret_cast<const BatchItem*>(b->dev + b->off_items);
    args.n_items = b->n_items;
    args.k = (uint32_t)b->k;
    args.state = reinterpret_cast<BatchState*>(b->dev + b->off_state);
    args.stats = reinterpret_cast<long long*>(b->dev + b->off_stats);
    args.last_obs = reinterpret_cast<long long*>(b->dev + b->off_last);
    switch (b->block) {
        case 128: k_batch<128><<<grid, 128, b->smem_bytes, st>>>(args); break;
        case 512: k_batch<512><<<grid, 512, b->smem_bytes, st>>>(args); break;
        default: k_batch<256><<<grid, 256, b->smem_bytes, st>>>(args); break;
    }
    return cudaGetLastError();
}

// Writes the descriptors (with the host mirror of t, parity, k and burn-in)
// and, with rebuild, the work items; a rebuild drops the captured graph.
int upload_descriptors(shk_batch* b, bool rebuild) {
    std::vector<BatchItem> items;
    if (rebuild) {
        build_items(b, &items);
        if (items.size() > b->items_capacity) return bfail(b, SHK_EINVAL, "shk_batch: too many tiles");
        b->n_items = (uint32_t)items.size();
    }
    for (BatchLattice& B : b->lat) {
        B.t = b->step;
        B.parity = b->parity;
        B.remaining = ~0ull;              // a batch lattice never runs out of steps
        B.burn_in = b->burn_in;
    }
    cudaError_t e = cudaMemcpyAsync(b->dev + b->off_lat, b->lat.data(), b->lat.size() * sizeof(BatchLattice),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && rebuild)
        e = cudaMemcpyAsync(b->dev + b->off_items, items.data(), items.size() * sizeof(BatchItem),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, SHK_ECUDA, "shk_batch upload: %s", cudaGetErrorString(e));
    if (rebuild && b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return SHK_OK;
}

}  // namespace

extern "C" {

size_t shk_batch_bytes(int n, const int* L) {
    if (n <= 0 || L == nullptr) return 0;
    std::vector<size_t> lo;
    size_t total, a, b2, c, d, e, cap;
    if (!batch_layout(n, L, &lo, &total, &a, &b2, &c, &d, &e, &cap)) return 0;
    return total;
}

int shk_batch_create(int n, const int* L, const double* q, const double* J, const uint64_t* seed,
                     const uint32_t* lattice_id, void* dev_mem, size_t bytes, void* stream,
                     shk_batch** out) {
    if (out == nullptr) return bfail(nullptr, SHK_EINVAL, "shk_batch_create: out is NULL");
    *out = nullptr;
    if (n <= 0 || !L || !q || !J || !seed || !lattice_id)
        return bfail(nullptr, SHK_EINVAL, "shk_batch_create: n must be positive and arrays non-NULL");
    for (int i = 0; i < n; ++i)
        if (L[i] < 32 || L[i] % 32 != 0 || L[i] > 65536)
            return bfail(nullptr, SHK_EINVAL, "shk_batch_create: lattice %d has L=%d (need 32 <= L <= 65536, L %% 32 == 0)",
                         i, L[i]);
    std::vector<size_t> lat_off;
    size_t total, off_state, off_lat, off_items, off_stats, off_last, cap;
    batch_layout(n, L, &lat_off, &total, &off_state, &off_lat, &off_items, &off_stats, &off_last, &cap);
    if (dev_mem == nullptr || (reinterpret_cast<uintptr_t>(dev_mem) & 255u) != 0)
        return bfail(nullptr, SHK_EINVAL, "shk_batch_create: dev_mem must be non-NULL and 256-byte aligned");
    if (bytes < total) return bfail(nullptr, SHK_ENOMEM, "shk_batch_create: %zu bytes given, %zu needed", bytes, total);
    shk_batch* b = new (std::nothrow) shk_batch();
    if (!b) return bfail(nullptr, SHK_ENOMEM, "shk_batch_create: host allocation failed");
    b->n = n;
    b->dev = static_cast<unsigned char*>(dev_mem);
    b->bytes = bytes;
    b->stream = static_cast<cudaStream_t>(stream);
    b->L.assign(L, L + n);
    b->q.assign(q, q + n);
    b->J.assign(J, J + n);
    b->seed.assign(seed, seed + n);
    b->lattice_id.assign(lattice_id, lattice_id + n);
    b->off_state = off_state;
    b->off_lat = off_lat;
    b->off_items = off_items;
    b->off_stats = off_stats;
    b->off_last = off_last;
    b->items_capacity = cap;
    b->lat.resize(n);
    for (int i = 0; i < n; ++i) {
        Geometry g;
        make_geometry(L[i], kBitpack, &g);
        BatchLattice& B = b->lat[i];
        std::memset(&B, 0, sizeof B);
        B.L = (uint32_t)L[i];
        B.Wr = g.Wr;
        B.div_wr = make_fastdiv(g.Wr);
        B.sigma_off[0] = lat_off[i];
        B.sigma_off[1] = lat_off[i] + g.plane_bytes;
        B.tau_off = lat_off[i] + 2 * g.plane_bytes;
        B.scratch_off = lat_off[i] + 3 * g.plane_bytes;
        uint32_t T[6];
        if (host_thresholds(q[i], J[i], T) != SHK_OK) {
            delete b;
            return bfail(nullptr, SHK_EINVAL, "shk_batch_create: lattice %d has non-finite q or J", i);
        }
        make_draw_params(seed[i], lattice_id[i], T, 0u, &B.P);
    }
    // zero the state, statistics, results and per-lattice scratch
    cudaError_t e = cudaMemsetAsync(b->dev, 0, total, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        delete b;
        return bfail(nullptr, SHK_ECUDA, "shk_batch_create: %s", cudaGetErrorString(e));
    }
    const int rc = upload_descriptors(b, true);
    if (rc != SHK_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return SHK_OK;
}

void shk_batch_destroy(shk_batch* b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    delete b;
}

const char* shk_batch_last_error(const shk_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

int shk_batch_configure(shk_batch* b, int steps_per_launch, int block_threads, int tile_sites) {
    if (!b) return bfail(nullptr, SHK_EINVAL, "shk_batch_configure: NULL handle");
    if (steps_per_launch < 1 || steps_per_launch > kMaxStepsPerLaunch)
        return bfail(b, SHK_EINVAL, "shk_batch_configure: steps_per_launch must be in 1..%d", kMaxStepsPerLaunch);
    if (block_threads != 128 && block_threads != 256 && block_threads != 512)
        return bfail(b, SHK_EINVAL, "shk_batch_configure: block_threads must be 128, 256 or 512");
    if (tile_sites < 1024) return bfail(b, SHK_EINVAL, "shk_batch_configure: tile_sites must be >= 1024");
    b->k = steps_per_launch;
    b->block = block_threads;
    b->tile_sites = tile_sites;
    const int rc = upload_descriptors(b, true);
    if (rc != SHK_OK) return rc;
    // refuse a tile that does not fit in shared memory
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa = {};
    const cudaError_t fe = cudaFuncGetAttributes(
        &fa, block_threads == 128 ? (const void*)k_batch<128> : block_threads == 512 ? (const void*)k_batch<512>
                                                                                    : (const void*)k_batch<256>);
    if (fe != cudaSuccess) return bfail(b, SHK_ECUDA, "shk_batch_configure: %s", cudaGetErrorString(fe));
    const size_t static_smem = fa.sharedSizeBytes;
    if (b->smem_bytes + static_smem > (size_t)optin)
        return bfail(b, SHK_EINVAL, "shk_batch_configure: a tile needs %zu bytes of shared memory (limit %d); lower tile_sites or steps_per_launch",
                     b->smem_bytes + static_smem, optin);
    return SHK_OK;
}

int shk_batch_init(shk_batch* b, int kind, uint64_t init_seed) {
    if (!b) return bfail(nullptr, SHK_EINVAL, "shk_batch_init: NULL handle");
    for (int i = 0; i < b->n; ++i) {
        const int rc = shk_init_plane(SHK_BITPACK, b->dev + b->lat[i].sigma_off[0], b->L[i], kind, init_seed,
                                      b->lattice_id[i], 0, b->stream);
        if (rc != SHK_OK) return bfail(b, rc, "shk_batch_init: %s", shk_last_error(nullptr));
        const int rc2 = shk_init_plane(SHK_BITPACK, b->dev + b->lat[i].tau_off, b->L[i], kind, init_seed,
                                       b->lattice_id[i], 1, b->stream);
        if (rc2 != SHK_OK) return bfail(b, rc2, "shk_batch_init: %s", shk_last_error(nullptr));
    }
    // state, statistics and last observables back to zero; sigma in buffer 0
    b->step = 0;
    b->parity = 0;
    const int rc = upload_descriptors(b, false);
    if (rc != SHK_OK) return rc;
    cudaError_t e = cudaMemsetAsync(b->dev + b->off_state, 0, 256, b->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->dev + b->off_stats, 0, (size_t)b->n * kStatFields * 8, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->dev + b->off_last, 0, (size_t)b->n * kNumObs * 8, b->stream);
    if (e != cudaSuccess) return bfail(b, SHK_ECUDA, "shk_batch_init: %s", cudaGetErrorString(e));
    return SHK_OK;
}

int shk_batch_run(shk_batch* b, uint64_t n_steps, uint64_t burn_in) {
    const TraceRange trace("shk_batch_run");
    if (!b) return bfail(nullptr, SHK_EINVAL, "shk_batch_run: NULL handle");
    if (n_steps == 0) return SHK_OK;
    if (b->step > SHK_MAX_STEP || n_steps > SHK_MAX_STEP - b->step)
        return bfail(b, SHK_EINVAL, "shk_batch_run: step counter would exceed 2^31");
    if (n_steps % (uint64_t)b->k != 0)
        return bfail(b, SHK_EINVAL, "shk_batch_run: n_steps=%llu is not a multiple of steps_per_launch=%d",
                     (unsigned long long)n_steps, b->k);
    if (burn_in != b->burn_in) {
        b->burn_in = burn_in;
        const int rc = upload_descriptors(b, false);
        if (rc != SHK_OK) return rc;
    }
    cudaError_t e;
    if (b->graph == nullptr) {
        // One graph for the whole run: a while node whose body is one launch
        // of the persistent kernel; the kernel ends the loop once the
        // device-side launch count is used up.
        int grid = 0;
        e = prepare_batch(b, &grid);
        if (e != cudaSuccess) return bfail(b, SHK_ECUDA, "shk_batch_run: %s", cudaGetErrorString(e));
        cudaGraph_t g = nullptr;
        cudaStream_t cap = nullptr;
        e = cudaGraphCreate(&g, 0);
        cudaGraphConditionalHandle cond = 0;
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(cap, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t le = launch_batch(b, grid, cap, true, cond);
            cudaGraph_t body = nullptr;
            e = cudaStreamEndCapture(cap, &body);
            if (le != cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (cap) cudaStreamDestroy(cap);
        if (e != cudaSuccess) return bfail(b, SHK_ECUDA, "shk_batch_run graph: %s", cudaGetErrorString(e));
    }
    // the run's launch count (stored on the device by a one-thread kernel, so
    // that the call stays asynchronous), then one graph launch for all of them
    const unsigned int launches = (unsigned int)(n_steps / (uint64_t)b->k);
    k_batch_set_launches<<<1, 1, 0, b->stream>>>(reinterpret_cast<BatchState*>(b->dev + b->off_state), launches);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaGraphLaunch(b->graph, b->stream);
    if (e != cudaSuccess) return bfail(b, SHK_ECUDA, "shk_batch_run launch: %s", cudaGetErrorString(e));
    b->step += n_steps;
    b->parity ^= launches & 1u;
    return SHK_OK;
}

int shk_batch_read_stats(shk_batch* b, int64_t* host_stats) {
    if (!b || !host_stats) return bfail(b, SHK_EINVAL, "shk_batch_read_stats: NULL argument");
    cudaError_t e = cudaMemcpyAsync(host_stats, b->dev + b->off_stats, (size_t)b->n * kStatFields * 8,
                                    cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, SHK_ECUDA, "shk_batch_read_stats: %s", cudaGetErrorString(e));
    return SHK_OK;
}

int shk_batch_read_observables(shk_batch* b, int64_t* host_obs) {
    if (!b || !host_obs) return bfail(b, SHK_EINVAL, "shk_batch_read_observables: NULL argument");
    cudaError_t e = cudaMemcpyAsync(host_obs, b->dev + b->off_last, (size_t)b->n * kNumObs * 8,
                                    cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, SHK_ECUDA, "shk_batch_read_observables: %s", cudaGetErrorString(e));
    return SHK_OK;
}

int shk_batch_get_step(shk_batch* b, uint64_t* step) {
    if (!b || !step) return bfail(b, SHK_EINVAL, "shk_batch_get_step: NULL argument");
    *step = b->step;
    return SHK_OK;
}

int shk_batch_read_spins(shk_batch* b, int idx, int plane, int8_t* host_out) {
    if (!b || !host_out || idx < 0 || idx >= b->n || (plane != 0 && plane != 1))
        return bfail(b, SHK_EINVAL, "shk_batch_read_spins: bad argument");
    const BatchLattice& B = b->lat[idx];
    const size_t off = plane == 0 ? B.sigma_off[b->parity] : B.tau_off;
    cudaError_t e;
    const int64_t N = (int64_t)B.L * B.L;
    std::vector<uint32_t> words((size_t)(N / 32));
    e = cudaMemcpyAsync(words.data(), b->dev + off, words.size() * 4, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, SHK_ECUDA, "shk_batch_read_spins: %s", cudaGetErrorString(e));
    for (int64_t u = 0; u < N; ++u) host_out[u] = ((words[u >> 5] >> (u & 31)) & 1u) ? 1 : -1;
    return SHK_OK;
}

}  // extern "C"

// ======================================================================
// Serving: continuous batching of simulation jobs over the batch kernel.
//
// Jobs wait in a FIFO queue.  At every tick the scheduler (1) admits queued
// jobs, oldest first, while a slot is free and the job's planes fit in the
// HBM budget (first-fit allocation in the caller's arena), initialising their
// lattices on the device; (2) advances every active job by min(slice,
// remaining) steps in one launch of the persistent kernel, each job's lattice,
// step counter and random-number key staying resident; (3) retires finished
// jobs, copying their exact statistics, last observables and a hash of the
// final sigma.  Jobs admitted at a tick share that tick's launch with jobs
// already running, so work of different jobs overlaps on the device, and a
// job's result does not depend on what else runs (its random numbers depend
// only on its own seed, lattice id and step).
// ======================================================================

#include <deque>
#include <map>

namespace {

constexpr uint32_t kMaxTilesPerJob = 512;
constexpr int kMaxServerL = 8192;

struct Slot {
    bool used = false;
    uint64_t job_id = 0;
    shk_job job{};
    uint64_t remaining = 0;
    size_t mem_off = 0, mem_bytes = 0;
    uint64_t submit_tick = 0, admit_tick = 0;
};

struct Pending {
    uint64_t job_id;
    shk_job job;
    uint64_t submit_tick;
};

// First-fit allocator over [0, capacity) with coalescing of freed ranges.
class Arena {
public:
    void reset(size_t capacity) {
        free_.clear();
        if (capacity) free_[0] = capacity;
    }
    bool alloc(size_t n, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n;
                const size_t start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n) {
        auto it = free_.emplace(off, n).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }

private:
    std::map<size_t, size_t> free_;
};

uint64_t fnv1a64(const unsigned char* p, size_t n) {
    uint64_t h = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

}  // namespace

struct shk_server {
    int max_slots = 0;
    size_t budget = 0, used = 0;
    unsigned char* dev = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    size_t off_state = 0, off_lat = 0, off_items = 0, off_stats = 0, off_last = 0, off_arena = 0;
    Arena arena;
    std::vector<Slot> slots;
    std::vector<BatchLattice> lat;
    std::deque<Pending> pending;
    std::vector<shk_result> done;
    size_t max_pending = 1u << 20;
    uint64_t next_id = 1;
    uint64_t tick = 0;
    int k = 2;                  // steps per launch
    int launches = 16;          // launches per tick
    int block = 256;
    int tile_sites = 1 << 18;   // largest tile; smaller while few jobs are active
    std::string err;
};

namespace {

thread_local std::string g_server_err;

int sfail(shk_server* s, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    else g_server_err = buf;
    set_thread_error(buf);
    return code;
}

size_t job_bytes(int L) {
    Geometry g;
    make_geometry(L, kBitpack, &g);
    return 3 * g.plane_bytes + kScratchPerLattice;
}

void server_layout(int max_slots, size_t* off_state, size_t* off_lat, size_t* off_items, size_t* off_stats,
                   size_t* off_last, size_t* off_arena) {
    size_t off = 0;
    *off_state = off;
    off += 256;
    *off_lat = off;
    off = align256(off + (size_t)max_slots * sizeof(BatchLattice));
    *off_items = off;
    off = align256(off + (size_t)max_slots * kMaxTilesPerJob * sizeof(BatchItem));
    *off_stats = off;
    off = align256(off + (size_t)max_slots * kStatFields * 8);
    *off_last = off;
    off = align256(off + (size_t)max_slots * kNumObs * 8);
    *off_arena = off;
}

void retire(shk_server* s, int i, int status, bool fetch) {
    Slot& sl = s->slots[i];
    shk_result r;
    std::memset(&r, 0, sizeof r);
    r.job_id = sl.job_id;
    r.status = status;
    r.steps_done = sl.job.n_steps - sl.remaining;
    r.submit_tick = sl.submit_tick;
    r.admit_tick = sl.admit_tick;
    r.done_tick = s->tick;
    if (fetch) {
        const BatchLattice& B = s->lat[i];
        cudaMemcpyAsync(r.stats, s->dev + s->off_stats + (size_t)i * kStatFields * 8, kStatFields * 8,
                        cudaMemcpyDeviceToHost, s->stream);
        cudaMemcpyAsync(r.last_obs, s->dev + s->off_last + (size_t)i * kNumObs * 8, kNumObs * 8,
                        cudaMemcpyDeviceToHost, s->stream);
        std::vector<unsigned char> sig((size_t)B.L * B.L / 8);
        cudaMemcpyAsync(sig.data(), s->dev + B.sigma_off[B.parity], sig.size(), cudaMemcpyDeviceToHost, s->stream);
        cudaStreamSynchronize(s->stream);
        r.sigma_hash = fnv1a64(sig.data(), sig.size());
    }
    s->done.push_back(r);
    s->arena.release(sl.mem_off, sl.mem_bytes);
    s->used -= sl.mem_bytes;
    sl = Slot();
}

}  // namespace

extern "C" {

size_t shk_server_bytes(int max_slots, size_t arena_bytes) {
    if (max_slots <= 0) return 0;
    size_t a, b, c, d, e, f;
    server_layout(max_slots, &a, &b, &c, &d, &e, &f);
    return f + arena_bytes;
}

int shk_server_create(int max_slots, size_t hbm_budget, void* dev_mem, size_t bytes, void* stream,
                      shk_server** out) {
    if (!out) return sfail(nullptr, SHK_EINVAL, "shk_server_create: out is NULL");
    *out = nullptr;
    if (max_slots <= 0 || max_slots > 65536)
        return sfail(nullptr, SHK_EINVAL, "shk_server_create: max_slots must be in 1..65536");
    if (!dev_mem || (reinterpret_cast<uintptr_t>(dev_mem) & 255u))
        return sfail(nullptr, SHK_EINVAL, "shk_server_create: dev_mem must be non-NULL and 256-byte aligned");
    shk_server* s = new (std::nothrow) shk_server();
    if (!s) return sfail(nullptr, SHK_ENOMEM, "shk_server_create: host allocation failed");
    server_layout(max_slots, &s->off_state, &s->off_lat, &s->off_items, &s->off_stats, &s->off_last,
                  &s->off_arena);
    if (bytes < s->off_arena + 4096) {
        const size_t need = s->off_arena + 4096;
        delete s;
        return sfail(nullptr, SHK_ENOMEM, "shk_server_create: %zu bytes given, at least %zu needed", bytes, need);
    }
    s->max_slots = max_slots;
    s->dev = static_cast<unsigned char*>(dev_mem);
    s->bytes = bytes;
    s->budget = hbm_budget;
    s->stream = static_cast<cudaStream_t>(stream);
    s->arena.reset(bytes - s->off_arena);
    s->slots.resize(max_slots);
    s->lat.resize(max_slots);
    std::memset(s->lat.data(), 0, s->lat.size() * sizeof(BatchLattice));
    cudaError_t e = cudaMemsetAsync(s->dev, 0, s->off_arena, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        delete s;
        return sfail(nullptr, SHK_ECUDA, "shk_server_create: %s", cudaGetErrorString(e));
    }
    *out = s;
    return SHK_OK;
}

void shk_server_destroy(shk_server* s) { delete s; }

const char* shk_server_last_error(const shk_server* s) { return s ? s->err.c_str() : g_server_err.c_str(); }

int shk_server_configure(shk_server* s, int steps_per_launch, int launches_per_tick, int block_threads,
                         int tile_sites, size_t max_pending) {
    if (!s) return sfail(nullptr, SHK_EINVAL, "shk_server_configure: NULL handle");
    if (steps_per_launch < 1 || steps_per_launch > kMaxStepsPerLaunch)
        return sfail(s, SHK_EINVAL, "shk_server_configure: steps_per_launch must be in 1..%d", kMaxStepsPerLaunch);
    if (launches_per_tick < 1 || launches_per_tick > 4096)
        return sfail(s, SHK_EINVAL, "shk_server_configure: launches_per_tick must be in 1..4096");
    if (block_threads != 128 && block_threads != 256 && block_threads != 512)
        return sfail(s, SHK_EINVAL, "shk_server_configure: block_threads must be 128, 256 or 512");
    if (tile_sites < 1024) return sfail(s, SHK_EINVAL, "shk_server_configure: tile_sites must be >= 1024");
    if (max_pending < 1) return sfail(s, SHK_EINVAL, "shk_server_configure: max_pending must be >= 1");
    s->k = steps_per_launch;
    s->launches = launches_per_tick;
    s->block = block_threads;
    s->tile_sites = tile_sites;
    s->max_pending = max_pending;
    return SHK_OK;
}

int shk_server_submit(shk_server* s, const shk_job* job, uint64_t* job_id) {
    if (!s || !job) return sfail(s, SHK_EINVAL, "shk_server_submit: NULL argument");
    if (job->L < 32 || job->L > kMaxServerL || job->L % 32 != 0)
        return sfail(s, SHK_EINVAL, "shk_server_submit: L=%d (need 32 <= L <= %d, L %% 32 == 0)", job->L, kMaxServerL);
    if (!std::isfinite(job->q) || !std::isfinite(job->J))
        return sfail(s, SHK_EINVAL, "shk_server_submit: q and J must be finite");
    if (job->n_steps < 1 || job->n_steps >= SHK_MAX_STEP)
        return sfail(s, SHK_EINVAL, "shk_server_submit: n_steps must be in 1..2^31-1");
    if (job->init_kind != SHK_INIT_ALL_UP && job->init_kind != SHK_INIT_ALL_DOWN && job->init_kind != SHK_INIT_RANDOM)
        return sfail(s, SHK_EINVAL, "shk_server_submit: unknown init_kind %d", job->init_kind);
    if (job_bytes(job->L) > s->budget)
        return sfail(s, SHK_EINVAL, "shk_server_submit: a lattice of side %d needs %zu bytes, more than the HBM budget",
                     job->L, job_bytes(job->L));
    if (s->pending.size() >= s->max_pending) return sfail(s, SHK_EBUSY, "shk_server_submit: queue full");
    const uint64_t id = s->next_id++;
    s->pending.push_back({id, *job, s->tick});
    if (job_id) *job_id = id;
    return SHK_OK;
}

int shk_server_cancel(shk_server* s, uint64_t job_id) {
    if (!s) return sfail(nullptr, SHK_EINVAL, "shk_server_cancel: NULL handle");
    for (auto it = s->pending.begin(); it != s->pending.end(); ++it) {
        if (it->job_id == job_id) {
            shk_result r;
            std::memset(&r, 0, sizeof r);
            r.job_id = job_id;
            r.status = SHK_ECANCELLED;
            r.submit_tick = it->submit_tick;
            r.done_tick = s->tick;
            s->done.push_back(r);
            s->pending.erase(it);
            return SHK_OK;
        }
    }
    for (int i = 0; i < s->max_slots; ++i) {
        if (s->slots[i].used && s->slots[i].job_id == job_id) {
            retire(s, i, SHK_ECANCELLED, false);
            return SHK_OK;
        }
    }
    return sfail(s, SHK_EINVAL, "shk_server_cancel: no queued or running job %llu", (unsigned long long)job_id);
}

int shk_server_tick(shk_server* s, int* n_active, int* n_pending) {
    const TraceRange trace("shk_server_tick");
    if (!s) return sfail(nullptr, SHK_EINVAL, "shk_server_tick: NULL handle");
    cudaError_t e = cudaSuccess;
    // (1) admission, oldest first, while a slot is free and the job fits
    while (!s->pending.empty()) {
        const Pending& p = s->pending.front();
        int slot = -1;
        for (int i = 0; i < s->max_slots; ++i)
            if (!s->slots[i].used) {
                slot = i;
                break;
            }
        if (slot < 0) break;
        const size_t need = job_bytes(p.job.L);
        if (s->used + need > s->budget) break;
        size_t off = 0;
        if (!s->arena.alloc(need, &off)) break;
        Slot& sl = s->slots[slot];
        sl.used = true;
        sl.job_id = p.job_id;
        sl.job = p.job;
        sl.remaining = p.job.n_steps;
        sl.mem_off = off;
        sl.mem_bytes = need;
        sl.submit_tick = p.submit_tick;
        sl.admit_tick = s->tick;
        s->used += need;
        Geometry g;
        make_geometry(p.job.L, kBitpack, &g);
        BatchLattice& B = s->lat[slot];
        std::memset(&B, 0, sizeof B);
        B.L = (uint32_t)p.job.L;
        B.Wr = g.Wr;
        B.div_wr = make_fastdiv(g.Wr);
        const size_t base = s->off_arena + off;
        B.sigma_off[0] = base;
        B.sigma_off[1] = base + g.plane_bytes;
        B.tau_off = base + 2 * g.plane_bytes;
        B.scratch_off = base + 3 * g.plane_bytes;
        B.t = 0;
        B.remaining = p.job.n_steps;
        B.burn_in = p.job.burn_in;
        B.parity = 0;
        uint32_t T[6];
        host_thresholds(p.job.q, p.job.J, T);
        make_draw_params(p.job.seed, p.job.lattice_id, T, 0u, &B.P);
        if (shk_init_plane(SHK_BITPACK, s->dev + B.sigma_off[0], B.L, p.job.init_kind, p.job.init_seed,
                           p.job.lattice_id, 0, s->stream) != SHK_OK ||
            shk_init_plane(SHK_BITPACK, s->dev + B.tau_off, B.L, p.job.init_kind, p.job.init_seed,
                           p.job.lattice_id, 1, s->stream) != SHK_OK)
            return sfail(s, SHK_ECUDA, "shk_server_tick: init: %s", shk_last_error(nullptr));
        e = cudaMemsetAsync(s->dev + B.scratch_off, 0, kScratchPerLattice, s->stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(s->dev + s->off_stats + (size_t)slot * kStatFields * 8, 0, kStatFields * 8, s->stream);
        if (e == cudaSuccess)   // the device copy of the descriptor is authoritative from here on
            e = cudaMemcpyAsync(s->dev + s->off_lat + (size_t)slot * sizeof(BatchLattice), &B, sizeof B,
                                cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return sfail(s, SHK_ECUDA, "shk_server_tick: %s", cudaGetErrorString(e));
        s->pending.pop_front();
    }
    // (2) tiles of every active job, smaller while little work is active so
    // that the launch still spreads over the GPU
    uint64_t active_sites = 0;
    for (int i = 0; i < s->max_slots; ++i)
        if (s->slots[i].used) active_sites += (uint64_t)s->lat[i].L * s->lat[i].L;
    const int64_t target_items = 4 * (int64_t)sm_count() * 2;
    const int64_t tile_sites = std::max<int64_t>(
        4096, std::min<int64_t>(s->tile_sites, (int64_t)(active_sites / (uint64_t)std::max<int64_t>(1, target_items))));
    std::vector<BatchItem> items;
    size_t smem_words = 0;
    for (int i = 0; i < s->max_slots; ++i) {
        if (!s->slots[i].used) continue;
        const BatchLattice& B = s->lat[i];
        uint32_t H = tile_rows_for(B.L, tile_sites);
        H = std::max<uint32_t>(H, (B.L + kMaxTilesPerJob - 1) / kMaxTilesPerJob);
        smem_words = std::max(smem_words, add_tiles(&items, (uint32_t)i, B.L, B.Wr, H, (uint32_t)s->k));
    }
    if (!items.empty()) {
        sort_items(&items, s->lat);
        e = cudaMemcpyAsync(s->dev + s->off_items, items.data(), items.size() * sizeof(BatchItem),
                            cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return sfail(s, SHK_ECUDA, "shk_server_tick upload: %s", cudaGetErrorString(e));
        // reuse the batch launcher through a view of the server's tables
        shk_batch view;
        view.dev = s->dev;
        view.off_state = s->off_state;
        view.off_lat = s->off_lat;
        view.off_items = s->off_items;
        view.off_stats = s->off_stats;
        view.off_last = s->off_last;
        view.n_items = (uint32_t)items.size();
        view.block = s->block;
        view.k = s->k;
        view.smem_bytes = smem_words * 4;
        int grid = 0;
        e = prepare_batch(&view, &grid);
        // several launches per tick: a job that finishes part-way skips its
        // tiles in the remaining launches (the kernel reads its remaining steps)
        for (int l = 0; e == cudaSuccess && l < s->launches; ++l) e = launch_batch(&view, grid, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return sfail(s, SHK_ECUDA, "shk_server_tick launch: %s", cudaGetErrorString(e));
        // (3) host mirror of what the launches did; retire finished jobs
        const uint64_t k = (uint64_t)s->k, per_tick = k * (uint64_t)s->launches;
        for (int i = 0; i < s->max_slots; ++i) {
            Slot& sl = s->slots[i];
            if (!sl.used) continue;
            BatchLattice& B = s->lat[i];
            const uint64_t adv = std::min<uint64_t>(sl.remaining, per_tick);
            const uint64_t nl = (adv + k - 1) / k;           // launches that did work
            B.t += adv;
            B.remaining -= adv;
            B.parity ^= (uint32_t)(nl & 1u);
            sl.remaining -= adv;
        }
        s->tick += 1;
        for (int i = 0; i < s->max_slots; ++i)
            if (s->slots[i].used && s->slots[i].remaining == 0) retire(s, i, SHK_OK, true);
    } else {
        s->tick += 1;
    }
    // (4) deadlines: unfinished jobs whose deadline tick has been reached
    for (int i = 0; i < s->max_slots; ++i) {
        const Slot& sl = s->slots[i];
        if (sl.used && sl.job.deadline_ticks && s->tick >= sl.submit_tick + sl.job.deadline_ticks)
            retire(s, i, SHK_ETIMEOUT, true);
    }
    for (auto it = s->pending.begin(); it != s->pending.end();) {
        if (it->job.deadline_ticks && s->tick >= it->submit_tick + it->job.deadline_ticks) {
            shk_result r;
            std::memset(&r, 0, sizeof r);
            r.job_id = it->job_id;
            r.status = SHK_ETIMEOUT;
            r.submit_tick = it->submit_tick;
            r.done_tick = s->tick;
            s->done.push_back(r);
            it = s->pending.erase(it);
        } else {
            ++it;
        }
    }
    int active = 0;
    for (const Slot& sl : s->slots) active += sl.used ? 1 : 0;
    if (n_active) *n_active = active;
    if (n_pending) *n_pending = (int)s->pending.size();
    return SHK_OK;
}

int shk_server_poll(shk_server* s, shk_result* out, int max, int* n_out) {
    if (!s || (!out && max > 0) || !n_out) return sfail(s, SHK_EINVAL, "shk_server_poll: bad argument");
    const int n = std::min<int>(max, (int)s->done.size());
    for (int i = 0; i < n; ++i) out[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + n);
    *n_out = n;
    return SHK_OK;
}

int shk_server_read_job(shk_server* s, uint64_t job_id, int plane, int8_t* host_out, size_t bytes,
                        uint64_t* steps_done) {
    if (!s || !host_out || !steps_done || (plane != 0 && plane != 1))
        return sfail(s, SHK_EINVAL, "shk_server_read_job: bad argument");
    for (int i = 0; i < s->max_slots; ++i) {
        const Slot& sl = s->slots[i];
        if (!sl.used || sl.job_id != job_id) continue;
        const BatchLattice& B = s->lat[i];
        const size_t off = plane == 0 ? B.sigma_off[B.parity] : B.tau_off;
        const int64_t N = (int64_t)B.L * B.L;
        if (bytes < (size_t)N)
            return sfail(s, SHK_ENOMEM, "shk_server_read_job: %zu bytes given, %lld needed", bytes, (long long)N);
        std::vector<uint32_t> words((size_t)(N / 32));
        cudaError_t e = cudaMemcpyAsync(words.data(), s->dev + off, words.size() * 4, cudaMemcpyDeviceToHost,
                                        s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return sfail(s, SHK_ECUDA, "shk_server_read_job: %s", cudaGetErrorString(e));
        for (int64_t u = 0; u < N; ++u) host_out[u] = ((words[u >> 5] >> (u & 31)) & 1u) ? 1 : -1;
        *steps_done = sl.job.n_steps - sl.remaining;
        return SHK_OK;
    }
    return sfail(s, SHK_EINVAL, "shk_server_read_job: job %llu is not running", (unsigned long long)job_id);
}

int shk_server_stats(shk_server* s, uint64_t* tick, size_t* used_bytes) {
    if (!s) return sfail(nullptr, SHK_EINVAL, "shk_server_stats: NULL handle");
    if (tick) *tick = s->tick;
    if (used_bytes) *used_bytes = s->used;
    return SHK_OK;
}

}  // extern "C"
