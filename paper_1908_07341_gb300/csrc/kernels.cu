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
#include "sweep_kernels.cuh"

namespace shk {

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

// Set non-zero by a sweep whose bounded wait on its own copies gave up; read
// and cleared by sweep_fault_take (shk_sweep_status and the lattice reads).
__device__ unsigned int g_sweep_fault;

// Device address of the fault word on the current device, looked up at each
// use (cheap next to a launch), so that it never outlives its context.
cudaError_t sweep_fault_word(unsigned int** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sweep_fault);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned int*>(p);
    return cudaSuccess;
}

// Reads and clears the fault word after synchronising `st`: true if a wait
// gave up since the last call.
cudaError_t sweep_fault_take(cudaStream_t st, bool* fault) {
    unsigned int v = 0;
    const unsigned int zero = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, g_sweep_fault, sizeof v);
    if (e == cudaSuccess && v != 0u) e = cudaMemcpyToSymbol(g_sweep_fault, &zero, sizeof zero);
    *fault = v != 0u;
    return e;
}

// One warp arms an mbarrier for 16 bytes that no copy will deliver and waits
// for it, bounded by limit_cycles: the wait gives up, the kernel sets the
// fault word and returns.  Nothing is in flight, so nothing else happens.
__global__ void k_bulk_wait_probe(unsigned int* fault, long long limit_cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncwarp();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16u);
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar, 0u, limit_cycles));
    if (!ok && threadIdx.x == 0) atomicOr(fault, 1u);
}

cudaError_t launch_bulk_wait_probe(long long limit_cycles, cudaStream_t st) {
    unsigned int* f = nullptr;
    cudaError_t e = sweep_fault_word(&f);
    if (e != cudaSuccess) return e;
    k_bulk_wait_probe<<<1, 32, 0, st>>>(f, limit_cycles);
    return cudaGetLastError();
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
    a.fault = nullptr;
    return a;
}

// ------------------------------------------------------------ sweep variants
//
// Launch shapes of the half-step sweeps, chosen per layout at run time
// (shk_set_sweep_variant; the autotuner times them and picks one).


struct SweepVariant {
    SweepKernel k[2];   // half A, half B
    int block;
    int row_blocks;     // rows must hold a multiple of this many blocks (32: L % 1024 == 0)
    const char* name;
    const char* jit[2]; // the same kernels as name expressions for run-time compilation (jit.cu), or null
    int waves;          // grid: at most this many full waves of resident blocks
    bool bulk;          // moves rows with bounded waits on bulk copies: gets the fault word
};

#define SHK_JIT_NAMES(kernel, args) {"shk::" #kernel "<0, " args ">", "shk::" #kernel "<1, " args ">"}

// The first entry of each table is the default (the fastest measured at
// L = 16384 on GB300); the autotuner may pick another per size.
static const SweepVariant kBpVariants[] = {
    {{k_sweep_qv<0, 4, 256, 3>, k_sweep_qv<1, 4, 256, 3>}, 256, 4, "queue-v4-256x3",
     SHK_JIT_NAMES(k_sweep_qv, "4, 256, 3")},
    {{k_sweep_qv<0, 4, 256, 3>, k_sweep_qv<1, 4, 256, 3>}, 256, 4, "queue-v4-256x3-w2",
     SHK_JIT_NAMES(k_sweep_qv, "4, 256, 3"), 2},
    {{k_sweep_qv<0, 4, 256, 3>, k_sweep_qv<1, 4, 256, 3>}, 256, 4, "queue-v4-256x3-w4",
     SHK_JIT_NAMES(k_sweep_qv, "4, 256, 3"), 4},
    {{k_sweep_q<0, kBitpack, 256, 3>, k_sweep_q<1, kBitpack, 256, 3>}, 256, 1, "queue-256x3",
     SHK_JIT_NAMES(k_sweep_q, "1, 256, 3")},
    {{k_sweep_qv<0, 2, 256, 3>, k_sweep_qv<1, 2, 256, 3>}, 256, 2, "queue-v2-256x3",
     SHK_JIT_NAMES(k_sweep_qv, "2, 256, 3")},
    {{k_sweep_qv<0, 4, 256, 2>, k_sweep_qv<1, 4, 256, 2>}, 256, 4, "queue-v4-256x2",
     SHK_JIT_NAMES(k_sweep_qv, "4, 256, 2")},
    {{k_sweep_strip_async<0, kBitpack, 256, 3, 4>, k_sweep_strip_async<1, kBitpack, 256, 3, 4>}, 256, 32,
     "strip-async4-256x3", SHK_JIT_NAMES(k_sweep_strip_async, "1, 256, 3, 4")},
    {{k_sweep_strip<0, kBitpack, 256, 3>, k_sweep_strip<1, kBitpack, 256, 3>}, 256, 32, "strip-256x3",
     SHK_JIT_NAMES(k_sweep_strip, "1, 256, 3")},
    {{k_sweep_q<0, kBitpack, 128, 6>, k_sweep_q<1, kBitpack, 128, 6>}, 128, 1, "queue-128x6",
     SHK_JIT_NAMES(k_sweep_q, "1, 128, 6")},
    {{k_sweep_q<0, kBitpack, 256, 4>, k_sweep_q<1, kBitpack, 256, 4>}, 256, 1, "queue-256x4",
     SHK_JIT_NAMES(k_sweep_q, "1, 256, 4")},
    {{k_sweep_bp<0, 1, false, 256, 1>, k_sweep_bp<1, 1, false, 256, 1>}, 256, 1, "plain-256", {nullptr, nullptr}},
};

static const SweepVariant kI8Variants[] = {
    {{k_sweep_strip_async<0, kInt8, 256, 3, 2>, k_sweep_strip_async<1, kInt8, 256, 3, 2>}, 256, 32,
     "strip-async2-256x3", SHK_JIT_NAMES(k_sweep_strip_async, "2, 256, 3, 2")},
    {{k_sweep_strip_async<0, kInt8, 256, 3, 2>, k_sweep_strip_async<1, kInt8, 256, 3, 2>}, 256, 32,
     "strip-async2-256x3-w2", SHK_JIT_NAMES(k_sweep_strip_async, "2, 256, 3, 2"), 2},
    {{k_sweep_strip_bulk<0, 256, 3, 4>, k_sweep_strip_bulk<1, 256, 3, 4>}, 256, 32, "strip-bulk4-256x3",
     SHK_JIT_NAMES(k_sweep_strip_bulk, "256, 3, 4"), 1, true},
    {{k_sweep_strip<0, kInt8, 256, 3>, k_sweep_strip<1, kInt8, 256, 3>}, 256, 32, "strip-256x3",
     SHK_JIT_NAMES(k_sweep_strip, "2, 256, 3")},
    {{k_sweep_q<0, kInt8, 256, 3>, k_sweep_q<1, kInt8, 256, 3>}, 256, 1, "queue-256x3",
     SHK_JIT_NAMES(k_sweep_q, "2, 256, 3")},
    {{k_sweep_q<0, kInt8, 256, 4>, k_sweep_q<1, kInt8, 256, 4>}, 256, 1, "queue-256x4",
     SHK_JIT_NAMES(k_sweep_q, "2, 256, 4")},
    {{k_sweep_i8a<0, false, 256, 1>, k_sweep_i8a<1, false, 256, 1>}, 256, 1, "plain-256", {nullptr, nullptr}},
};

constexpr int kNumBpVariants = sizeof(kBpVariants) / sizeof(kBpVariants[0]);
constexpr int kNumI8Variants = sizeof(kI8Variants) / sizeof(kI8Variants[0]);
constexpr int kBpRowFallback = 3;   // variant used when rows are too short for the chosen one (queue-256x3)
constexpr int kI8RowFallback = 4;

static std::atomic<int> g_bp_variant{0};
static std::atomic<int> g_i8_variant{0};

int sweep_variant_count(int layout) {
    return layout == kBitpack ? kNumBpVariants : layout == kInt8 ? kNumI8Variants : 0;
}

bool sweep_variant_jit(int layout, int v, const char** e0, const char** e1, int* block) {
    if (v < 0 || v >= sweep_variant_count(layout)) return false;
    const SweepVariant& sv = layout == kBitpack ? kBpVariants[v] : kI8Variants[v];
    *e0 = sv.jit[0];
    *e1 = sv.jit[1];
    *block = sv.block;
    return true;
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
                            long long* obs_prev, long long* zero_slot, cudaStream_t st,
                            bool loaded_only) {
    SweepArgs a = sweep_args(g, src, dst, P, hs, obs_cur, half == 0 ? obs_prev : nullptr, zero_slot);
    if (g.layout == kBitpack || g.aligned) {
        const SweepVariant* table = g.layout == kBitpack ? kBpVariants : kI8Variants;
        int vi = g.layout == kBitpack ? g_bp_variant.load() : g_i8_variant.load();
        const int fallback = g.layout == kBitpack ? kBpRowFallback : kI8RowFallback;
        // strip-walk and vector variants need rows of a multiple of their block count
        if ((g.Wr % (uint32_t)table[vi].row_blocks) != 0) vi = fallback;
        // a vector variant (V blocks per thread) below one full wave of threads
        // leaves SMs idle: the one-block-per-thread queue sweep is faster there
        // (at L <= 2048 on a GB300)
        const int rb = table[vi].row_blocks;
        if (rb > 1 && rb < 32 && g.nblocks / (uint32_t)rb < (uint32_t)(sm_count() * 768)) vi = fallback;
        const SweepVariant& v = table[vi];
        cudaError_t e = cudaSuccess;
        const int waves = v.waves > 0 ? v.waves : 1;
        if (v.bulk) {
            const cudaError_t fe = sweep_fault_word(&a.fault);
            if (fe != cudaSuccess) return fe;
        }
        if (jit_launch(v.jit[0], v.jit[1], v.block, half, g.nblocks, a, st, &e, loaded_only, waves)) return e;
        SweepKernel k = v.k[half];
        return launch_pdl(k, grid_for(k, v.block, g.nblocks, waves), v.block, st, a);
    } else {
        const int block = 256;
        SweepKernel k = half == 0 ? k_sweep_i8g<0> : k_sweep_i8g<1>;
        return launch_pdl(k, grid_for(k, block, g.nblocks), block, st, a);
    }
    return cudaGetLastError();
}

cudaError_t launch_cnn(const Geometry& g, const void* sigma, long long* obs, cudaStream_t st) {
    DrawParams P{};
    const SweepArgs a = sweep_args(g, sigma, nullptr, P, 0, obs, nullptr, nullptr);
    const int block = 256;
    SweepKernel k = g.layout == kBitpack ? k_cnn<kBitpack, true> : g.aligned ? k_cnn<kInt8, true> : k_cnn<kInt8, false>;
    return launch_pdl(k, grid_for(k, block, g.nblocks), block, st, a);
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
    // Lattices up to 2^15 sites per plane (L <= 181) run faster inside one CTA
    // than as a sequence of grid-wide launches: on a GB300 a step takes 2.6 us
    // at L = 128 in one CTA, 8.3 us at L = 256, against about 5 us on the grid
    // path (whose launches overlap, see pdl_begin) from L = 256 to 1024.
    return g.N <= 32768;
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
