// coop.cu -- a whole run of n full steps of one bit-packed lattice in a
// single cooperative launch.
//
// For mid-size lattices (a few hundred thousand to a few million sites per
// plane) a half-step takes a microsecond or two on the GPU, less than the
// host needs to issue its launch.  Here every CTA of the grid is resident
// (cooperative launch, grid of at most one full wave) and a grid barrier
// separates the half-steps, so n steps cost one launch.  The draws, the
// per-step sums and the ring of observable slots are those of the
// per-launch path (Eqs. leftTrans / rightTrans, two-phase draw with the warp
// queue, C_nn of sigma_t reduced in half-step A of step t+1 plus a tail pass).
//
// The barrier spins with a bounded number of polls: a CTA that gives up
// records the timeout in a device status word and the whole kernel returns,
// so a broken barrier cannot hang the GPU; the host then reports
// SHK_ETIMEOUT.
#define SHK_TU_ID 4
#include "internal.h"
#include "sweep.cuh"
#include "prefix.cuh"

namespace shk {

struct CoopArgs {
    uint32_t* sigma;
    uint32_t* tau;
    uint32_t L, Wr, nblocks, n_steps;
    FastDiv div_row;
    uint32_t pad;
    unsigned long long t0;
    long long* obs;        // nullable: n_steps rows of kNumObs, zeroed by the host
    long long* ring;       // 4 slots of 8 int64; slot t0 % 4 zeroed by the host
    unsigned int* bar;     // [0] arrivals, [1] generation, [2] timeout flag; zeroed by the host
    unsigned int spin_limit;
    DrawParams P;
};

// Grid-wide barrier of a cooperative launch.  Thread 0 of each CTA arrives;
// the last arrival resets the count and opens the next generation.  Returns
// false (and raises the timeout flag) if the generation did not move within
// the spin limit, or if another CTA has already timed out.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int spin_limit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int* gen = bar + 1;
        volatile unsigned int* flag = bar + 2;
        const unsigned int my_gen = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
            ok = 1;
        } else {
            unsigned int spins = 0;
            while (*gen == my_gen && *flag == 0u && spins < spin_limit) {
                if (spins >= 1024u) __nanosleep(64);   // poll tightly first, then back off
                ++spins;
            }
            ok = (*gen != my_gen) ? 1 : 0;
            if (!ok) atomicExch(bar + 2, 1u);
        }
        __threadfence();
        if (*flag != 0u) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

// One half-step of the whole plane by this CTA's warps: the two-phase draw
// with the warp queue (as in the per-launch sweep), the fused sums added to
// the slots.  src/dst: bit planes; obs_cur: sums of this step; obs_prev (A
// only, nullable): C_nn of the source plane for the previous step.
template <int HALF>
__device__ __forceinline__ void coop_pass(const CoopArgs& a, const uint32_t* src, uint32_t* dst, uint32_t hs,
                                          const PhiloxPrefix (&pre)[8], uint32_t (*q)[kQueueCap],
                                          long long* obs_cur, long long* obs_prev) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t stride = ((gridDim.x * blockDim.x) >> 5) * 32;
    const uint32_t below = (1u << lane) - 1u;
    const bool cnn = HALF == 0 && obs_prev != nullptr;
    int acc[3] = {0, 0, 0};
    uint32_t head = 0;
    int count = 0;
    auto finish = [&](uint32_t w, uint32_t up, uint32_t S, uint32_t N1, uint32_t N2) {
        *checked(dst, w, a.nblocks, SHK_SITE) = up;
        if (HALF == 0) {
            acc[0] += 2 * __popc(up) - 32;                                               // M_tau
            if (cnn) acc[1] += 64 - 2 * (__popc(S ^ N1) + __popc(S ^ N2));               // C_nn(sigma_{t-1})
        } else {
            acc[0] += 2 * __popc(up) - 32;                                               // M_sigma
            acc[1] += 32 - 2 * __popc(up ^ S);                                           // S_q
            acc[2] += 64 - 2 * (__popc(up ^ N1) + __popc(up ^ N2));                      // S_J
        }
    };
    auto drain = [&](int n) {
        const bool has = (int)lane < n;
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
        const uint32_t res = draw_rest_pre(block_class(S, N1, N2), w, und, up, pre, a.P);
        if (has) finish(w, res, S, N1, N2);
    };
    for (uint32_t base = gwarp * 32; base < a.nblocks; base += stride) {
        const uint32_t w = base + lane;
        const uint32_t row = fdiv(w, a.div_row);
        uint32_t S, N1, N2;
        words_aligned<HALF>(src, w, row, w - row * a.Wr, a.L, a.Wr, a.nblocks, S, N1, N2);
        const BlockClass k = block_class(S, N1, N2);
        uint32_t und, up;
        draw_first_two_pre(k, w, 0xffffffffu, pre, a.P, und, up);
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
            finish(w, up, S, N1, N2);
        }
        count += __popc(mask);
        if (count >= 32) {
            __syncwarp();
            drain(32);
            __syncwarp();
            head = (head + 32) & (kQueueCap - 1);
            count -= 32;
        }
    }
    if (count > 0) {
        __syncwarp();
        drain(count);
    }
    if (HALF == 0) {
        const int v[2] = {acc[0], acc[1]};
        long long* const d[2] = {obs_cur + 1, obs_prev ? obs_prev + 4 : nullptr};
        block_accumulate<2>(v, d);
    } else {
        const int v[3] = {acc[0], acc[1], acc[2]};
        long long* const d[3] = {obs_cur + 0, obs_cur + 2, obs_cur + 3};
        block_accumulate<3>(v, d);
    }
}

__global__ void __launch_bounds__(256, 3) k_run_coop(const __grid_constant__ CoopArgs a) {
    __shared__ uint32_t qbuf[8][6][kQueueCap];
    __shared__ PhiloxPrefix pre[8];
    uint32_t (*q)[kQueueCap] = qbuf[threadIdx.x >> 5];
    auto slot = [&](unsigned long long t) -> long long* {
        return a.obs ? a.obs + (size_t)kNumObs * (t - a.t0) : a.ring + 8 * (t % 4);
    };
    for (uint32_t k = 0; k < a.n_steps; ++k) {
        const unsigned long long t = a.t0 + k;
        // ring mode: clear the next step's slot (nothing reads or writes it in this step)
        if (a.obs == nullptr && k + 1 < a.n_steps && blockIdx.x == 0 && threadIdx.x < kNumObs)
            slot(t + 1)[threadIdx.x] = 0;
        for (int half = 0; half < 2; ++half) {
            const uint32_t hs = (uint32_t)(2 * t + (unsigned long long)half);
            if (threadIdx.x < 8) pre[threadIdx.x] = philox_prefix_dev(a.P, hs, (int)threadIdx.x);
            __syncthreads();
            if (half == 0)
                coop_pass<0>(a, a.sigma, a.tau, hs, pre, q, slot(t), k > 0 ? slot(t - 1) : nullptr);
            else
                coop_pass<1>(a, a.tau, a.sigma, hs, pre, q, slot(t), nullptr);
            if (!grid_barrier(a.bar, a.spin_limit)) return;
        }
    }
    // tail pass: C_nn of the final sigma into the last step's slot
    long long* last = slot(a.t0 + a.n_steps - 1);
    int c = 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < a.nblocks; w += stride) {
        const uint32_t row = fdiv(w, a.div_row);
        uint32_t S, N1, N2;
        words_aligned<0>(a.sigma, w, row, w - row * a.Wr, a.L, a.Wr, a.nblocks, S, N1, N2);
        c += 64 - 2 * (__popc(S ^ N1) + __popc(S ^ N2));
    }
    const int v[1] = {c};
    long long* const d[1] = {last + 4};
    block_accumulate<1>(v, d);
}

// For the failure test only: two CTAs wait at a barrier whose arrival count
// the host has started past the last arrival, so the wait can only end by the
// spin limit.
__global__ void __launch_bounds__(256) k_barrier_probe(unsigned int* bar, unsigned int spin_limit) {
    (void)grid_barrier(bar, spin_limit);
}

// Largest resident grid of k_run_coop (one full wave), 0 if the device cannot
// launch cooperatively.
static int coop_grid() {
    static int grid = -1;
    if (grid < 0) {
        int dev = 0, coop = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        grid = coop ? blocks_per_sm(reinterpret_cast<const void*>(k_run_coop), 256) * sm_count() : 0;
    }
    return grid;
}

bool coop_path_fits(const Geometry& g) {
    // bit-packed, past the one-CTA path, and small enough that launches,
    // not the sweeps, dominate the per-launch path
    return g.layout == kBitpack && g.aligned && g.N > 65536 && g.L <= 4096 && coop_grid() > 0;
}

cudaError_t launch_run_coop(const Geometry& g, void* sigma, void* tau, const DrawParams& P, uint64_t t0,
                            uint64_t n, long long* obs, long long* ring, unsigned int* bar,
                            unsigned int spin_limit, cudaStream_t st) {
    CoopArgs a;
    a.sigma = static_cast<uint32_t*>(sigma);
    a.tau = static_cast<uint32_t*>(tau);
    a.L = (uint32_t)g.L;
    a.Wr = g.Wr;
    a.nblocks = g.nblocks;
    a.n_steps = (uint32_t)n;
    a.div_row = make_fastdiv(g.Wr);
    a.pad = 0;
    a.t0 = t0;
    a.obs = obs;
    a.ring = ring;
    a.bar = bar;
    a.spin_limit = spin_limit;
    a.P = P;
    const int need = (int)std::min<uint64_t>((g.nblocks + 255) / 256, (uint64_t)coop_grid());
    const int grid = std::max(1, need);
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_run_coop), grid, 256, args, 0, st);
}

cudaError_t launch_barrier_probe(unsigned int* bar, unsigned int spin_limit, cudaStream_t st) {
    // two CTAs; the caller starts the arrival count past the last arrival
    void* args[] = {&bar, &spin_limit};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_barrier_probe), 2, 256, args, 0, st);
}

unsigned bounds_site_coop() { return take_bounds_site(); }

}  // namespace shk
