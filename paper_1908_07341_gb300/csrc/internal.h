// internal.h -- host-side interface between the C ABI (api.cu) and the
// kernel launchers (kernels.cu).  Not installed; not part of the ABI.
#pragma once

#include <atomic>
#include <cstddef>
#include <string>
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "device.cuh"

namespace shk {

// Geometry of one L x L plane in a layout.
struct Geometry {
    int L = 0;
    int layout = 0;
    int64_t N = 0;          // L * L sites
    uint32_t nblocks = 0;   // 32-site blocks: ceil(N / 32)
    uint32_t Wr = 0;        // bit-packed words (32-site blocks) per row, L % 32 == 0 only
    bool aligned = false;   // L % 32 == 0
    size_t plane_bytes = 0; // device bytes of one plane (padded to 256)
};

bool make_geometry(int L, int layout, Geometry* g);
FastDiv make_fastdiv(uint32_t d);

// Host-side threshold table (own implementation of the rule in shaken.h).
int host_thresholds(double q, double J, uint32_t out[6]);

// Draw parameters for a seed / lattice id / table; false if the table breaks
// the complement rule T[k] + T[5-k] = 2^32.
bool make_draw_params(uint64_t seed, uint32_t lattice_id, const uint32_t T[6], uint32_t domain,
                      DrawParams* P);

// One half-step over a plane.  obs_cur receives the reductions of the drawn
// plane (A: M_tau at [1]; B: M_sigma [0], S_q [2], S_J [3]); obs_prev (A only,
// nullable) receives C_nn of the source plane at [4]; zero_slot (nullable)
// is cleared by the launch (five int64).
// loaded_only: launch a run-time specialised sweep only if it is already
// compiled and loaded on this device; never queue a compile, compile, load a
// module or wait (the allocation-free entry point), else the generic kernel.
cudaError_t launch_halfstep(const Geometry& g, int half, const void* src, void* dst,
                            const DrawParams& P, uint32_t hs, long long* obs_cur,
                            long long* obs_prev, long long* zero_slot, cudaStream_t st,
                            bool loaded_only = false);

// Launch-shape variants of the half-step sweeps (per layout; the int8 table
// applies to L % 32 == 0).  The choice is process-wide.
int sweep_variant_count(int layout);
const char* sweep_variant_name(int layout, int v);
int get_sweep_variant(int layout);
bool set_sweep_variant(int layout, int v);

// Diagonal correlation sums of a bit-packed plane added to out (SW-NE then
// NW-SE, n_lags each; n_lags <= 8).
cudaError_t launch_diag_corr(const Geometry& g, const void* plane, const int* lags, int n_lags, long long* out,
                             cudaStream_t st);

// Coupled top/bottom chains (coalescence times); one CTA per pair.
size_t coalesce_smem_bytes(int L);
size_t coalesce_pair_bytes();
void fill_coalesce_pair(void* dst, int L, const DrawParams& P);
constexpr int kDynShaken = 0, kDynCheckerboard = 1;
cudaError_t launch_cftp(int dyn, const void* pairs, uint32_t n_pairs, int max_L, int k_max, uint32_t* samples,
                        uint32_t sample_words, int* k_out, cudaStream_t st);
cudaError_t launch_coalesce(int dyn, const void* pairs, uint32_t n_pairs, int max_L, uint64_t max_steps,
                            unsigned long long* T, cudaStream_t st);

// Checkerboard heat-bath half-step in place on a bit-packed plane; after the
// odd half (parity 1) the magnetisation and C_nn are added to obs[0..1]
// (obs nullable).
cudaError_t launch_checkerboard(const Geometry& g, void* plane, const DrawParams& P, uint32_t hs, int parity,
                                long long* obs, cudaStream_t st);

// C_nn of a sigma plane added to obs[4].
cudaError_t launch_cnn(const Geometry& g, const void* sigma, long long* obs, cudaStream_t st);

// Initial state of one plane.
cudaError_t launch_init(const Geometry& g, void* plane, int kind, uint64_t init_seed,
                        uint32_t lattice_id, uint32_t plane_index, cudaStream_t st);

// Whole run of n steps inside one CTA (both planes in shared memory).
// obs (nullable) gets n rows of five sums; last gets the last row.
bool small_path_fits(const Geometry& g);
cudaError_t launch_run_small(const Geometry& g, void* sigma, void* tau, const DrawParams& P,
                             uint64_t t0, uint64_t n, long long* obs, long long* last,
                             cudaStream_t st);

// Fault word of the sweeps' bounded waits on their own bulk copies: its
// device address, a synchronising read-and-clear, and a probe kernel whose
// wait cannot complete (the failure path, tested without a fault).
cudaError_t sweep_fault_word(unsigned int** out);
cudaError_t sweep_fault_take(cudaStream_t st, bool* fault);
cudaError_t launch_bulk_wait_probe(long long limit_cycles, cudaStream_t st);

// True when p is 16-byte aligned (the sweeps use 16-byte vector accesses).
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

// Number of SMs of the current device (cached).
int sm_count();

// Message returned by shk_last_error(NULL) on this host thread.
void set_thread_error(const char* msg);

// Half-step sweeps compiled at run time for one threshold table (jit.cu).
// jit_launch launches half `half` of the kernel pair named e0 / e1 and
// returns true, or returns false without launching when no such kernel is
// ready (disabled, compile still queued or running, no NVRTC,
// compile failure).  g_jit_mode: 0 off, 1 compile in the background
// (default), 2 compile at first use and wait for it.
struct SweepArgs;
bool jit_launch(const char* e0, const char* e1, int block, int half, uint32_t work_items, const SweepArgs& a,
                cudaStream_t st, cudaError_t* err, bool loaded_only = false, int waves = 1);
extern std::atomic<int> g_jit_mode;
// Queues (wait: and waits for) the specialised compile of sweep variant
// `variant` of `layout` for threshold table T; SHK_OK or an error status with
// the reason in *why.
int jit_prepare(int layout, int variant, const uint32_t T[6], bool wait, std::string* why);
// The run-time compilation names of a sweep variant (null when it has none)
// and its block size; false for an unknown (layout, variant).
bool sweep_variant_jit(int layout, int variant, const char** e0, const char** e1, int* block);

// First bounds-check failure site recorded by each translation unit in the
// debug build (0 = none; always 0 in the normal build), cleared on read.
unsigned bounds_site_kernels();
unsigned bounds_site_batch();
unsigned bounds_site_sampling();

// Named range on the host timeline for profilers that record NVTX (no-op
// when no tool is attached).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace shk
