// api.cu -- the extern "C" interface declared in include/shaken.h.
//
// Host runtime of the library: argument validation, the threshold table,
// lattice handles over caller-owned device memory, dispatch of a run to the
// one-CTA path (small lattices) or to the grid-wide half-step sweeps, and the
// observable ring that keeps the last step's sums on the device.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "shaken.h"
#include "internal.h"
#include "bounds.cuh"

namespace shk {

// Philox4x32 Weyl key increments (Salmon et al., 2011).
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    uint32_t s = 0;
    while ((1ull << s) < d) ++s;
    f.s = s;
    const unsigned __int128 num = ((unsigned __int128)1 << 32) * (((unsigned __int128)1 << s) - d);
    f.m = (uint32_t)(num / d + 1);
    return f;
}

bool make_geometry(int L, int layout, Geometry* g) {
    if (L < 2 || L > SHK_MAX_L) return false;
    if (layout != kBitpack && layout != kInt8) return false;
    if (layout == kBitpack && (L % 32) != 0) return false;
    g->L = L;
    g->layout = layout;
    g->N = (int64_t)L * L;
    g->nblocks = (uint32_t)((g->N + 31) / 32);
    g->aligned = (L % 32) == 0;
    g->Wr = g->aligned ? (uint32_t)(L / 32) : 0u;
    const size_t raw = layout == kBitpack ? (size_t)g->N / 8 : (size_t)g->N;
    g->plane_bytes = (raw + 255) & ~(size_t)255;
    return true;
}

static uint32_t threshold_of(double h) {
    if (h == 0.0) return 0x80000000u;
    const double a = std::fabs(h);
    const double p = 1.0 / (1.0 + std::exp(-2.0 * a));
    const double fl = std::floor(std::ldexp(p, 32));
    const uint32_t pos = fl >= 4294967295.0 ? 0xffffffffu : (uint32_t)fl;
    return h > 0.0 ? pos : (uint32_t)(0u - pos);
}

int host_thresholds(double q, double J, uint32_t out[6]) {
    if (!std::isfinite(q) || !std::isfinite(J) || out == nullptr) return SHK_EINVAL;
    for (int k = 0; k < 6; ++k) {
        const double s = (k >= 3) ? 1.0 : -1.0;
        const int n = k % 3;
        out[k] = threshold_of(q * s + J * (double)(2 * n - 2));
    }
    return SHK_OK;
}

bool make_draw_params(uint64_t seed, uint32_t lattice_id, const uint32_t T[6], uint32_t domain,
                      DrawParams* P) {
    for (int n = 0; n < 3; ++n)
        if ((uint64_t)T[n] + (uint64_t)T[5 - n] != (1ull << 32)) return false;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (uint32_t r = 0; r < 10; ++r) {
        P->rk0[r] = k0 + r * kPhiloxW0;
        P->rk1[r] = k1 + r * kPhiloxW1;
    }
    const uint32_t U[3] = {T[3], T[4], T[5]};
    for (int b = 0; b < 32; ++b) {
        uint32_t m[3];
        for (int k = 0; k < 3; ++k) m[k] = ((U[k] >> (31 - b)) & 1u) ? 0xffffffffu : 0u;
        P->m0[b] = m[0];
        P->d01[b] = m[0] ^ m[1];
        P->d12[b] = m[1] ^ m[2];
    }
    P->lattice_id = lattice_id;
    P->c3_base = 256u * domain;
    return true;
}

}  // namespace shk

using namespace shk;

struct shk_lattice {
    Geometry g;
    unsigned char* dev = nullptr;
    size_t bytes = 0;
    void* plane[2] = {nullptr, nullptr};
    long long* ring = nullptr;      // 4 slots x 8 int64
    long long* last_obs = nullptr;  // device row of the last completed step
    cudaStream_t stream = nullptr;
    double q = 0.0, J = 0.0;
    uint32_t T[6] = {0, 0, 0, 0, 0, 0};
    bool params_set = false;
    uint64_t seed = 0;
    uint32_t lattice_id = 0;
    uint64_t step = 0;
    std::string err;
};

namespace {

thread_local std::string g_thread_err;

int fail(shk_lattice* lat, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (lat) lat->err = buf;
    else g_thread_err = buf;
    return code;
}

int cuda_fail(shk_lattice* lat, cudaError_t e, const char* what) {
    return fail(lat, SHK_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

constexpr size_t kRingBytes = 512;   // 4 observable slots of 8 int64, then 256 reserved bytes

}  // namespace

void shk::set_thread_error(const char* msg) { g_thread_err = msg ? msg : ""; }

extern "C" {

const char* shk_strerror(int status) {
    switch (status) {
        case SHK_OK: return "ok";
        case SHK_EINVAL: return "invalid argument";
        case SHK_ENOMEM: return "buffer too small";
        case SHK_ECUDA: return "CUDA error";
        case SHK_ESTATE: return "handle not ready";
        case SHK_EBUSY: return "busy";
        case SHK_ETIMEOUT: return "timed out";
        case SHK_ECANCELLED: return "cancelled";
        default: return "unknown status";
    }
}

const char* shk_last_error(const void* handle) {
    if (handle == nullptr) return g_thread_err.c_str();
    return static_cast<const shk_lattice*>(handle)->err.c_str();
}

int shk_version(void) { return 100; }

int shk_debug_bounds(uint32_t* first_site) {
    if (first_site == nullptr) return fail(nullptr, SHK_EINVAL, "shk_debug_bounds: first_site is NULL");
    *first_site = 0;
    if (!kBoundsChecked)
        return fail(nullptr, SHK_ESTATE, "shk_debug_bounds: the library was built without bounds checks");
    const unsigned sites[3] = {bounds_site_kernels(), bounds_site_batch(), bounds_site_sampling()};
    for (unsigned v : sites)
        if (v != 0 && *first_site == 0) *first_site = v;
    return SHK_OK;
}

int shk_thresholds(double q, double J, uint32_t out[6]) {
    const int rc = host_thresholds(q, J, out);
    if (rc != SHK_OK) return fail(nullptr, rc, "shk_thresholds: q and J must be finite and out non-NULL");
    return SHK_OK;
}

size_t shk_plane_bytes(int L, int layout) {
    Geometry g;
    return make_geometry(L, layout, &g) ? g.plane_bytes : 0;
}

// Plane pointers of the stateless calls: the kernels read and write them in
// 16-byte vectors.
int shk_halfstep(int layout, int half, const void* src, void* dst, int L, const uint32_t T[6],
                 uint64_t seed, uint32_t lattice_id, uint32_t hs, int64_t* obs_accum,
                 void* stream) {
    Geometry g;
    if (!make_geometry(L, layout, &g))
        return fail(nullptr, SHK_EINVAL, "shk_halfstep: invalid L=%d for layout %d", L, layout);
    if (half != SHK_HALF_A && half != SHK_HALF_B)
        return fail(nullptr, SHK_EINVAL, "shk_halfstep: half must be SHK_HALF_A or SHK_HALF_B");
    if (src == nullptr || dst == nullptr || T == nullptr || src == dst)
        return fail(nullptr, SHK_EINVAL, "shk_halfstep: src, dst, T must be non-NULL and src != dst");
    if (!aligned16(src) || !aligned16(dst))
        return fail(nullptr, SHK_EINVAL, "shk_halfstep: src and dst must be 16-byte aligned");
    DrawParams P;
    if (!make_draw_params(seed, lattice_id, T, 0u, &P))
        return fail(nullptr, SHK_EINVAL, "shk_halfstep: threshold table violates T[k] + T[5-k] = 2^32");
    long long* acc = reinterpret_cast<long long*>(obs_accum);
    const cudaError_t e = launch_halfstep(g, half, src, dst, P, hs, acc, acc, nullptr,
                                          static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "shk_halfstep launch");
    return SHK_OK;
}

int shk_sweep_variant_count(int layout) { return sweep_variant_count(layout); }

const char* shk_sweep_variant_name(int layout, int variant) { return sweep_variant_name(layout, variant); }

int shk_get_sweep_variant(int layout) {
    if (sweep_variant_count(layout) == 0)
        return fail(nullptr, SHK_EINVAL, "shk_get_sweep_variant: unknown layout %d", layout);
    return get_sweep_variant(layout);
}

int shk_set_sweep_variant(int layout, int variant) {
    if (!set_sweep_variant(layout, variant))
        return fail(nullptr, SHK_EINVAL, "shk_set_sweep_variant: no variant %d for layout %d", variant, layout);
    return SHK_OK;
}

int shk_diag_correlations(const void* plane, int L, const int* lags, int n_lags, int64_t* out, void* stream) {
    Geometry g;
    if (!make_geometry(L, kBitpack, &g))
        return fail(nullptr, SHK_EINVAL, "shk_diag_correlations: L=%d must be a multiple of 32 in 32..%d", L, SHK_MAX_L);
    if (plane == nullptr || out == nullptr || lags == nullptr)
        return fail(nullptr, SHK_EINVAL, "shk_diag_correlations: NULL argument");
    if (!aligned16(plane)) return fail(nullptr, SHK_EINVAL, "shk_diag_correlations: plane must be 16-byte aligned");
    if (n_lags < 1 || n_lags > 8) return fail(nullptr, SHK_EINVAL, "shk_diag_correlations: n_lags must be 1..8");
    for (int k = 0; k < n_lags; ++k)
        if (lags[k] < 0 || lags[k] >= L)
            return fail(nullptr, SHK_EINVAL, "shk_diag_correlations: lag %d outside 0..L-1", lags[k]);
    const cudaError_t e = launch_diag_corr(g, plane, lags, n_lags, reinterpret_cast<long long*>(out),
                                           static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "shk_diag_correlations launch");
    return SHK_OK;
}

int shk_checkerboard_thresholds(double J, uint32_t out[5]) {
    if (!std::isfinite(J) || out == nullptr)
        return fail(nullptr, SHK_EINVAL, "shk_checkerboard_thresholds: J must be finite and out non-NULL");
    for (int n = 0; n < 5; ++n) out[n] = threshold_of(J * (double)(2 * n - 4));
    return SHK_OK;
}

// The checkerboard draw folded onto the three-class machinery: a six-entry
// table whose upper half is (T[2], T[3], T[4]) and whose lower half is its
// complement, with the checkerboard stream domain 2.
static bool checkerboard_draw_params(double J, uint64_t seed, uint32_t lattice_id, DrawParams* P) {
    uint32_t T5[5];
    if (!std::isfinite(J)) return false;
    for (int n = 0; n < 5; ++n) T5[n] = threshold_of(J * (double)(2 * n - 4));
    const uint32_t T6[6] = {0u - T5[4], 0u - T5[3], 0u - T5[2], T5[2], T5[3], T5[4]};
    return make_draw_params(seed, lattice_id, T6, 2u, P);
}

int shk_checkerboard_run(void* plane, int L, double J, uint64_t seed, uint32_t lattice_id, uint64_t t0,
                         uint64_t n_steps, int64_t* dev_obs, void* stream) {
    const TraceRange trace("shk_checkerboard_run");
    Geometry g;
    if (!make_geometry(L, kBitpack, &g))
        return fail(nullptr, SHK_EINVAL, "shk_checkerboard_run: L=%d must be a multiple of 32 in 32..%d", L, SHK_MAX_L);
    if (plane == nullptr) return fail(nullptr, SHK_EINVAL, "shk_checkerboard_run: plane is NULL");
    if (!aligned16(plane)) return fail(nullptr, SHK_EINVAL, "shk_checkerboard_run: plane must be 16-byte aligned");
    if (t0 > SHK_MAX_STEP || n_steps > SHK_MAX_STEP - t0)
        return fail(nullptr, SHK_EINVAL, "shk_checkerboard_run: step index would exceed 2^31");
    DrawParams P;
    if (!checkerboard_draw_params(J, seed, lattice_id, &P))
        return fail(nullptr, SHK_EINVAL, "shk_checkerboard_run: J must be finite");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (dev_obs) {
        const cudaError_t e = cudaMemsetAsync(dev_obs, 0, (size_t)n_steps * 2 * sizeof(int64_t), st);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "shk_checkerboard_run memset");
    }
    for (uint64_t k = 0; k < n_steps; ++k) {
        const uint64_t t = t0 + k;
        long long* row = dev_obs ? reinterpret_cast<long long*>(dev_obs) + 2 * k : nullptr;
        cudaError_t e = launch_checkerboard(g, plane, P, (uint32_t)(2 * t), 0, nullptr, st);
        if (e == cudaSuccess) e = launch_checkerboard(g, plane, P, (uint32_t)(2 * t + 1), 1, row, st);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "shk_checkerboard_run launch");
    }
    return SHK_OK;
}

// Validates the pairs of shk_coalescence_times / shk_cftp and writes their
// descriptors to host; returns SHK_OK and the largest L, or an error.
static int build_pairs(const char* who, int dynamics, int n_pairs, const int* L, const double* q,
                       const double* J, const uint64_t* seed, const uint32_t* lattice_id,
                       std::vector<unsigned char>& host, int* max_L) {
    if (dynamics != SHK_DYN_SHAKEN && dynamics != SHK_DYN_CHECKERBOARD)
        return fail(nullptr, SHK_EINVAL, "%s: unknown dynamics %d", who, dynamics);
    if (n_pairs <= 0 || !L || !J || !seed || !lattice_id || (dynamics == SHK_DYN_SHAKEN && !q))
        return fail(nullptr, SHK_EINVAL, "%s: bad argument", who);
    host.assign((size_t)n_pairs * coalesce_pair_bytes(), 0);
    *max_L = 32;
    for (int i = 0; i < n_pairs; ++i) {
        if (L[i] < 32 || L[i] > 256 || L[i] % 32 != 0)
            return fail(nullptr, SHK_EINVAL, "%s: pair %d has L=%d (need 32..256, L %% 32 == 0)", who, i, L[i]);
        DrawParams P;
        bool ok;
        if (dynamics == SHK_DYN_SHAKEN) {
            uint32_t T[6];
            ok = host_thresholds(q[i], J[i], T) == SHK_OK && make_draw_params(seed[i], lattice_id[i], T, 0u, &P);
        } else {
            ok = checkerboard_draw_params(J[i], seed[i], lattice_id[i], &P);
        }
        if (!ok) return fail(nullptr, SHK_EINVAL, "%s: pair %d has non-finite parameters", who, i);
        fill_coalesce_pair(host.data() + (size_t)i * coalesce_pair_bytes(), L[i], P);
        *max_L = std::max(*max_L, L[i]);
    }
    return SHK_OK;
}

static size_t pairs_bytes_aligned(int n_pairs) {
    return ((size_t)n_pairs * coalesce_pair_bytes() + 255) & ~(size_t)255;
}

size_t shk_coalescence_scratch_bytes(int n_pairs) {
    if (n_pairs <= 0) return 0;
    return pairs_bytes_aligned(n_pairs) + (size_t)n_pairs * 8;
}

int shk_coalescence_times(int dynamics, int n_pairs, const int* L, const double* q, const double* J,
                          const uint64_t* seed, const uint32_t* lattice_id, uint64_t max_steps, void* dev_scratch,
                          size_t bytes, uint64_t* host_T, void* stream) {
    const TraceRange trace("shk_coalescence_times");
    if (!dev_scratch || !host_T) return fail(nullptr, SHK_EINVAL, "shk_coalescence_times: bad argument");
    if (max_steps == 0 || max_steps >= SHK_MAX_STEP)
        return fail(nullptr, SHK_EINVAL, "shk_coalescence_times: max_steps must be in 1..2^31-1");
    std::vector<unsigned char> host;
    int max_L = 32;
    const int rc = build_pairs("shk_coalescence_times", dynamics, n_pairs, L, q, J, seed, lattice_id, host, &max_L);
    if (rc != SHK_OK) return rc;
    if (bytes < shk_coalescence_scratch_bytes(n_pairs))
        return fail(nullptr, SHK_ENOMEM, "shk_coalescence_times: %zu bytes given, %zu needed", bytes,
                    shk_coalescence_scratch_bytes(n_pairs));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* dev = static_cast<unsigned char*>(dev_scratch);
    const size_t off_T = pairs_bytes_aligned(n_pairs);
    cudaError_t e = cudaMemcpyAsync(dev, host.data(), host.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_coalesce(dynamics, dev, (uint32_t)n_pairs, max_L, max_steps,
                            reinterpret_cast<unsigned long long*>(dev + off_T), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_T, dev + off_T, (size_t)n_pairs * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "shk_coalescence_times");
    return SHK_OK;
}

size_t shk_cftp_scratch_bytes(int n_pairs) {
    if (n_pairs <= 0) return 0;
    return pairs_bytes_aligned(n_pairs) + (size_t)n_pairs * 4;
}

int shk_cftp(int dynamics, int n_pairs, const int* L, const double* q, const double* J, const uint64_t* seed,
             const uint32_t* lattice_id, int k_max, void* dev_samples, size_t sample_stride_bytes,
             void* dev_scratch, size_t bytes, int32_t* host_k, void* stream) {
    const TraceRange trace("shk_cftp");
    if (!dev_samples || !dev_scratch || !host_k) return fail(nullptr, SHK_EINVAL, "shk_cftp: bad argument");
    if (k_max < 0 || k_max > SHK_CFTP_MAX_K)
        return fail(nullptr, SHK_EINVAL, "shk_cftp: k_max=%d outside 0..%d", k_max, SHK_CFTP_MAX_K);
    std::vector<unsigned char> host;
    int max_L = 32;
    const int rc = build_pairs("shk_cftp", dynamics, n_pairs, L, q, J, seed, lattice_id, host, &max_L);
    if (rc != SHK_OK) return rc;
    if (sample_stride_bytes % 4 != 0 || sample_stride_bytes < (size_t)max_L * max_L / 8 ||
        sample_stride_bytes / 4 > 0xffffffffull)
        return fail(nullptr, SHK_EINVAL, "shk_cftp: sample stride %zu must be a multiple of 4 and >= %d",
                    sample_stride_bytes, max_L * max_L / 8);
    if ((reinterpret_cast<uintptr_t>(dev_samples) & 3u) != 0)
        return fail(nullptr, SHK_EINVAL, "shk_cftp: dev_samples must be 4-byte aligned");
    if (bytes < shk_cftp_scratch_bytes(n_pairs))
        return fail(nullptr, SHK_ENOMEM, "shk_cftp: %zu bytes given, %zu needed", bytes, shk_cftp_scratch_bytes(n_pairs));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* dev = static_cast<unsigned char*>(dev_scratch);
    const size_t off_k = pairs_bytes_aligned(n_pairs);
    cudaError_t e = cudaMemcpyAsync(dev, host.data(), host.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_cftp(dynamics, dev, (uint32_t)n_pairs, max_L, k_max, static_cast<uint32_t*>(dev_samples),
                        (uint32_t)(sample_stride_bytes / 4), reinterpret_cast<int*>(dev + off_k), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_k, dev + off_k, (size_t)n_pairs * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "shk_cftp");
    return SHK_OK;
}

int shk_init_plane(int layout, void* plane, int L, int kind, uint64_t init_seed,
                   uint32_t lattice_id, uint32_t plane_index, void* stream) {
    Geometry g;
    if (!make_geometry(L, layout, &g))
        return fail(nullptr, SHK_EINVAL, "shk_init_plane: invalid L=%d for layout %d", L, layout);
    if (plane == nullptr) return fail(nullptr, SHK_EINVAL, "shk_init_plane: plane is NULL");
    if (!aligned16(plane)) return fail(nullptr, SHK_EINVAL, "shk_init_plane: plane must be 16-byte aligned");
    if (kind != SHK_INIT_ALL_UP && kind != SHK_INIT_ALL_DOWN && kind != SHK_INIT_RANDOM)
        return fail(nullptr, SHK_EINVAL, "shk_init_plane: unknown kind %d", kind);
    const cudaError_t e = launch_init(g, plane, kind, init_seed, lattice_id, plane_index,
                                      static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "shk_init_plane launch");
    return SHK_OK;
}

size_t shk_lattice_bytes(int L, int layout) {
    Geometry g;
    if (!make_geometry(L, layout, &g)) return 0;
    return 2 * g.plane_bytes + kRingBytes;
}

int shk_lattice_create(int L, int layout, void* dev_mem, size_t bytes, void* stream,
                       shk_lattice** out) {
    if (out == nullptr) return fail(nullptr, SHK_EINVAL, "shk_lattice_create: out is NULL");
    *out = nullptr;
    Geometry g;
    if (!make_geometry(L, layout, &g))
        return fail(nullptr, SHK_EINVAL,
                    "shk_lattice_create: invalid L=%d for layout %d (2 <= L <= %d; bit-packed needs L %% 32 == 0)",
                    L, layout, SHK_MAX_L);
    if (dev_mem == nullptr || (reinterpret_cast<uintptr_t>(dev_mem) & 255u) != 0)
        return fail(nullptr, SHK_EINVAL, "shk_lattice_create: dev_mem must be non-NULL and 256-byte aligned");
    const size_t need = 2 * g.plane_bytes + kRingBytes;
    if (bytes < need)
        return fail(nullptr, SHK_ENOMEM, "shk_lattice_create: %zu bytes given, %zu needed", bytes, need);
    shk_lattice* lat = new (std::nothrow) shk_lattice();
    if (lat == nullptr) return fail(nullptr, SHK_ENOMEM, "shk_lattice_create: host allocation failed");
    lat->g = g;
    lat->dev = static_cast<unsigned char*>(dev_mem);
    lat->bytes = bytes;
    lat->plane[0] = lat->dev;
    lat->plane[1] = lat->dev + g.plane_bytes;
    lat->ring = reinterpret_cast<long long*>(lat->dev + 2 * g.plane_bytes);
    lat->stream = static_cast<cudaStream_t>(stream);
    *out = lat;
    return SHK_OK;
}

void shk_lattice_destroy(shk_lattice* lat) { delete lat; }

int shk_lattice_init(shk_lattice* lat, int kind, uint64_t init_seed) {
    if (lat == nullptr) return fail(nullptr, SHK_EINVAL, "shk_lattice_init: NULL handle");
    for (uint32_t p = 0; p < 2; ++p) {
        const int rc = shk_init_plane(lat->g.layout, lat->plane[p], lat->g.L, kind, init_seed,
                                      lat->lattice_id, p, lat->stream);
        if (rc != SHK_OK) return fail(lat, rc, "%s", g_thread_err.c_str());
    }
    lat->step = 0;
    lat->last_obs = nullptr;
    return SHK_OK;
}

int shk_set_params(shk_lattice* lat, double q, double J) {
    if (lat == nullptr) return fail(nullptr, SHK_EINVAL, "shk_set_params: NULL handle");
    uint32_t T[6];
    if (host_thresholds(q, J, T) != SHK_OK)
        return fail(lat, SHK_EINVAL, "shk_set_params: q=%g and J=%g must be finite", q, J);
    lat->q = q;
    lat->J = J;
    std::memcpy(lat->T, T, sizeof T);
    lat->params_set = true;
    return SHK_OK;
}

int shk_set_seed(shk_lattice* lat, uint64_t seed, uint32_t lattice_id) {
    if (lat == nullptr) return fail(nullptr, SHK_EINVAL, "shk_set_seed: NULL handle");
    lat->seed = seed;
    lat->lattice_id = lattice_id;
    return SHK_OK;
}

int shk_set_step(shk_lattice* lat, uint64_t step) {
    if (lat == nullptr) return fail(nullptr, SHK_EINVAL, "shk_set_step: NULL handle");
    if (step >= SHK_MAX_STEP) return fail(lat, SHK_EINVAL, "shk_set_step: step must be < 2^31");
    lat->step = step;
    return SHK_OK;
}

int shk_get_step(const shk_lattice* lat, uint64_t* step) {
    if (lat == nullptr || step == nullptr) return fail(nullptr, SHK_EINVAL, "shk_get_step: NULL argument");
    *step = lat->step;
    return SHK_OK;
}

int shk_run(shk_lattice* lat, uint64_t n_steps, int64_t* dev_obs) {
    const TraceRange trace("shk_run");
    if (lat == nullptr) return fail(nullptr, SHK_EINVAL, "shk_run: NULL handle");
    if (!lat->params_set) return fail(lat, SHK_ESTATE, "shk_run: call shk_set_params first");
    if (n_steps == 0) return SHK_OK;
    if (n_steps > SHK_MAX_STEP - lat->step)
        return fail(lat, SHK_EINVAL, "shk_run: step counter would exceed 2^31");
    DrawParams P;
    make_draw_params(lat->seed, lat->lattice_id, lat->T, 0u, &P);
    const Geometry& g = lat->g;
    cudaStream_t st = lat->stream;
    const uint64_t t0 = lat->step, t_last = t0 + n_steps - 1;
    long long* obs = reinterpret_cast<long long*>(dev_obs);
    cudaError_t e;
    if (small_path_fits(g) && n_steps <= 0xffffffffull) {
        e = launch_run_small(g, lat->plane[0], lat->plane[1], P, t0, n_steps, obs, lat->ring, st);
        if (e != cudaSuccess) return cuda_fail(lat, e, "shk_run (one-CTA path)");
        lat->last_obs = lat->ring;
    } else {
        auto slot = [&](uint64_t t) -> long long* {
            return obs ? obs + (size_t)kNumObs * (t - t0) : lat->ring + 8 * (t % 4);
        };
        e = obs ? cudaMemsetAsync(obs, 0, (size_t)kNumObs * sizeof(long long) * n_steps, st)
                : cudaMemsetAsync(slot(t0), 0, (size_t)kNumObs * sizeof(long long), st);
        if (e != cudaSuccess) return cuda_fail(lat, e, "shk_run memset");
        for (uint64_t t = t0; t <= t_last; ++t) {
            long long* zero = (obs == nullptr && t < t_last) ? slot(t + 1) : nullptr;
            e = launch_halfstep(g, 0, lat->plane[0], lat->plane[1], P, (uint32_t)(2 * t), slot(t),
                                t > t0 ? slot(t - 1) : nullptr, zero, st);
            if (e != cudaSuccess) return cuda_fail(lat, e, "shk_run half-step A");
            e = launch_halfstep(g, 1, lat->plane[1], lat->plane[0], P, (uint32_t)(2 * t + 1),
                                slot(t), nullptr, nullptr, st);
            if (e != cudaSuccess) return cuda_fail(lat, e, "shk_run half-step B");
        }
        e = launch_cnn(g, lat->plane[0], slot(t_last), st);
        if (e != cudaSuccess) return cuda_fail(lat, e, "shk_run C_nn pass");
        if (obs) {
            e = cudaMemcpyAsync(lat->ring, slot(t_last), kNumObs * sizeof(long long),
                                cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(lat, e, "shk_run copy of last row");
            lat->last_obs = lat->ring;
        } else {
            lat->last_obs = slot(t_last);
        }
    }
    lat->step += n_steps;
    return SHK_OK;
}

int shk_sweep_status(void* stream) {
    bool fault = false;
    const cudaError_t e = sweep_fault_take(static_cast<cudaStream_t>(stream), &fault);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "shk_sweep_status");
    if (fault)
        return fail(nullptr, SHK_ETIMEOUT,
                    "shk_sweep_status: a sweep's wait on its own row copies gave up; its output is incomplete");
    return SHK_OK;
}

int shk_bulk_wait_timeout_test(uint32_t limit_cycles, int* timed_out, void* stream) {
    if (timed_out == nullptr || limit_cycles == 0 || limit_cycles > (1u << 30))
        return fail(nullptr, SHK_EINVAL, "shk_bulk_wait_timeout_test: bad argument (limit_cycles in 1..2^30)");
    *timed_out = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    bool fault = false;
    cudaError_t e = sweep_fault_take(st, &fault);   // start from a clear word
    if (e == cudaSuccess) e = launch_bulk_wait_probe((long long)limit_cycles, st);
    if (e == cudaSuccess) e = sweep_fault_take(st, &fault);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "shk_bulk_wait_timeout_test");
    *timed_out = fault ? 1 : 0;
    return SHK_OK;
}

// After a synchronising read: SHK_ETIMEOUT if a sweep's bounded wait gave up.
static int sweep_fault_status(shk_lattice* lat) {
    bool fault = false;
    const cudaError_t e = sweep_fault_take(lat->stream, &fault);
    if (e != cudaSuccess) return cuda_fail(lat, e, "reading the sweep fault word");
    if (fault) return fail(lat, SHK_ETIMEOUT, "a sweep's wait on its own row copies gave up; the state is incomplete");
    return SHK_OK;
}

int shk_read_observables(shk_lattice* lat, int64_t host_out[SHK_NOBS]) {
    if (lat == nullptr || host_out == nullptr)
        return fail(lat, SHK_EINVAL, "shk_read_observables: NULL argument");
    if (lat->last_obs == nullptr) return fail(lat, SHK_ESTATE, "shk_read_observables: no step has run");
    cudaError_t e = cudaMemcpyAsync(host_out, lat->last_obs, kNumObs * sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) return cuda_fail(lat, e, "shk_read_observables");
    return sweep_fault_status(lat);
}

int shk_read_spins(shk_lattice* lat, int plane, int8_t* host_out) {
    if (lat == nullptr || host_out == nullptr || (plane != 0 && plane != 1))
        return fail(lat, SHK_EINVAL, "shk_read_spins: bad handle, plane or buffer");
    const Geometry& g = lat->g;
    cudaError_t e;
    if (g.layout == kInt8) {
        e = cudaMemcpyAsync(host_out, lat->plane[plane], (size_t)g.N, cudaMemcpyDeviceToHost, lat->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    } else {
        std::vector<uint32_t> words(g.nblocks);
        e = cudaMemcpyAsync(words.data(), lat->plane[plane], (size_t)g.nblocks * 4, cudaMemcpyDeviceToHost,
                            lat->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
        if (e == cudaSuccess)
            for (int64_t u = 0; u < g.N; ++u) host_out[u] = ((words[u >> 5] >> (u & 31)) & 1u) ? 1 : -1;
    }
    if (e != cudaSuccess) return cuda_fail(lat, e, "shk_read_spins");
    return sweep_fault_status(lat);
}

int shk_write_spins(shk_lattice* lat, int plane, const int8_t* host_in) {
    if (lat == nullptr || host_in == nullptr || (plane != 0 && plane != 1))
        return fail(lat, SHK_EINVAL, "shk_write_spins: bad handle, plane or buffer");
    const Geometry& g = lat->g;
    for (int64_t u = 0; u < g.N; ++u)
        if (host_in[u] != 1 && host_in[u] != -1)
            return fail(lat, SHK_EINVAL, "shk_write_spins: entry %lld is %d, not +1 or -1", (long long)u,
                        (int)host_in[u]);
    cudaError_t e;
    if (g.layout == kInt8) {
        e = cudaMemcpyAsync(lat->plane[plane], host_in, (size_t)g.N, cudaMemcpyHostToDevice, lat->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    } else {
        std::vector<uint32_t> words(g.nblocks, 0u);
        for (int64_t u = 0; u < g.N; ++u)
            if (host_in[u] > 0) words[u >> 5] |= 1u << (u & 31);
        e = cudaMemcpyAsync(lat->plane[plane], words.data(), (size_t)g.nblocks * 4, cudaMemcpyHostToDevice,
                            lat->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    }
    if (e != cudaSuccess) return cuda_fail(lat, e, "shk_write_spins");
    lat->last_obs = nullptr;
    return SHK_OK;
}

int shk_upload_plane(shk_lattice* lat, int plane, const void* host_raw, size_t bytes) {
    if (lat == nullptr || host_raw == nullptr || (plane != 0 && plane != 1))
        return fail(lat, SHK_EINVAL, "shk_upload_plane: bad handle, plane or buffer");
    const size_t n = lat->g.layout == kBitpack ? (size_t)lat->g.N / 8 : (size_t)lat->g.N;
    if (bytes < n) return fail(lat, SHK_ENOMEM, "shk_upload_plane: %zu bytes given, %zu needed", bytes, n);
    const cudaError_t e = cudaMemcpyAsync(lat->plane[plane], host_raw, n, cudaMemcpyHostToDevice, lat->stream);
    if (e != cudaSuccess) return cuda_fail(lat, e, "shk_upload_plane");
    lat->last_obs = nullptr;
    return SHK_OK;
}

int shk_download_plane(shk_lattice* lat, int plane, void* host_raw, size_t bytes) {
    if (lat == nullptr || host_raw == nullptr || (plane != 0 && plane != 1))
        return fail(lat, SHK_EINVAL, "shk_download_plane: bad handle, plane or buffer");
    const size_t n = lat->g.layout == kBitpack ? (size_t)lat->g.N / 8 : (size_t)lat->g.N;
    if (bytes < n) return fail(lat, SHK_ENOMEM, "shk_download_plane: %zu bytes given, %zu needed", bytes, n);
    const cudaError_t e = cudaMemcpyAsync(host_raw, lat->plane[plane], n, cudaMemcpyDeviceToHost, lat->stream);
    if (e != cudaSuccess) return cuda_fail(lat, e, "shk_download_plane");
    return SHK_OK;
}

void* shk_plane_ptr(shk_lattice* lat, int plane) {
    if (lat == nullptr || (plane != 0 && plane != 1)) return nullptr;
    return lat->plane[plane];
}

}  // extern "C"
