// noalloc.cu -- an entry point that runs the shaken chain without allocating.
//
// Some callers cannot call cudaMalloc.  Examples are a host application that
// owns every byte of device memory through its own pool and forbids outside
// allocations, and a latency-critical loop in which cudaMalloc's implicit
// device synchronisation is not acceptable.  Such a caller passes only the
// sigma plane (input and output) and an optional 5-entry result buffer.  The
// transient tau plane and the per-step observable accumulators live in the
// file-scope array below.  Every GPU that loads the library reserves this
// array until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  The accumulators are cleared at the start of each call.  The tau
// part needs no clearing: half-step A overwrites all of it before anything
// reads it.  Two calls whose work overlaps on the GPU (on different streams,
// or from different host threads) race on the array and give wrong results.
//
// The call compiles and loads nothing either: a half-step runs the sweep
// specialised for its threshold table only when an earlier call of the
// library has already loaded that kernel on this device (loading a module
// allocates device memory), and the generic sweep otherwise.  Both compute
// the same spins and sums.
#include "shaken.h"
#include "internal.h"

namespace {

// Scratch: [observable ring: 4 slots x 8 int64 = 256 B][tau plane, <= 8 MiB].
constexpr size_t kRingBytes = 256;
constexpr size_t kTauBytes = SHK_STATIC_SCRATCH_PLANE_BYTES;

static __device__ __align__(256) unsigned char g_static_scratch[kRingBytes + kTauBytes];

int fail(int code, const char* msg) {
    shk::set_thread_error(msg);
    return code;
}

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in, so the address comes from cudaGetSymbolAddress,
// with the device current.  It is looked up on every call (cheap next to the
// launches), so an address never outlives the context it belongs to.
cudaError_t scratch_address(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" int shk_shaken_run_static(int layout, void* sigma, int L, double q, double J,
                                     uint64_t seed, uint32_t lattice_id, uint64_t t0,
                                     uint64_t n_steps, int64_t* last_obs, void* stream) {
    using namespace shk;
    Geometry g;
    if (!make_geometry(L, layout, &g))
        return fail(SHK_EINVAL, "shk_shaken_run_static: invalid L or layout");
    if (g.plane_bytes > kTauBytes)
        return fail(SHK_EINVAL,
                    "shk_shaken_run_static: lattice too large for the static scratch "
                    "(at most 8 MiB per plane: bit-packed L <= 8192, int8 L <= 2896)");
    if (sigma == nullptr) return fail(SHK_EINVAL, "shk_shaken_run_static: sigma is NULL");
    if (!aligned16(sigma) || (last_obs != nullptr && !aligned8(last_obs)))
        return fail(SHK_EINVAL,
                    "shk_shaken_run_static: sigma must be 16-byte aligned and last_obs 8-byte aligned");
    if (t0 > SHK_MAX_STEP || n_steps > SHK_MAX_STEP - t0)
        return fail(SHK_EINVAL, "shk_shaken_run_static: step index would exceed 2^31");
    uint32_t T[6];
    if (host_thresholds(q, J, T) != SHK_OK)
        return fail(SHK_EINVAL, "shk_shaken_run_static: q and J must be finite");
    if (n_steps == 0) return SHK_OK;
    DrawParams P;
    make_draw_params(seed, lattice_id, T, 0u, &P);

    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return fail(SHK_ECUDA, cudaGetErrorString(e));
    long long* ring = static_cast<long long*>(base);
    void* tau = static_cast<unsigned char*>(base) + kRingBytes;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto slot = [&](uint64_t t) { return ring + 8 * (t % 4); };

    const uint64_t t_last = t0 + n_steps - 1;
    e = cudaMemsetAsync(slot(t0), 0, kNumObs * sizeof(long long), st);
    for (uint64_t t = t0; e == cudaSuccess && t <= t_last; ++t) {
        e = launch_halfstep(g, 0, sigma, tau, P, (uint32_t)(2 * t), slot(t),
                            t > t0 ? slot(t - 1) : nullptr, t < t_last ? slot(t + 1) : nullptr, st,
                            /*loaded_only=*/true);
        if (e == cudaSuccess)
            e = launch_halfstep(g, 1, tau, sigma, P, (uint32_t)(2 * t + 1), slot(t), nullptr,
                                nullptr, st, /*loaded_only=*/true);
    }
    if (e == cudaSuccess) e = launch_cnn(g, sigma, slot(t_last), st);
    if (e == cudaSuccess && last_obs != nullptr)
        e = cudaMemcpyAsync(last_obs, slot(t_last), kNumObs * sizeof(long long),
                            cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(SHK_ECUDA, cudaGetErrorString(e));
    return SHK_OK;
}
