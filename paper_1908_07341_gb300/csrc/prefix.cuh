// prefix.cuh -- device-side Philox round prefixes, for kernels whose
// half-step index changes inside a launch (the host computes them for the
// per-launch sweeps; the fields are documented with PhiloxPrefix in
// device.cuh).
#pragma once

#include "device.cuh"

namespace shk {

// The warp-uniform Philox prefix of call c in half-step hs (device side of
// the host's philox_prefix: the uniform words of rounds 1 to 3).
__device__ __forceinline__ PhiloxPrefix philox_prefix_dev(const DrawParams& P, uint32_t hs, int c) {
    const uint32_t p0lo = kPhiloxM0 * hs, p0hi = __umulhi(kPhiloxM0, hs);
    const uint32_t p1lo = kPhiloxM1 * P.lattice_id, p1hi = __umulhi(kPhiloxM1, P.lattice_id);
    const uint32_t c2 = p0hi ^ (P.c3_base + (uint32_t)c) ^ P.rk1[0];
    const uint32_t q1lo = kPhiloxM1 * c2, q1hi = __umulhi(kPhiloxM1, c2);
    const uint32_t B = q1hi ^ p1lo ^ P.rk0[1];
    PhiloxPrefix u;
    u.A = p1hi ^ P.rk0[0];
    u.K2 = p0lo ^ P.rk1[1];
    u.K3 = q1lo ^ P.rk0[2];
    u.H3 = __umulhi(kPhiloxM0, B) ^ P.rk1[2];
    u.D = kPhiloxM0 * B;
    return u;
}

// The 8 prefixes of half-step hs into pre[] (threads 0..7 of the CTA; the
// caller synchronises before use).
__device__ __forceinline__ void fill_prefixes(PhiloxPrefix* pre, const DrawParams& P, uint32_t hs) {
    if (threadIdx.x < 8) pre[threadIdx.x] = philox_prefix_dev(P, hs, (int)threadIdx.x);
}

}  // namespace shk
