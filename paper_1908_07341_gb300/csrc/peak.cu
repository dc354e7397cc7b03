// peak.cu -- measured ceiling of the arithmetic that bounds the bit-packed
// half-step: the library's own Philox4x32-10 with no memory traffic.
//
// Every thread runs `iters` calls on distinct counters (the same counter
// layout and round keys as the half-steps) and folds the outputs with XOR;
// one atomic XOR per warp keeps the result live.  Independent iterations
// give the scheduler all the instruction-level parallelism it can use, so
// calls / second of this kernel is the rate no draw can exceed.
#include <cstdint>

#include "shaken.h"
#include "internal.h"
#include "device.cuh"

namespace shk {

__global__ void __launch_bounds__(256) k_philox_peak(const DrawParams P, uint32_t iters, uint32_t* out) {
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
#pragma unroll 2
    for (uint32_t i = 0; i < iters; ++i) {
        uint32_t x0 = i, x1 = w, x2 = P.lattice_id, x3 = P.c3_base;
        philox10(x0, x1, x2, x3, P);
        acc ^= x0 ^ x1 ^ x2 ^ x3;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicXor(out, acc);
}

}  // namespace shk

using namespace shk;

extern "C" int shk_philox_peak(int blocks, uint32_t iters, uint32_t* dev_out, void* stream) {
    if (blocks <= 0 || iters == 0 || dev_out == nullptr) {
        set_thread_error("shk_philox_peak: blocks and iters must be positive and dev_out non-NULL");
        return SHK_EINVAL;
    }
    const uint32_t T[6] = {0x40000000u, 0x60000000u, 0x70000000u, 0x90000000u, 0xA0000000u, 0xC0000000u};
    DrawParams P;
    make_draw_params(0x0123456789ABCDEFull, 0u, T, 0u, &P);
    k_philox_peak<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(P, iters, dev_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_thread_error(cudaGetErrorString(e));
        return SHK_ECUDA;
    }
    return SHK_OK;
}
