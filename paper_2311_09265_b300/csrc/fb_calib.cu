// fb_calib.cu -- register-only throughput probe of the integer dot-product
// instruction (dp4a) that carries Eq. 1, used as the ALU roofline denominator of the
// patch-match kernels.  Not part of the method.
#include "fb_internal.h"

namespace fb {
namespace {

constexpr int kChains = kDp4aProbeChains;  // independent accumulators per thread

__global__ void __launch_bounds__(256) dp4a_probe_kernel(uint32_t seed, int iters,
                                                         uint32_t* __restrict__ sink) {
    uint32_t a = seed ^ (threadIdx.x * 0x9E3779B9u), b = seed + blockIdx.x;
    uint32_t acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = a + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = __dp4a(a, b + c, acc[c]);
        a = a * 1664525u + 1013904223u;  // fresh operand each round; chains stay independent
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) r ^= acc[c];
    if (r == 0x12345678u) sink[blockIdx.x] = r;  // practically never taken; defeats DCE
}

}  // namespace

cudaError_t launch_dp4a_probe(int blocks, int iters, uint32_t* sink, cudaStream_t st) {
    dp4a_probe_kernel<<<blocks, 256, 0, st>>>(0xC0FFEEu, iters, sink);
    return cudaGetLastError();
}

}  // namespace fb
