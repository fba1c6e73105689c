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

// The instruction sequences the patch-match kernels evaluate Eq. 1 with, on register
// operands.  k = 5 (paired rows): per candidate two 8-word slots and one 4-word half slot
// (the five 15-byte patch rows, zero padded), each word with three dp4a (<s, t>, |s|^2,
// |t|^2), each slot closed by acc += |s|^2 + |t|^2 - 2 <s, t> and the early-exit compare
// against the incumbent's error.  k = 7: seven 6-word rows, three dp4a per word likewise,
// each row closed the same way.  The compare is never taken
// here (the bound is the kernel argument); dp4a is issued through volatile asm so that no
// product is hoisted or folded: every candidate pays the whole sequence, as in the
// kernels.  3k^2 byte pairs of Eq. 1 per candidate.
__device__ __forceinline__ uint32_t dp4a_kept(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

template <int K>
__global__ void __launch_bounds__(256) ssd_mix_probe_kernel(uint32_t seed, uint32_t bound, int iters,
                                                            uint32_t* __restrict__ sink) {
    constexpr int NWORDS = K == 5 ? 20 : 42;
    uint32_t t[NWORDS], s[NWORDS];
#pragma unroll
    for (int w = 0; w < NWORDS; ++w) {
        t[w] = (seed * static_cast<uint32_t>(w + 1)) ^ (threadIdx.x * 0x9E3779B9u) ^ blockIdx.x;
        s[w] = t[w] + 0x01010101u * static_cast<uint32_t>(w & 3);
    }
    uint32_t total = 0;
    for (int i = 0; i < iters; ++i) {
        uint32_t acc = 0;
        if constexpr (K == 5) {
#pragma unroll
            for (int slot = 0; slot < 3; ++slot) {
                const int w0 = 8 * slot, nw = slot < 2 ? 8 : 4;
                uint32_t dot = 0, ss = 0, te = 0;
#pragma unroll
                for (int w = 0; w < nw; ++w) {
                    dot = dp4a_kept(s[w0 + w], t[w0 + w], dot);
                    ss = dp4a_kept(s[w0 + w], s[w0 + w], ss);
                    te = dp4a_kept(t[w0 + w], t[w0 + w], te);
                }
                acc += ss + te - 2u * dot;
                if (acc >= bound) break;
            }
        } else {
#pragma unroll
            for (int a = 0; a < 7; ++a) {
                uint32_t dot = 0, ss = 0, te = 0;
#pragma unroll
                for (int w = 0; w < 6; ++w) {
                    dot = dp4a_kept(s[6 * a + w], t[6 * a + w], dot);
                    ss = dp4a_kept(s[6 * a + w], s[6 * a + w], ss);
                    te = dp4a_kept(t[6 * a + w], t[6 * a + w], te);
                }
                acc += ss + te - 2u * dot;
                if (acc >= bound) break;
            }
        }
        total += acc;
    }
    if (total == 0x12345678u) sink[blockIdx.x] = total;  // practically never taken; defeats DCE
}


// Scattered 32-byte loads, the L1 traffic of the patch-match kernels: per round every
// thread issues four independent 256-bit loads of pseudo-randomly chosen 32-byte slots of
// a buffer of mask + 1 slots (indices masked into it), so the loads' latency overlaps and
// the rate of the L1 data pipe (or, for buffers beyond L1, of L2) is what is measured.
__global__ void __launch_bounds__(256) gather_probe_kernel(const uint32_t* __restrict__ buf, uint32_t mask,
                                                           int iters, uint32_t* __restrict__ sink) {
    uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
    uint32_t acc = 0;
    for (int i = 0; i < iters; ++i) {
        uint32_t w[4][8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            x = x * 1664525u + 1013904223u;
            const uint32_t* p = buf + static_cast<size_t>((x >> 7) & mask) * 8;
            asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(w[q][0]), "=r"(w[q][1]), "=r"(w[q][2]), "=r"(w[q][3]), "=r"(w[q][4]),
                           "=r"(w[q][5]), "=r"(w[q][6]), "=r"(w[q][7])
                         : "l"(p));
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) acc ^= w[q][0] ^ w[q][3] ^ w[q][7];
    }
    if (acc == 0x12345678u) sink[blockIdx.x] = acc;  // practically never taken; keeps the loads
}
}  // namespace

cudaError_t launch_ssd_mix_probe(int k, int blocks, int iters, uint32_t* sink, cudaStream_t st) {
    if (k == 5)
        ssd_mix_probe_kernel<5><<<blocks, 256, 0, st>>>(0xC0FFEEu, 0xFFFFFFFFu, iters, sink);
    else if (k == 7)
        ssd_mix_probe_kernel<7><<<blocks, 256, 0, st>>>(0xC0FFEEu, 0xFFFFFFFFu, iters, sink);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_dp4a_probe(int blocks, int iters, uint32_t* sink, cudaStream_t st) {
    dp4a_probe_kernel<<<blocks, 256, 0, st>>>(0xC0FFEEu, iters, sink);
    return cudaGetLastError();
}

cudaError_t launch_gather_probe(const uint32_t* buf, uint32_t slots, int blocks, int iters, uint32_t* sink,
                                cudaStream_t st) {
    if (slots == 0 || (slots & (slots - 1)) != 0) return cudaErrorInvalidValue;
    gather_probe_kernel<<<blocks, 256, 0, st>>>(buf, slots - 1, iters, sink);
    return cudaGetLastError();
}

}  // namespace fb
