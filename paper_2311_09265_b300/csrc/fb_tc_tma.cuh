// fb_tc_tma.cuh -- the forward 3x3 convolution (stride s = 1 or 2) of the learned NNF
// initialiser as a tcgen05 GEMM whose operands the Tensor Memory Accelerator stages:
//
//   Y[p][co] = sum_{tap, ci} X[s p + tap - (1, 1)][ci] W[co][tap][ci]    (M = output
//   pixels, N = Cout, K = 9 Cin, walked tap-major in blocks of 64 input channels)
//
// A CTA of 128 threads owns 128 output pixels -- whole output rows (R rows of one image,
// or I whole images when an image has fewer than 128 output pixels) -- by BN output
// channels.  For K chunk (tap, channel block) one elected thread issues two tiled TMA
// loads into a stage of shared memory: the activation box {64 channels, s Wo, s R, I}
// traversed with element stride s along the image axes and displaced by the tap
// (coordinates -1 and beyond the image are filled with zeros: the convolution's padding,
// no bounds arithmetic in the kernel), which lands as the 128 x 64 A tile, and the
// weight box {64 channels, 1 tap, BN}.  Both land in the 128-byte-swizzled K-major
// layout the tensor core reads (128-byte rows, 8-row atoms 1024 bytes apart), signalled
// by the stage's "full" mbarrier with the byte count; the same thread waits for it,
// issues the chunk's K = 16 MMAs into the TMEM accumulator and commits them to the
// stage's "empty" mbarrier, which gates the stage's next TMA load S - 1 chunks later.
// The epilogue reads TMEM with tcgen05.ld.  Every wait is bounded: on expiry the kernel
// records an error, waits (bounded) for its outstanding copies, skips the epilogue and
// releases TMEM.
#pragma once

#include <cstdint>

#include <cuda.h>

#include "fb_tc_gemm.cuh"

namespace fb {
namespace tc {

// Shared-memory matrix descriptor of a K-major operand in the 128-byte swizzle layout:
// start >> 4, stride between 8-row atoms (1024 bytes) >> 4 at bit 32, descriptor version
// 1 at bit 46, layout type 2 (128-byte swizzle) at bit 61; the leading offset is unused
// for this layout and set to 1.  Stepping K by 16 elements advances the start by 32
// bytes inside the swizzle atom.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (1ull << 16) |
           (static_cast<uint64_t>(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// ... and of a K-major operand in the no-swizzle layout: 8-row x 16-byte core matrices,
// lbo bytes between core matrices adjacent in K, sbo bytes between those adjacent in M/N.
__device__ __forceinline__ uint64_t smem_desc_plain(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
        "%5, %6}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, "
        "%5}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

// Geometry of the TMA convolution: output Ho x Wo; a tile is R output rows of one image
// (I = 1) or I whole images (R = Ho).
struct TmaConvGeom {
    int Ho, Wo, Cin;  // output size, input channels
    int Cout;
    int M;            // n * Ho * Wo output pixels
    int R, I;         // output rows and images per 128-pixel tile
    int stride;
    int n;            // images
};

// Two operand arrangements.  Wide (Cin >= 64): K chunk = (tap, 64-channel block), one
// activation box of 64 channels landing in the 128-byte swizzle layout; the weights as a
// {Cin, 9, Cout} tensor.  Packed (Cin < 64): the K axis is the tap-major sequence of
// 8-channel columns, eight per chunk; each column is one activation box of 8 channels
// landing as 128 rows x 16 bytes (the no-swizzle layout: core matrices 128 bytes apart
// along M, columns 2048 bytes apart along K), so no channels beyond Cin are moved; a
// column that only pads the chunk's last K = 16 step is a box lying wholly outside the
// tensor (zeros); the weights as a {9 Cin, Cout} matrix in the 128-byte swizzle layout.

template <int BN, int S, bool PACKED, class Epi>
__global__ void __launch_bounds__(128)
    tc_conv_tma_kernel(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w,
                       Epi epi, TmaConvGeom g, int* status) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 128, "tile N");
    static_assert(S >= 2 && S <= 8, "stages");
    constexpr int A_BYTES = BM * BK * 2;   // 16 KB: 128 rows of 128 bytes
    constexpr int B_BYTES = BN * BK * 2;   // BN rows of 128 bytes (multiple of 1 KB for BN % 8 == 0)
    constexpr int STAGE = A_BYTES + B_BYTES;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ __align__(8) uint64_t empty[S];
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int ncb = (g.Cin + BK - 1) / BK;
    const int cpt = g.Cin / 8;            // packed: 8-channel columns per tap
    const int ncols = 9 * cpt;
    const int n_chunks = PACKED ? (ncols + 7) / 8 : 9 * ncb;
    constexpr uint32_t COL = BM * 16;     // packed: bytes of one 8-channel column
    const int img0 = m0 / (g.Ho * g.Wo);
    const int y0 = (m0 - img0 * g.Ho * g.Wo) / g.Wo;
    // 1024-byte alignment of every stage (the swizzle atoms) inside the dynamic buffer
    const uint32_t s0 = (smem_u32(smem) + 1023u) & ~1023u;

    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s]);
            mbar_init(&empty[s]);
        }
        s_ok = 1;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TmemCols<BN>::value));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = instr_desc(BN);

    if (threadIdx.x == 0) {
        bool ok = true;
        int issued = 0;   // chunks whose loads were issued
        auto issue = [&](int c) {
            const int s = c % S;
            const uint32_t sa = s0 + s * STAGE;
            if constexpr (PACKED) {
                const int nq = min(8, ncols - 8 * c), nz = nq & 1;
                mbar_expect_tx(&full[s], static_cast<uint32_t>((nq + nz) * COL + B_BYTES));
                for (int q = 0; q < nq; ++q) {
                    const int col = 8 * c + q, tap = col / cpt, ch8 = col - tap * cpt;
                    const int dy = tap / 3, dx = tap - 3 * dy;
                    tma_load_4d(sa + q * COL, &map_x, &full[s], 8 * ch8, dx - 1, g.stride * y0 + dy - 1, img0);
                }
                if (nz) tma_load_4d(sa + nq * COL, &map_x, &full[s], 0, 0, 0, g.n);  // all outside: zeros
                tma_load_2d(sa + A_BYTES, &map_w, &full[s], BK * c, n0);
            } else {
                const int tap = c / ncb, cb = c - tap * ncb;
                const int dy = tap / 3, dx = tap - 3 * dy;
                mbar_expect_tx(&full[s], static_cast<uint32_t>(STAGE));
                tma_load_4d(sa, &map_x, &full[s], BK * cb, dx - 1, g.stride * y0 + dy - 1, img0);
                tma_load_3d(sa + A_BYTES, &map_w, &full[s], BK * cb, tap, n0);
            }
            ++issued;
        };
        for (int c = 0; c < S - 1 && c < n_chunks; ++c) issue(c);
        int done = 0;     // chunks whose MMAs were committed
        for (int i = 0; i < n_chunks && ok; ++i) {
            const int s = i % S;
            ok = mbar_wait(&full[s], (i / S) & 1);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = s0 + s * STAGE, sb = sa + A_BYTES;
            if constexpr (PACKED) {
                const int steps = (min(8, ncols - 8 * i) + 1) / 2;
                for (int j = 0; j < steps; ++j)
                    mma_bf16(tmem, smem_desc_plain(sa + 2u * COL * j, COL, 128u), smem_desc_sw128(sb + 32u * j),
                             idesc, (i > 0 || j > 0) ? 1u : 0u);
            } else {
                const int steps = (min(BK, g.Cin - BK * (i % ncb)) + 15) / 16;
                for (int j = 0; j < steps; ++j)
                    mma_bf16(tmem, smem_desc_sw128(sa + 32u * j), smem_desc_sw128(sb + 32u * j), idesc,
                             (i > 0 || j > 0) ? 1u : 0u);
            }
            mma_commit(&empty[s]);
            ++done;
            const int nxt = i + S - 1;
            if (nxt < n_chunks) {
                const int prev = nxt - S;   // the chunk that last used nxt's stage
                if (prev >= 0) ok = mbar_wait(&empty[prev % S], (prev / S) & 1);
                if (ok) issue(nxt);
            }
        }
        if (ok && done > 0) ok = mbar_wait(&empty[(done - 1) % S], ((done - 1) / S) & 1);
        if (!ok) {
            // Let the MMAs already committed finish and the copies already issued land
            // before TMEM and the CTA's shared memory go away (each wait bounded).
            if (done > 0) mbar_wait(&empty[(done - 1) % S], ((done - 1) / S) & 1);
            for (int c = done; c < issued; ++c) mbar_wait(&full[c % S], (c / S) & 1);
            s_ok = 0;
            atomicExch(status, 1);
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (s_ok) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
            if (row < g.M && n0 + c0 < g.Cout) epi.store(row, n0 + c0, v);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TmemCols<BN>::value));
}

// Dynamic shared memory: S stages plus up to 1 KB to align the first to 1024 bytes.
template <int BN, int S>
constexpr int conv_tma_smem_bytes() {
    return S * (BM * BK * 2 + BN * BK * 2) + 1024;
}

}  // namespace tc
}  // namespace fb
