// fb_tc_tma.cuh -- the 3x3 convolutions of the learned NNF initialiser as tcgen05 GEMMs
// whose operands the Tensor Memory Accelerator stages: tc_conv_tma_kernel (forward, stride
// s = 1 or 2, one box per tap; with FLIP the stride-1 input gradient), described here;
// tc_conv_tma_rows_kernel (the same with the three row taps of a column sharing one halo
// box); tc_conv_tma_s2grad_kernel (the stride-2 input gradient by output parity);
// tc_wgrad_tma_kernel (the weight gradient, both operands MN-major).  Each is described
// above its definition.
//
//   Y[p][co] = sum_{tap, ci} X[s p + tap - (1, 1)][ci] W[co][tap][ci]    (M = output
//   pixels, N = Cout, K = 9 Cin, walked tap-major in chunks of K = 64)
//
// A CTA of 128 threads owns 128 output pixels -- whole output rows (R rows of one image,
// or I whole images when an image has fewer than 128 output pixels) -- by BN output
// channels.  The K axis is the tap-major sequence of CB-channel columns (CB = 64, 32, 16
// or 8, the widest that divides Cin), 64 / CB columns per chunk of K = 64.  For each
// chunk one elected thread issues tiled TMA loads into a stage of shared memory: per
// column the activation box {CB channels, s Wo, s R, I}, traversed with element stride s
// along the image axes and displaced by the column's tap (coordinates -1 and beyond the
// image are filled with zeros: the convolution's padding, no bounds arithmetic in the
// kernel), landing as 128 rows of 2 CB bytes in the K-major layout the tensor core reads
// (swizzled over 2 CB bytes, none for CB = 8); and the weight box {64 of the 9 Cin K
// elements, BN} in the 128-byte swizzle layout.  Completion is signalled by the stage's
// "full" mbarrier with the byte count; the same thread waits for it, issues the chunk's
// K = 16 MMAs into the TMEM accumulator and commits them to the stage's "empty" mbarrier,
// which gates the stage's next TMA loads S - 1 chunks later.  No channel beyond Cin is
// moved.  The epilogue reads TMEM with tcgen05.ld.  Every wait is bounded: on expiry the
// kernel records an error, waits (bounded) for its outstanding MMAs and copies, skips the
// epilogue and releases TMEM.
#pragma once

#include <cstdint>

#include <cuda.h>

#include "fb_tc_gemm.cuh"

namespace fb {
namespace tc {

// Shared-memory matrix descriptor of a K-major operand whose rows of RB = 32, 64 or 128
// bytes are swizzled over RB: start >> 4, stride between 8-row atoms (8 RB bytes) >> 4 at
// bit 32, descriptor version 1 at bit 46, layout type at bit 61 (6: 32-byte, 4: 64-byte,
// 2: 128-byte swizzle); the leading offset is unused for these layouts and set to 1.
// Stepping K by 16 elements inside a row advances the start by 32 bytes.
template <int RB>
__device__ __forceinline__ uint64_t smem_desc_sw(uint32_t saddr) {
    static_assert(RB == 32 || RB == 64 || RB == 128, "swizzle width");
    constexpr uint64_t layout = RB == 128 ? 2 : RB == 64 ? 4 : 6;
    return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (1ull << 16) |
           (static_cast<uint64_t>((8 * RB) >> 4) << 32) | (1ull << 46) | (layout << 61);
}
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) { return smem_desc_sw<128>(saddr); }

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

// FLIP = true mirrors every tap's displacement ((dy, dx) -> (2 - dy, 2 - dx)): the
// stride-1 input gradient dX[p][ci] = sum_{tap, co} dZ[p + (1, 1) - tap][co] WT[ci][tap][co]
// is this same GEMM over dZ with the transposed weights WT as the {9 Cout, Cin} matrix.
template <int BN, int S, int CB, class Epi, bool FLIP = false>
__global__ void __launch_bounds__(128)
    tc_conv_tma_kernel(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w,
                       Epi epi, TmaConvGeom g, int* status) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 128, "tile N");
    static_assert(S >= 2 && S <= 8, "stages");
    static_assert(CB == 8 || CB == 16 || CB == 32 || CB == 64, "column width");
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
    constexpr int RB = 2 * CB;            // bytes of one row of a column
    constexpr uint32_t COL = BM * RB;     // bytes of one column (128 rows)
    constexpr int PER = BK / CB;          // columns per chunk
    const int cpt = g.Cin / CB;           // columns per tap (Cin % CB == 0)
    const int ktot = 9 * g.Cin;
    const int n_chunks = (ktot + BK - 1) / BK;
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
        const long lim = progress_limit();
        auto issue = [&](int c) {
            const int s = c % S;
            const uint32_t sa = s0 + s * STAGE;
            const int nq = min(BK, ktot - BK * c) / CB;   // columns of this chunk
            const int nz = CB == 8 ? (nq & 1) : 0;        // zero column completing a K = 16 step
            mbar_expect_tx(&full[s], static_cast<uint32_t>((nq + nz) * COL + B_BYTES));
            for (int q = 0; q < nq; ++q) {
                const int col = PER * c + q, tap = col / cpt, blk = col - tap * cpt;
                const int dy = FLIP ? 2 - tap / 3 : tap / 3, dx = FLIP ? 2 - (tap - 3 * (tap / 3)) : tap - 3 * dy;
                tma_load_4d(sa + q * COL, &map_x, &full[s], CB * blk, dx - 1, g.stride * y0 + dy - 1, img0);
            }
            if (nz) tma_load_4d(sa + nq * COL, &map_x, &full[s], 0, 0, 0, g.n);  // wholly outside: zeros
            tma_load_2d(sa + A_BYTES, &map_w, &full[s], BK * c, n0);
            ++issued;
        };
        for (int c = 0; c < S - 1 && c < n_chunks; ++c) issue(c);
        int done = 0;     // chunks whose MMAs were committed
        for (int i = 0; i < n_chunks && ok; ++i) {
            const int s = i % S;
            ok = mbar_wait(&full[s], (i / S) & 1, lim);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = s0 + s * STAGE, sb = sa + A_BYTES;
            const int steps = (min(BK, ktot - BK * i) + 15) / 16;
            for (int j = 0; j < steps; ++j) {
                uint64_t da;
                if constexpr (CB == 8)   // two 16-byte columns per step, 128-byte core-matrix groups
                    da = smem_desc_plain(sa + 2u * COL * j, COL, 128u);
                else                     // the step's 32 bytes inside one swizzled row
                    da = smem_desc_sw<RB>(sa + (16u * j / CB) * COL + (32u * j) % RB);
                mma_bf16(tmem, da, smem_desc_sw128(sb + 32u * j), idesc, (i > 0 || j > 0) ? 1u : 0u);
            }
            mma_commit(&empty[s]);
            ++done;
            const int nxt = i + S - 1;
            if (nxt < n_chunks) {
                const int prev = nxt - S;   // the chunk that last used nxt's stage
                if (prev >= 0) ok = mbar_wait(&empty[prev % S], (prev / S) & 1, lim);
                if (ok) issue(nxt);
            }
        }
        if (ok && done > 0) ok = mbar_wait(&empty[(done - 1) % S], ((done - 1) / S) & 1, lim);
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

// ---------------------------------------------------------------------------------
// The same stride-1 convolution with the three row taps of a tap column sharing one halo
// box ("row reuse").  A tile is R whole output rows y0 .. y0 + R - 1 of one image; for a
// column displacement ex in {-1, 0, 1} and a CB-channel block the activation box
// {CB channels, Wo, R + 2, 1} at (x = ex, y = y0 - 1) holds input rows y0 - 1 .. y0 + R,
// and the row displacement ey in {-1, 0, 1} is the 128-row view starting (ey + 1) Wo rows
// into it: a whole number of 8-row swizzle atoms when Wo % 8 == 0, so the view is an
// ordinary K-major operand.  One stage per (ex, block): the box plus the three taps' weight
// boxes {CB of the 9 Cin K elements, BN}, then 3 CB / 16 MMAs.  The activation bytes per
// tile fall from 9 R Wo rows to 3 (R + 2) Wo rows per block; the products are the same,
// accumulated in (ex, block, ey) order instead of tap-major order.
// ---------------------------------------------------------------------------------
template <int BN, int S, int CB, class Epi, bool FLIP = false>
__global__ void __launch_bounds__(128)
    tc_conv_tma_rows_kernel(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w,
                            Epi epi, TmaConvGeom g, int* status) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 128, "tile N");
    static_assert(S >= 2 && S <= 4, "stages");
    static_assert(CB == 32 || CB == 64, "column width");
    constexpr int RB = 2 * CB;                      // bytes of one activation / weight row
    constexpr uint32_t WB = static_cast<uint32_t>(BN) * RB;   // one weight box
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ __align__(8) uint64_t empty[S];
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const uint32_t a_bytes = static_cast<uint32_t>(BM + 2 * g.Wo) * RB;   // R + 2 rows of Wo pixels
    const uint32_t stage = (a_bytes + 3 * WB + 1023u) & ~1023u;
    const int cpt = g.Cin / CB;                     // channel blocks (Cin % CB == 0)
    const int n_groups = 3 * cpt;
    const int img0 = m0 / (g.Ho * g.Wo);
    const int y0 = (m0 - img0 * g.Ho * g.Wo) / g.Wo;
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
        int issued = 0;
        const long lim = progress_limit();
        auto issue = [&](int gi) {
            const int s = gi % S;
            const uint32_t sa = s0 + s * stage;
            const int ex = gi / cpt - 1, blk = gi - (ex + 1) * cpt;
            mbar_expect_tx(&full[s], a_bytes + 3 * WB);
            tma_load_4d(sa, &map_x, &full[s], CB * blk, ex, y0 - 1, img0);
#pragma unroll
            for (int e = 0; e < 3; ++e) {   // row displacement ey = e - 1
                const int tap = FLIP ? (2 - e) * 3 + (1 - ex) : e * 3 + (ex + 1);
                tma_load_2d(sa + a_bytes + e * WB, &map_w, &full[s], tap * g.Cin + CB * blk, n0);
            }
            ++issued;
        };
        for (int c = 0; c < S - 1 && c < n_groups; ++c) issue(c);
        int done = 0;
        for (int i = 0; i < n_groups && ok; ++i) {
            const int s = i % S;
            ok = mbar_wait(&full[s], (i / S) & 1, lim);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = s0 + s * stage, sb = sa + a_bytes;
#pragma unroll
            for (int e = 0; e < 3; ++e)
#pragma unroll
                for (int j = 0; j < CB / 16; ++j)
                    mma_bf16(tmem, smem_desc_sw<RB>(sa + static_cast<uint32_t>(e * g.Wo) * RB + 32u * j),
                             smem_desc_sw<RB>(sb + e * WB + 32u * j), idesc, (i > 0 || e > 0 || j > 0) ? 1u : 0u);
            mma_commit(&empty[s]);
            ++done;
            const int nxt = i + S - 1;
            if (nxt < n_groups) {
                const int prev = nxt - S;
                if (prev >= 0) ok = mbar_wait(&empty[prev % S], (prev / S) & 1, lim);
                if (ok) issue(nxt);
            }
        }
        if (ok && done > 0) ok = mbar_wait(&empty[(done - 1) % S], ((done - 1) / S) & 1, lim);
        if (!ok) {
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

// ---------------------------------------------------------------------------------
// Input gradient of a stride-2 layer by output parity.  The forward reads input pixel
// (2 oy + ty - 1, 2 ox + tx - 1) for output (oy, ox) and tap (ty, tx), so an input row
// 2 m + py receives tap row ty = 1 from output row m (py = 0), or tap rows 0 and 2 from
// output rows m + 1 and m (py = 1); likewise for columns.  Each of the four parity classes
// (py, px) of dX is therefore a stride-1 convolution over the output gradient's grid with
// one, two or four taps at displacements 0 or +1 (past the far edge: the box's zero fill):
//   dX[2 m + py][2 m' + px][ci] = sum_{class taps, co} dZ[m + sy][m' + sx][co] WT[ci][tap][co].
// blockIdx.z is the class; a tile is 128 class pixels (the forward's whole-row tiles of the
// Ho x Wo grid); each K column is one (tap, CB-channel block): the box {CB, Wo, R, I} of dZ
// at (x = sx, y = y0 + sy) and the weight box {CB of the 9 C K elements, BN}; the epilogue
// stores row (img, 2 m + py, 2 m' + px) of dX.
// ---------------------------------------------------------------------------------
struct ParityClasses {
    int ntaps[4];
    int sx[4][4], sy[4][4], tap[4][4];   // per class and tap: displacements, weight tap index
};

template <int BN, int S, int CB, class Epi>
__global__ void __launch_bounds__(128)
    tc_conv_tma_s2grad_kernel(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_w,
                              Epi epi, TmaConvGeom g, ParityClasses pc, int* status) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 128, "tile N");
    static_assert(S >= 2 && S <= 4, "stages");
    static_assert(CB == 32 || CB == 64, "column width");
    constexpr int RB = 2 * CB;
    constexpr uint32_t A_BYTES = BM * RB;
    constexpr uint32_t WB = static_cast<uint32_t>(BN) * RB;
    constexpr uint32_t STAGE = (A_BYTES + WB + 1023u) & ~1023u;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ __align__(8) uint64_t empty[S];
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN, cls = blockIdx.z;
    const int py = cls >> 1, px = cls & 1;
    const int cpt = g.Cin / CB;                    // channel blocks of dZ (Cin % CB == 0)
    const int n_cols = pc.ntaps[cls] * cpt;
    const int img0 = m0 / (g.Ho * g.Wo);
    const int y0 = (m0 - img0 * g.Ho * g.Wo) / g.Wo;
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
        int issued = 0;
        const long lim = progress_limit();
        auto issue = [&](int q) {
            const int s = q % S;
            const uint32_t sa = s0 + s * STAGE;
            const int t = q / cpt, blk = q - t * cpt;
            mbar_expect_tx(&full[s], A_BYTES + WB);
            tma_load_4d(sa, &map_x, &full[s], CB * blk, pc.sx[cls][t], y0 + pc.sy[cls][t], img0);
            tma_load_2d(sa + A_BYTES, &map_w, &full[s], pc.tap[cls][t] * g.Cin + CB * blk, n0);
            ++issued;
        };
        for (int c = 0; c < S - 1 && c < n_cols; ++c) issue(c);
        int done = 0;
        for (int i = 0; i < n_cols && ok; ++i) {
            const int s = i % S;
            ok = mbar_wait(&full[s], (i / S) & 1, lim);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = s0 + s * STAGE;
#pragma unroll
            for (int j = 0; j < CB / 16; ++j)
                mma_bf16(tmem, smem_desc_sw<RB>(sa + 32u * j), smem_desc_sw<RB>(sa + A_BYTES + 32u * j), idesc,
                         (i > 0 || j > 0) ? 1u : 0u);
            mma_commit(&empty[s]);
            ++done;
            const int nxt = i + S - 1;
            if (nxt < n_cols) {
                const int prev = nxt - S;
                if (prev >= 0) ok = mbar_wait(&empty[prev % S], (prev / S) & 1, lim);
                if (ok) issue(nxt);
            }
        }
        if (ok && done > 0) ok = mbar_wait(&empty[(done - 1) % S], ((done - 1) / S) & 1, lim);
        if (!ok) {
            if (done > 0) mbar_wait(&empty[(done - 1) % S], ((done - 1) / S) & 1);
            for (int c = done; c < issued; ++c) mbar_wait(&full[c % S], (c / S) & 1);
            s_ok = 0;
            atomicExch(status, 1);
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (s_ok) {
        const int m = m0 + warp * 32 + lane;   // class pixel: (img, oy, ox) of the Ho x Wo grid
        const int img = m / (g.Ho * g.Wo), rem = m - img * g.Ho * g.Wo;
        const int oy = rem / g.Wo, ox = rem - oy * g.Wo;
        const int row = (img * (2 * g.Ho) + 2 * oy + py) * (2 * g.Wo) + 2 * ox + px;   // dX pixel
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
            if (m < g.M && n0 + c0 < g.Cout) epi.store(row, n0 + c0, v);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TmemCols<BN>::value));
}

// Bytes of one stage of the row-reuse kernel and the dynamic shared memory of S stages.
inline int conv_rows_stage_bytes(int BN, int CB, int Wo) {
    return ((BM + 2 * Wo) * 2 * CB + 3 * BN * 2 * CB + 1023) / 1024 * 1024;
}

// ---------------------------------------------------------------------------------
// Weight gradient of the 3x3 convolution, with both operands MN-major:
//
//   dW[co][tap][ci] = sum_p X[s p + tap - (1, 1)][ci] dZ[p][co]
//
// as the GEMM D[r][co] = sum_p A[r][p] B[co][p] with r = tap Cp + ci (M = 9 Cp rows,
// tap-major, Cp = Cin rounded up to 32), N = 32 NB >= Cout and K = the output pixels p.
// Neither operand is transposed: for a chunk of 128 consecutive output pixels (whole output
// rows, as in the forward) the activation box {32 channels, s Wo, s R, I} of one tap --
// displaced by the tap, zeros outside the image and past the last channel -- lands as 128
// rows of 64 bytes, pixel-major, i.e. K rows of 32 contiguous M elements: the MN-major
// layout in the 64-byte swizzle (8 K rows x 64 bytes per atom, atoms along K 512 bytes
// apart).  A 128-row M tile is four such boxes (32-channel blocks of one or two taps), 8 KB
// apart; the output gradient's box {32 channels, 128 pixels} of the [P][Cout] matrix (zeros
// past Cout) is the same layout for B, NB boxes.  Rows of padding channels and columns past
// Cout are computed as zeros and not stored.  Per chunk the elected thread issues eight K = 16 MMAs (start + 1 KB each) into
// the 128 x Cout fp32 accumulator.  CTAs split the pixel axis (grid.y); each stores its
// partial sums to its own slice part[blockIdx.y] (laid out like dW), and a separate
// reduction adds the slices in split order, so the sum does not depend on which CTA ends
// first.
// Waits, drains and the timeout report are those of the forward kernel.
// ---------------------------------------------------------------------------------

// Shared-memory matrix descriptor of an MN-major operand in the 64-byte swizzle layout:
// atoms of 8 K rows x 64 bytes (32 MN elements); lbo bytes between atoms adjacent along
// MN, sbo bytes between atoms adjacent along K; version 1 at bit 46, layout type 4.
__device__ __forceinline__ uint64_t smem_desc_mn_sw64(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (4ull << 61);
}

// Instruction descriptor of kind::f16 with both operands MN-major (bits 15 and 16).
__host__ __device__ constexpr uint32_t instr_desc_mn(int n) { return instr_desc(n) | (1u << 15) | (1u << 16); }

struct TmaWgradGeom {
    int Cin, Cp;     // input channels, and rounded up to 32
    int Cout;        // output channels (<= 32 NB)
    int rows;        // 9 Cin: columns of dW
    int HoWo, Wo;    // output pixels per image, output width
    int stride;
    int chunks;      // pixel chunks of 128 (the last may run past the last image: zeros)
    int per_split;   // chunks per CTA along grid.y
};

constexpr int kWgradChunk = 128 * 64;          // bytes of one 32-wide box of 128 K rows
constexpr int kWgradSlack = 8 * 1024;          // dynamic shared memory past the last stage

template <int NB, int S>
__host__ __device__ constexpr int wgrad_tma_smem_bytes() {
    return S * (4 + NB) * kWgradChunk + 1024 + kWgradSlack;
}

template <int NB, int S>
__global__ void __launch_bounds__(128)
    tc_wgrad_tma_kernel(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_dz,
                        float* __restrict__ part, TmaWgradGeom g, int* status) {
    static_assert(NB >= 1 && NB <= 4, "Cout = 32 NB");
    static_assert(S >= 2 && S <= 6, "stages");
    static_assert(wgrad_tma_smem_bytes<NB, S>() <= 227 * 1024 - 1024, "shared memory per CTA");
    constexpr int BN = 32 * NB;
    constexpr int A_BYTES = 4 * kWgradChunk;
    constexpr int STAGE = A_BYTES + NB * kWgradChunk;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[S];
    __shared__ __align__(8) uint64_t empty[S];
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM;
    const int c_begin = blockIdx.y * g.per_split;
    const int c_end = min(g.chunks, c_begin + g.per_split);
    if (c_begin >= c_end) return;                      // uniform over the CTA
    const int n_local = c_end - c_begin;
    const int na = min(4, (9 * g.Cp - m0) / 32);       // 32-row blocks of this M tile
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
    constexpr uint32_t idesc = instr_desc_mn(BN);

    if (threadIdx.x == 0) {
        bool ok = true;
        int issued = 0;   // local chunks whose loads were issued
        const long lim = progress_limit();
        auto issue = [&](int i) {
            const int s = i % S;
            const uint32_t sa = s0 + s * STAGE;
            const int p0 = 128 * (c_begin + i);
            const int img0 = p0 / g.HoWo;
            const int y0 = (p0 - img0 * g.HoWo) / g.Wo;
            mbar_expect_tx(&full[s], static_cast<uint32_t>((na + NB) * kWgradChunk));
            for (int q = 0; q < na; ++q) {
                const int r0 = m0 + 32 * q, tap = r0 / g.Cp, ci0 = r0 - tap * g.Cp;
                const int dy = tap / 3, dx = tap - 3 * dy;
                tma_load_4d(sa + q * kWgradChunk, &map_x, &full[s], ci0, dx - 1, g.stride * y0 + dy - 1, img0);
            }
#pragma unroll
            for (int b = 0; b < NB; ++b)
                tma_load_2d(sa + A_BYTES + b * kWgradChunk, &map_dz, &full[s], 32 * b, p0);
            ++issued;
        };
        for (int i = 0; i < S - 1 && i < n_local; ++i) issue(i);
        int done = 0;     // local chunks whose MMAs were committed
        for (int i = 0; i < n_local && ok; ++i) {
            const int s = i % S;
            ok = mbar_wait(&full[s], (i / S) & 1, lim);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = s0 + s * STAGE, sb = sa + A_BYTES;
#pragma unroll
            for (int j = 0; j < 8; ++j)   // K rows 16 j .. 16 j + 15: two atoms along K
                mma_bf16(tmem, smem_desc_mn_sw64(sa + 1024u * j, kWgradChunk, 512u),
                         smem_desc_mn_sw64(sb + 1024u * j, kWgradChunk, 512u), idesc, (i > 0 || j > 0) ? 1u : 0u);
            mma_commit(&empty[s]);
            ++done;
            const int nxt = i + S - 1;
            if (nxt < n_local) {
                const int prev = nxt - S;   // the chunk that last used nxt's stage
                if (prev >= 0) ok = mbar_wait(&empty[prev % S], (prev / S) & 1, lim);
                if (ok) issue(nxt);
            }
        }
        if (ok && done > 0) ok = mbar_wait(&empty[(done - 1) % S], ((done - 1) / S) & 1, lim);
        if (!ok) {
            if (done > 0) mbar_wait(&empty[(done - 1) % S], ((done - 1) / S) & 1);
            for (int c = done; c < issued; ++c) mbar_wait(&full[c % S], (c / S) & 1);
            s_ok = 0;
            atomicExch(status, 1);
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (s_ok) {
        const int rp = m0 + warp * 32 + lane, tap = rp / g.Cp, ci = rp - tap * g.Cp;
        const bool real = rp < 9 * g.Cp && ci < g.Cin;   // not a padding channel
        const int row = tap * g.Cin + ci;                 // column of dW
        float* slice = part + static_cast<size_t>(blockIdx.y) * g.Cout * g.rows;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
            if (real) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (c0 + j < g.Cout) slice[static_cast<size_t>(c0 + j) * g.rows + row] = v[j];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TmemCols<BN>::value));
}

}  // namespace tc
}  // namespace fb
