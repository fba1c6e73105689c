// fb_net.cu -- the learned NNF initialiser: a small BF16 convolutional pyramid that
// maps a pair of guide frames to an offset field, used to start Alg. 1 close to its
// answer so that fewer iterations are needed.  The paper's method is model-free; this
// network is an addition that the method itself trains (targets are NNFs computed by
// Alg. 1).  Convolutions run on tcgen05 (fb_net_ops.cuh); training (forward, loss,
// backward, Adam) runs entirely in this file's kernels.
//
// Network, at a quarter of the guide resolution (Hq = H/4, Wq = W/4), NHWC bf16:
//   in    8 ch: source RGB, target RGB (each 4x4 box mean / 255 - 0.5), 2 zero ch
//   e0a 8->32, e0b 32->32            (Hq)
//   e1a 32->64 /2, e1b 64->64        (Hq/2)
//   e2a 64->96 /2, e2b 96->96        (Hq/4)
//   e3a 96->128 /2, e3b 128->128     (Hq/8)
//   d2  [up(e3b), e2b] 224->96       (Hq/4)
//   d1  [up(d2), e1b] 160->64        (Hq/2)
//   d0  [up(d1), e0b] 96->32         (Hq)
//   head 32->8 (channels 0,1 used): offset = 16 * head, in full-resolution pixels
// 3x3 kernels, zero padding, ReLU after every layer but the head; 779,592 parameters.
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "fb.h"
#include "fb_internal.h"
#include "fb_net_ops.cuh"
#include "fb_tc_tma.cuh"

namespace fb {
namespace net {
namespace {

constexpr int kOffsetScale = 16;

// ---------------------------------------------------------------------------------
// Conv launchers
// ---------------------------------------------------------------------------------
// K chunks per split and the number of splits the gathered GEMM runs for a requested
// split count: every split gets at least one chunk.
int gemm_per_split(int K, int splits) {
    const int chunks = (K + tc::BK - 1) / tc::BK;
    if (splits < 1) splits = 1;
    if (splits > chunks) splits = chunks;
    return (chunks + splits - 1) / splits;
}
int gemm_splits(int K, int splits) {
    const int chunks = (K + tc::BK - 1) / tc::BK, per = gemm_per_split(K, splits);
    return (chunks + per - 1) / per;
}

template <int BN, class G, class E>
cudaError_t launch_gemm(const G& gth, const E& epi, int M, int N, int K, int splits, int* status,
                        cudaStream_t st) {
    const int per = gemm_per_split(K, splits);
    splits = gemm_splits(K, splits);
    const dim3 grid((M + tc::BM - 1) / tc::BM, (N + BN - 1) / BN, splits);
    constexpr int smem = tc::gemm_smem_bytes<BN>();
    auto kern = tc::tc_gemm_kernel<BN, G, E>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 128, smem, st>>>(gth, epi, M, N, K, per, status);
    return cudaGetLastError();
}

#ifndef FB_GEMM_STAGES
#define FB_GEMM_STAGES 3
#endif
#ifndef FB_GEMM_LOOKAHEAD
#define FB_GEMM_LOOKAHEAD (FB_GEMM_STAGES - 1)
#endif
constexpr int kStages = FB_GEMM_STAGES;
constexpr int kLookahead = FB_GEMM_LOOKAHEAD;

// Forward and input-gradient convolutions: the pipelined asynchronous-copy GEMM.
template <int BN, class G, class E>
cudaError_t launch_gemm_async(const G& gth, const E& epi, int M, int N, int K, int* status,
                              cudaStream_t st) {
    const dim3 grid((M + tc::BM - 1) / tc::BM, (N + BN - 1) / BN);
    constexpr int smem = tc::gemm_async_smem_bytes<BN, kStages>();
    auto kern = tc::tc_gemm_async_kernel<BN, kStages, G, E, kLookahead>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, 128, smem, st>>>(gth, epi, M, N, K, status);
    return cudaGetLastError();
}

// ---- TMA-staged forward convolution (stride 1) ---------------------------------------
#ifndef FB_TMA_STAGES
#define FB_TMA_STAGES 3
#endif
constexpr int kTmaStages = FB_TMA_STAGES;
std::atomic<int> g_gemm_path{0};  // 0: TMA where eligible, row reuse where eligible; 1: gathers only;
                                  // 2: TMA without row reuse
std::atomic<unsigned long long> g_tma_launches{0};

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// The TMA path needs whole output rows per 128-pixel tile: Wo divides 128 and either an
// image holds a multiple of 128 output pixels (R = 128 / Wo rows) or 128 is a multiple
// of the image (I images of R = Ho rows); 16-byte aligned tensors and strides
// (Cin % 8 == 0); the strided box s Wo within the TMA limit of 256.  Output channels
// beyond 128 take further tiles along grid.y (the input gradients of the concatenated
// decoder layers: 160 and 224 channels).
bool tma_conv_geom(const ConvGeom& g, const void* X, const void* Wt, tc::TmaConvGeom& t) {
    if ((g.stride != 1 && g.stride != 2) || g.Cin % 8 || g.Wo < 1 || 128 % g.Wo) return false;
    if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Wt)) & 15) return false;
    const int px = g.Ho * g.Wo;
    int R, I;
    if (px >= 128) {
        if (px % 128) return false;
        R = 128 / g.Wo;
        I = 1;
    } else {
        if (128 % px) return false;
        R = g.Ho;
        I = 128 / px;
    }
    if (g.stride * g.Wo > 256 || g.stride * R > 256) return false;
    t = tc::TmaConvGeom{g.Ho, g.Wo, g.Cin, g.Cout, g.n * px, R, I, g.stride, g.n};
    return true;
}

template <int BN, class Epi = EpiFwd, bool FLIP = false>
cudaError_t launch_conv_tma(const ConvGeom& g, const tc::TmaConvGeom& t, const bf16* X, const bf16* Wt,
                            const Epi& epi, int* status, cudaStream_t st, bool* used) {
    *used = false;
    const auto encode = tensor_map_encoder();
    if (!encode) return cudaSuccess;
    alignas(64) CUtensorMap mx, mw;
    // column width: the widest of 64, 32, 16, 8 channels dividing Cin
    const int cb = g.Cin % 64 == 0 ? 64 : g.Cin % 32 == 0 ? 32 : g.Cin % 16 == 0 ? 16 : 8;
    const CUtensorMapSwizzle sw = cb == 64   ? CU_TENSOR_MAP_SWIZZLE_128B
                                  : cb == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                  : cb == 16 ? CU_TENSOR_MAP_SWIZZLE_32B
                                             : CU_TENSOR_MAP_SWIZZLE_NONE;
    const cuuint64_t xdim[4] = {static_cast<cuuint64_t>(g.Cin), static_cast<cuuint64_t>(g.W),
                                static_cast<cuuint64_t>(g.H), static_cast<cuuint64_t>(g.n)};
    const cuuint64_t xstr[3] = {static_cast<cuuint64_t>(g.Cin) * 2, static_cast<cuuint64_t>(g.W) * g.Cin * 2,
                                static_cast<cuuint64_t>(g.H) * g.W * g.Cin * 2};
    const cuuint32_t xbox[4] = {static_cast<cuuint32_t>(cb), static_cast<cuuint32_t>(g.stride * g.Wo),
                                static_cast<cuuint32_t>(g.stride * t.R), static_cast<cuuint32_t>(t.I)};
    const cuuint32_t xstep[4] = {1, static_cast<cuuint32_t>(g.stride), static_cast<cuuint32_t>(g.stride), 1};
    const cuuint32_t ones[2] = {1, 1};
    const CUresult rx = encode(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(X), xdim, xstr, xbox,
                               xstep, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    // weights as the {9 Cin, Cout} matrix (K = tap-major channels)
    const cuuint64_t wdim[2] = {static_cast<cuuint64_t>(9) * g.Cin, static_cast<cuuint64_t>(g.Cout)};
    const cuuint64_t wstr[1] = {static_cast<cuuint64_t>(9) * g.Cin * 2};
    const cuuint32_t wbox[2] = {static_cast<cuuint32_t>(tc::BK), static_cast<cuuint32_t>(BN)};
    const CUresult rw = encode(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(Wt), wdim, wstr, wbox,
                               ones, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rx != CUDA_SUCCESS || rw != CUDA_SUCCESS)
        return cudaSuccess;  // not expressible as tensor maps: the gather path runs instead
    constexpr int smem = tc::conv_tma_smem_bytes<BN, kTmaStages>();
    auto kern = cb == 64   ? tc::tc_conv_tma_kernel<BN, kTmaStages, 64, Epi, FLIP>
                : cb == 32 ? tc::tc_conv_tma_kernel<BN, kTmaStages, 32, Epi, FLIP>
                : cb == 16 ? tc::tc_conv_tma_kernel<BN, kTmaStages, 16, Epi, FLIP>
                           : tc::tc_conv_tma_kernel<BN, kTmaStages, 8, Epi, FLIP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((t.M + tc::BM - 1) / tc::BM, (g.Cout + BN - 1) / BN);
    kern<<<grid, 128, smem, st>>>(mx, mw, epi, t, status);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        *used = true;
        ++g_tma_launches;
    }
    return e;
}

// The row-reuse form of the TMA convolution (tc_conv_tma_rows_kernel): stride 1, tiles of
// R whole rows of one image (I == 1), Wo a multiple of 8 (the row views start on swizzle
// atoms), Cin a multiple of 32 (channel blocks of 32).  Padding 8-channel inputs to
// 32-wide blocks with the boxes' zero fill was measured and is slower (the 8 -> 32 input
// layer 86 -> ~250 us): the per-column kernel moves 8-channel columns as they are.
bool tma_rows_geom(const ConvGeom& g, const tc::TmaConvGeom& t) {
    return g.stride == 1 && t.I == 1 && g.Wo % 8 == 0 && g.Cin % 32 == 0 && t.R + 2 <= 256 && g.Wo <= 256;
}

template <int BN, class Epi, bool FLIP>
cudaError_t launch_conv_tma_rows(const ConvGeom& g, const tc::TmaConvGeom& t, const bf16* X, const bf16* Wt,
                                 const Epi& epi, int* status, cudaStream_t st, bool* used) {
    *used = false;
    const auto encode = tensor_map_encoder();
    if (!encode) return cudaSuccess;
    // 32-channel blocks even when Cin % 64 == 0: 64-channel ones double the stage, which cost
    // two of three CTAs per SM (the 64-channel 32x32 layer: 78 us against 56 per tap).
    constexpr int cb = 32;
    const CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_64B;
    alignas(64) CUtensorMap mx, mw;
    const cuuint64_t xdim[4] = {static_cast<cuuint64_t>(g.Cin), static_cast<cuuint64_t>(g.W),
                                static_cast<cuuint64_t>(g.H), static_cast<cuuint64_t>(g.n)};
    const cuuint64_t xstr[3] = {static_cast<cuuint64_t>(g.Cin) * 2, static_cast<cuuint64_t>(g.W) * g.Cin * 2,
                                static_cast<cuuint64_t>(g.H) * g.W * g.Cin * 2};
    const cuuint32_t xbox[4] = {static_cast<cuuint32_t>(cb), static_cast<cuuint32_t>(g.Wo),
                                static_cast<cuuint32_t>(t.R + 2), 1u};
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    const CUresult rx = encode(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(X), xdim, xstr, xbox,
                               ones, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    // weights as the {9 Cin, Cout} matrix; one box per tap and channel block
    const cuuint64_t wdim[2] = {static_cast<cuuint64_t>(9) * g.Cin, static_cast<cuuint64_t>(g.Cout)};
    const cuuint64_t wstr[1] = {static_cast<cuuint64_t>(9) * g.Cin * 2};
    const cuuint32_t wbox[2] = {static_cast<cuuint32_t>(cb), static_cast<cuuint32_t>(BN)};
    const CUresult rw = encode(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(Wt), wdim, wstr, wbox,
                               ones, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rx != CUDA_SUCCESS || rw != CUDA_SUCCESS) return cudaSuccess;
    // Three stages or none: with two the row reuse lost to the per-column kernel (the
    // 160-channel input gradient of the 32x32 decoder layer: 202 against 180 us).
#ifndef FB_ROWS_STAGES
#define FB_ROWS_STAGES 3
#endif
    constexpr int S = FB_ROWS_STAGES;
    const int stage = tc::conv_rows_stage_bytes(BN, cb, g.Wo);
    if (3 * stage + 1024 > 200 * 1024) return cudaSuccess;   // the column kernel runs instead
    const int smem = S * stage + 1024;
    auto kern = tc::tc_conv_tma_rows_kernel<BN, S, cb, Epi, FLIP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((t.M + tc::BM - 1) / tc::BM, (g.Cout + BN - 1) / BN);
    kern<<<grid, 128, smem, st>>>(mx, mw, epi, t, status);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        *used = true;
        ++g_tma_launches;
    }
    return e;
}

// TMA-fed convolution of output-channel tile BN: the row-reuse kernel where its geometry
// holds (path 0), else the per-column kernel.
template <int BN, class Epi, bool FLIP>
cudaError_t launch_conv_any(const ConvGeom& g, const tc::TmaConvGeom& t, const bf16* X, const bf16* Wt,
                            const Epi& epi, int* status, cudaStream_t st, bool* used) {
    if (g_gemm_path.load() == 0 && tma_rows_geom(g, t)) {
        cudaError_t e = launch_conv_tma_rows<BN, Epi, FLIP>(g, t, X, Wt, epi, status, st, used);
        if (e != cudaSuccess || *used) return e;
    }
    return launch_conv_tma<BN, Epi, FLIP>(g, t, X, Wt, epi, status, st, used);
}

cudaError_t conv_forward(const ConvGeom& g, const bf16* X, const bf16* Wt, const float* bias,
                         int relu, bf16* Y, float* Yf, int* status, cudaStream_t st) {
    const int M = g.n * g.Ho * g.Wo, K = 9 * g.Cin, ncb = (g.Cin + 63) / 64;
    EpiFwd epi{Y, Yf, bias, g.Cout, relu};
    tc::TmaConvGeom t;
    if (g_gemm_path.load() != 1 && tma_conv_geom(g, X, Wt, t)) {
        bool used = false;
        cudaError_t e = g.Cout <= 16   ? launch_conv_any<16, EpiFwd, false>(g, t, X, Wt, epi, status, st, &used)
                        : g.Cout <= 32 ? launch_conv_any<32, EpiFwd, false>(g, t, X, Wt, epi, status, st, &used)
                        : g.Cout <= 64 ? launch_conv_any<64, EpiFwd, false>(g, t, X, Wt, epi, status, st, &used)
                        : g.Cout == 96 ? launch_conv_any<96, EpiFwd, false>(g, t, X, Wt, epi, status, st, &used)
                                       : launch_conv_any<128, EpiFwd, false>(g, t, X, Wt, epi, status, st, &used);
        if (e != cudaSuccess || used) return e;
    }
    if (g.Cout <= 16) return launch_gemm_async<16>(GatherFwd<16>{X, Wt, g, M, K, ncb}, epi, M, g.Cout, K, status, st);
    if (g.Cout <= 32) return launch_gemm_async<32>(GatherFwd<32>{X, Wt, g, M, K, ncb}, epi, M, g.Cout, K, status, st);
    if (g.Cout <= 64) return launch_gemm_async<64>(GatherFwd<64>{X, Wt, g, M, K, ncb}, epi, M, g.Cout, K, status, st);
    return launch_gemm_async<128>(GatherFwd<128>{X, Wt, g, M, K, ncb}, epi, M, g.Cout, K, status, st);
}

// Input gradient of a stride-2 layer by output parity (tc_conv_tma_s2grad_kernel): gz is
// the output gradient's grid as a stride-1 geometry (Cin = the layer's Cout, the GEMM's K
// channels; Cout = the layer's Cin, its N), t its whole-row tiles.
template <int BN, class Epi>
cudaError_t launch_conv_tma_s2grad(const ConvGeom& gz, const tc::TmaConvGeom& t, const bf16* dZ,
                                   const bf16* WT, const Epi& epi, int* status, cudaStream_t st, bool* used) {
    *used = false;
    const auto encode = tensor_map_encoder();
    if (!encode) return cudaSuccess;
    const int cb = gz.Cin % 64 == 0 ? 64 : 32;
    const CUtensorMapSwizzle sw = cb == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    alignas(64) CUtensorMap mx, mw;
    const cuuint64_t xdim[4] = {static_cast<cuuint64_t>(gz.Cin), static_cast<cuuint64_t>(gz.W),
                                static_cast<cuuint64_t>(gz.H), static_cast<cuuint64_t>(gz.n)};
    const cuuint64_t xstr[3] = {static_cast<cuuint64_t>(gz.Cin) * 2, static_cast<cuuint64_t>(gz.W) * gz.Cin * 2,
                                static_cast<cuuint64_t>(gz.H) * gz.W * gz.Cin * 2};
    const cuuint32_t xbox[4] = {static_cast<cuuint32_t>(cb), static_cast<cuuint32_t>(gz.Wo),
                                static_cast<cuuint32_t>(t.R), static_cast<cuuint32_t>(t.I)};
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    const CUresult rx = encode(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(dZ), xdim, xstr, xbox,
                               ones, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    const cuuint64_t wdim[2] = {static_cast<cuuint64_t>(9) * gz.Cin, static_cast<cuuint64_t>(gz.Cout)};
    const cuuint64_t wstr[1] = {static_cast<cuuint64_t>(9) * gz.Cin * 2};
    const cuuint32_t wbox[2] = {static_cast<cuuint32_t>(cb), static_cast<cuuint32_t>(BN)};
    const CUresult rw = encode(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(WT), wdim, wstr, wbox,
                               ones, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rx != CUDA_SUCCESS || rw != CUDA_SUCCESS) return cudaSuccess;
    // tap row options per parity: (tap row, displacement) -- py = 0: (1, 0); py = 1: (0, +1), (2, 0)
    tc::ParityClasses pc{};
    for (int cls = 0; cls < 4; ++cls) {
        const int py = cls >> 1, px = cls & 1;
        const int ny = py ? 2 : 1, nx = px ? 2 : 1;
        int k = 0;
        for (int a = 0; a < ny; ++a)
            for (int b = 0; b < nx; ++b) {
                const int ty = py ? (a == 0 ? 0 : 2) : 1, sy = py && a == 0 ? 1 : 0;
                const int tx = px ? (b == 0 ? 0 : 2) : 1, sx = px && b == 0 ? 1 : 0;
                pc.tap[cls][k] = ty * 3 + tx;
                pc.sy[cls][k] = sy;
                pc.sx[cls][k] = sx;
                ++k;
            }
        pc.ntaps[cls] = k;
    }
    constexpr int S = 3;
    const int stage = (tc::BM * 2 * cb + BN * 2 * cb + 1023) / 1024 * 1024;
    const int smem = S * stage + 1024;
    auto kern = cb == 64 ? tc::tc_conv_tma_s2grad_kernel<BN, S, 64, Epi> : tc::tc_conv_tma_s2grad_kernel<BN, S, 32, Epi>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((t.M + tc::BM - 1) / tc::BM, (gz.Cout + BN - 1) / BN, 4);
    kern<<<grid, 128, smem, st>>>(mx, mw, epi, t, pc, status);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        *used = true;
        ++g_tma_launches;
    }
    return e;
}

template <class Epi>
cudaError_t conv_dgrad_epi(const ConvGeom& g, const bf16* dZ, const bf16* WT, const Epi& epi, int* status,
                           cudaStream_t st) {
    // Stride 2 with an even input: by output parity, from TMA-staged boxes of dZ.
    if (g.stride == 2 && g_gemm_path.load() != 1 && g.H == 2 * g.Ho && g.W == 2 * g.Wo && g.Cout % 32 == 0) {
        const ConvGeom gz{g.n, g.Ho, g.Wo, g.Cout, g.Ho, g.Wo, g.Cin, 1};
        tc::TmaConvGeom t;
        if (tma_conv_geom(gz, dZ, WT, t)) {
            bool used = false;
            cudaError_t e = gz.Cout <= 16   ? launch_conv_tma_s2grad<16, Epi>(gz, t, dZ, WT, epi, status, st, &used)
                            : gz.Cout <= 32 ? launch_conv_tma_s2grad<32, Epi>(gz, t, dZ, WT, epi, status, st, &used)
                            : gz.Cout <= 64 ? launch_conv_tma_s2grad<64, Epi>(gz, t, dZ, WT, epi, status, st, &used)
                            : gz.Cout == 96 ? launch_conv_tma_s2grad<96, Epi>(gz, t, dZ, WT, epi, status, st, &used)
                                            : launch_conv_tma_s2grad<128, Epi>(gz, t, dZ, WT, epi, status, st, &used);
            if (e != cudaSuccess || used) return e;
        }
    }
    const int M = g.n * g.H * g.W, K = 9 * g.Cout, ncb = (g.Cout + 63) / 64;
    // Stride 1: the input gradient is the 3x3 convolution of dZ with the tap-mirrored
    // transposed weights, staged by TMA like the forward layers (FLIP), where the boxes tile.
    tc::TmaConvGeom t;
    const ConvGeom gd{g.n, g.Ho, g.Wo, g.Cout, g.H, g.W, g.Cin, 1};
    if (g.stride == 1 && g_gemm_path.load() != 1 && tma_conv_geom(gd, dZ, WT, t)) {
        bool used = false;
        cudaError_t e = gd.Cout <= 16   ? launch_conv_any<16, Epi, true>(gd, t, dZ, WT, epi, status, st, &used)
                        : gd.Cout <= 32 ? launch_conv_any<32, Epi, true>(gd, t, dZ, WT, epi, status, st, &used)
                        : gd.Cout <= 64 ? launch_conv_any<64, Epi, true>(gd, t, dZ, WT, epi, status, st, &used)
                        : gd.Cout == 96 ? launch_conv_any<96, Epi, true>(gd, t, dZ, WT, epi, status, st, &used)
                                        : launch_conv_any<128, Epi, true>(gd, t, dZ, WT, epi, status, st, &used);
        if (e != cudaSuccess || used) return e;
    }
    if (g.Cin <= 16) return launch_gemm_async<16>(GatherDgrad<16>{dZ, WT, g, M, K, ncb}, epi, M, g.Cin, K, status, st);
    if (g.Cin <= 32) return launch_gemm_async<32>(GatherDgrad<32>{dZ, WT, g, M, K, ncb}, epi, M, g.Cin, K, status, st);
    if (g.Cin <= 64) return launch_gemm_async<64>(GatherDgrad<64>{dZ, WT, g, M, K, ncb}, epi, M, g.Cin, K, status, st);
    return launch_gemm_async<128>(GatherDgrad<128>{dZ, WT, g, M, K, ncb}, epi, M, g.Cin, K, status, st);
}

cudaError_t conv_dgrad(const ConvGeom& g, const bf16* dZ, const bf16* WT, float* dX, int accumulate,
                       int* status, cudaStream_t st) {
    return conv_dgrad_epi(g, dZ, WT, EpiDgrad{dX, g.Cin, accumulate}, status, st);
}

// The TMA-fed weight gradient (tc_wgrad_tma_kernel): both operands MN-major in 32-channel
// boxes (channel counts padded to 32 by the boxes' zero fill; Cin and Cout multiples of 8
// for 16-byte strides, Cout <= 128); the pixel chunks are the forward's 128-pixel tiles of
// whole output rows or whole images.
bool tma_wgrad_geom(const ConvGeom& g, const void* X, const void* dZ, int* R, int* I) {
    if ((g.stride != 1 && g.stride != 2) || g.Cin % 8 || g.Cout % 8 || g.Cout > 128 || g.Wo < 1 || 128 % g.Wo)
        return false;
    if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(dZ)) & 15) return false;
    const int px = g.Ho * g.Wo;
    if (px >= 128) {
        if (px % 128) return false;
        *R = 128 / g.Wo;
        *I = 1;
    } else {
        if (128 % px) return false;
        *R = g.Ho;
        *I = 128 / px;
    }
    return g.stride * g.Wo <= 256 && g.stride * *R <= 256;
}

#ifndef FB_WGRAD_STAGES1
#define FB_WGRAD_STAGES1 2
#endif
#ifndef FB_WGRAD_STAGES2
#define FB_WGRAD_STAGES2 4
#endif
template <int NB>
constexpr int wgrad_stages() { return NB == 1 ? FB_WGRAD_STAGES1 : NB == 2 ? FB_WGRAD_STAGES2 : 3; }  // 40-64 KB stages
template <int NB>
constexpr int wgrad_per_sm() { return (228 * 1024) / (tc::wgrad_tma_smem_bytes<NB, wgrad_stages<NB>()>() + 2048); }

// Pixel splits of the TMA-fed weight gradient: at most one wave of the CTAs that fit on the
// SMs at once, every split at least one chunk of 128 pixels.
int wgrad_tma_splits_max(const ConvGeom& g, int nb, int sms) {
    const int per_sm = nb == 1 ? wgrad_per_sm<1>() : nb == 2 ? wgrad_per_sm<2>()
                     : nb == 3 ? wgrad_per_sm<3>() : wgrad_per_sm<4>();
    const int mt = (9 * ((g.Cin + 31) / 32 * 32) + tc::BM - 1) / tc::BM;
    return per_sm * sms / mt > 0 ? per_sm * sms / mt : 1;
}

// Split count the gathered weight gradient asks for: two CTAs per SM over its N tiles.
int wgrad_gather_splits(const ConvGeom& g, int sms) {
    const int ntiles = (9 * g.Cin + 127) / 128;
    return (2 * sms + ntiles - 1) / ntiles;
}

template <int NB>
cudaError_t launch_wgrad_tma(const ConvGeom& g, int R, int I, const bf16* dZ, const bf16* X, float* part, int sms,
                             int* status, cudaStream_t st, bool* used, int* splits_out) {
    constexpr int S = wgrad_stages<NB>();
    *used = false;
    const auto encode = tensor_map_encoder();
    if (!encode) return cudaSuccess;
    alignas(64) CUtensorMap mx, mz;
    const cuuint64_t xdim[4] = {static_cast<cuuint64_t>(g.Cin), static_cast<cuuint64_t>(g.W),
                                static_cast<cuuint64_t>(g.H), static_cast<cuuint64_t>(g.n)};
    const cuuint64_t xstr[3] = {static_cast<cuuint64_t>(g.Cin) * 2, static_cast<cuuint64_t>(g.W) * g.Cin * 2,
                                static_cast<cuuint64_t>(g.H) * g.W * g.Cin * 2};
    const cuuint32_t xbox[4] = {32u, static_cast<cuuint32_t>(g.stride * g.Wo), static_cast<cuuint32_t>(g.stride * R),
                                static_cast<cuuint32_t>(I)};
    const cuuint32_t xstep[4] = {1, static_cast<cuuint32_t>(g.stride), static_cast<cuuint32_t>(g.stride), 1};
    const CUresult rx = encode(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(X), xdim, xstr, xbox,
                               xstep, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    const long long P = static_cast<long long>(g.n) * g.Ho * g.Wo;
    const cuuint64_t zdim[2] = {static_cast<cuuint64_t>(g.Cout), static_cast<cuuint64_t>(P)};
    const cuuint64_t zstr[1] = {static_cast<cuuint64_t>(g.Cout) * 2};
    const cuuint32_t zbox[2] = {32u, 128u};
    const cuuint32_t ones[2] = {1, 1};
    const CUresult rz = encode(&mz, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(dZ), zdim, zstr, zbox,
                               ones, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rx != CUDA_SUCCESS || rz != CUDA_SUCCESS) return cudaSuccess;  // the gathered kernel runs instead
    tc::TmaWgradGeom t{};
    t.Cin = g.Cin;
    t.Cp = (g.Cin + 31) / 32 * 32;
    t.Cout = g.Cout;
    t.rows = 9 * g.Cin;
    t.HoWo = g.Ho * g.Wo;
    t.Wo = g.Wo;
    t.stride = g.stride;
    t.chunks = static_cast<int>((P + 127) / 128);
    const int mt = (9 * t.Cp + tc::BM - 1) / tc::BM;
    const int splits_max = wgrad_tma_splits_max(g, NB, sms);
    t.per_split = (t.chunks + splits_max - 1) / splits_max;
    const int splits = (t.chunks + t.per_split - 1) / t.per_split;
    constexpr int smem = tc::wgrad_tma_smem_bytes<NB, S>();
    auto kern = tc::tc_wgrad_tma_kernel<NB, S>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(mt, splits), 128, smem, st>>>(mx, mz, part, t, status);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        *used = true;
        *splits_out = splits;
        ++g_tma_launches;
    }
    return e;
}

// Floats of the per-split slices conv_wgrad may write for geometry g (either path).
size_t wgrad_part_floats(const ConvGeom& g, int sms) {
    const int tma = wgrad_tma_splits_max(g, (g.Cout + 31) / 32, sms), gth = wgrad_gather_splits(g, sms);
    return static_cast<size_t>(tma > gth ? tma : gth) * g.Cout * 9 * g.Cin;
}

// Weight gradient of one layer as per-split partial sums: slice s of part (floats
// [Cout][9 Cin], at least wgrad_part_floats(g, sms) in all) holds split s's sum, *splits
// receives the split count; split_sum_kernel adds the slices.
cudaError_t conv_wgrad(const ConvGeom& g, const bf16* dZ, const bf16* X, float* part, int sms,
                       int* status, cudaStream_t st, int* splits) {
    int R = 0, I = 0;
    if (g_gemm_path.load() != 1 && tma_wgrad_geom(g, X, dZ, &R, &I)) {
        bool used = false;
        const int nb = (g.Cout + 31) / 32;
        cudaError_t e = nb == 1   ? launch_wgrad_tma<1>(g, R, I, dZ, X, part, sms, status, st, &used, splits)
                        : nb == 2 ? launch_wgrad_tma<2>(g, R, I, dZ, X, part, sms, status, st, &used, splits)
                        : nb == 3 ? launch_wgrad_tma<3>(g, R, I, dZ, X, part, sms, status, st, &used, splits)
                                  : launch_wgrad_tma<4>(g, R, I, dZ, X, part, sms, status, st, &used, splits);
        if (e != cudaSuccess || used) return e;
    }
    const int P = g.n * g.Ho * g.Wo, N = 9 * g.Cin;
    const int want = wgrad_gather_splits(g, sms);
    *splits = gemm_splits(P, want);
    return launch_gemm<128>(GatherWgrad<128>{dZ, X, g, P}, EpiWgrad{part, N, static_cast<size_t>(g.Cout) * N},
                            g.Cout, N, P, want, status, st);
}

// One sum of per-split slices: out[i] = (out[i] +) sum over s < splits of part[s n + i]
// (n a multiple of 4, 16-byte aligned arrays).  A block covers v4 quads of outputs with
// groups x v4 threads (groups a power of two, groups x v4 <= 512).
struct SplitSum {
    const float* part;
    int splits, n;
    float* out;
    int v4, groups;
};

// Blocks [0, blocks_a) reduce a, the rest b.  Thread (g, v) adds the slices s = g, g +
// groups, ... of output quad v in increasing s; the groups' sums are then added by a fixed
// pairwise tree.  A fixed order: the result is the same on every run.
__global__ void __launch_bounds__(512) split_sum_kernel(SplitSum a, SplitSum b, int blocks_a, int accumulate) {
    __shared__ float4 red[512];
    const bool first = static_cast<int>(blockIdx.x) < blocks_a;
    const SplitSum t = first ? a : b;
    const int blk = first ? blockIdx.x : blockIdx.x - blocks_a;
    const int v = static_cast<int>(threadIdx.x) % t.v4, g = static_cast<int>(threadIdx.x) / t.v4;
    const int n4 = t.n / 4, i4 = blk * t.v4 + v;
    const bool live = g < t.groups && i4 < n4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
        const float4* p = reinterpret_cast<const float4*>(t.part) + i4;
#pragma unroll 4
        for (int s = g; s < t.splits; s += t.groups) {
            const float4 x = __ldg(p + static_cast<size_t>(s) * n4);
            acc.x += x.x;
            acc.y += x.y;
            acc.z += x.z;
            acc.w += x.w;
        }
    }
    if (g < t.groups) red[g * t.v4 + v] = acc;
    __syncthreads();
    for (int h = t.groups / 2; h > 0; h >>= 1) {   // uniform over the block
        if (g < h) {
            float4& x = red[g * t.v4 + v];
            const float4 y = red[(g + h) * t.v4 + v];
            x.x += y.x;
            x.y += y.y;
            x.z += y.z;
            x.w += y.w;
        }
        __syncthreads();
    }
    if (g == 0 && live) {
        float4 r = red[v];
        float4* o = reinterpret_cast<float4*>(t.out) + i4;
        if (accumulate) {
            const float4 x = *o;
            r.x += x.x;
            r.y += x.y;
            r.z += x.z;
            r.w += x.w;
        }
        *o = r;
    }
}

// The block shape of one sum: up to 32 output quads, and the largest power of two of split
// groups that fits 512 threads (at most the split count).
SplitSum split_sum(const float* part, int splits, int n, float* out) {
    SplitSum t{part, splits, n, out, 1, 1};
    t.v4 = n / 4 < 32 ? (n / 4 > 0 ? n / 4 : 1) : 32;
    while (t.groups * 2 * t.v4 <= 512 && t.groups < splits) t.groups *= 2;
    return t;
}

cudaError_t launch_split_sum(const SplitSum& a, const SplitSum& b, int accumulate, cudaStream_t st) {
    for (const SplitSum* t : {&a, &b})
        if (t->n % 4 || ((reinterpret_cast<uintptr_t>(t->part) | reinterpret_cast<uintptr_t>(t->out)) & 15))
            return cudaErrorInvalidValue;
    const int ba = (a.n / 4 + a.v4 - 1) / a.v4, bb = (b.n / 4 + b.v4 - 1) / b.v4;
    if (ba + bb == 0) return cudaSuccess;
    split_sum_kernel<<<ba + bb, 512, 0, st>>>(a, b, ba, accumulate);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Elementwise kernels
// ---------------------------------------------------------------------------------
inline unsigned blocks(size_t n, unsigned per = 256) { return static_cast<unsigned>((n + per - 1) / per); }

// Channel sums of the DS pixels (3 DS bytes, DS = 4 or 8) starting at p, read as 4- or
// 8-byte words (3 DS is a multiple of 12 and p = 3 DS (W qx + ...) keeps them aligned).
template <int DS>
__device__ __forceinline__ void row_channel_sums(const uint8_t* __restrict__ p, uint32_t (&s)[3]) {
    constexpr int WORDS = 3 * DS / 4;
    const uint32_t* q = reinterpret_cast<const uint32_t*>(p);
    uint32_t w[WORDS];
    if constexpr (DS == 8) {
#pragma unroll
        for (int k = 0; k < WORDS / 2; ++k) {
            const uint2 v = __ldg(reinterpret_cast<const uint2*>(q) + k);
            w[2 * k] = v.x;
            w[2 * k + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < WORDS; ++k) w[k] = __ldg(q + k);
    }
#pragma unroll
    for (int b = 0; b < 3 * DS; ++b) s[b % 3] += (w[b >> 2] >> (8 * (b & 3))) & 0xFFu;
}

// Network input: DS x DS box means of both guides, scaled to [-0.5, 0.5], 8 channels.  The
// block sums are exact integers, so the result does not depend on the summation order.
template <int DS>
__device__ __forceinline__ void box_means(const uint8_t* __restrict__ src, const uint8_t* __restrict__ tgt,
                                         int W, int qy, int qx, bf16* __restrict__ o) {
    uint32_t a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    for (int dy = 0; dy < DS; ++dy) {
        const size_t p = (static_cast<size_t>(DS * qy + dy) * W + DS * qx) * 3;
        row_channel_sums<DS>(src + p, a);
        row_channel_sums<DS>(tgt + p, b);
    }
    const float scale = 1.f / (static_cast<float>(DS * DS) * 255.f);
    for (int ch = 0; ch < 3; ++ch) {
        o[ch] = __float2bfloat16_rn(static_cast<float>(a[ch]) * scale - 0.5f);
        o[3 + ch] = __float2bfloat16_rn(static_cast<float>(b[ch]) * scale - 0.5f);
    }
    o[6] = o[7] = __float2bfloat16_rn(0.f);
}

// The same sums read byte by byte, for caller stacks that are not 8-byte aligned.
__device__ __forceinline__ void box_means_bytes(const uint8_t* __restrict__ src, const uint8_t* __restrict__ tgt,
                                                int W, int DS, int qy, int qx, bf16* __restrict__ o) {
    uint32_t a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    for (int dy = 0; dy < DS; ++dy)
        for (int dx = 0; dx < DS; ++dx) {
            const size_t p = (static_cast<size_t>(DS * qy + dy) * W + DS * qx + dx) * 3;
            for (int ch = 0; ch < 3; ++ch) {
                a[ch] += src[p + ch];
                b[ch] += tgt[p + ch];
            }
        }
    const float scale = 1.f / (static_cast<float>(DS * DS) * 255.f);
    for (int ch = 0; ch < 3; ++ch) {
        o[ch] = __float2bfloat16_rn(static_cast<float>(a[ch]) * scale - 0.5f);
        o[3 + ch] = __float2bfloat16_rn(static_cast<float>(b[ch]) * scale - 0.5f);
    }
    o[6] = o[7] = __float2bfloat16_rn(0.f);
}

__global__ void prep_input_kernel(const uint8_t* __restrict__ src, const uint8_t* __restrict__ tgt,
                                  int n, int H, int W, int DS, int aligned, bf16* __restrict__ out) {
    const int Hq = H / DS, Wq = W / DS;
    const size_t total = static_cast<size_t>(n) * Hq * Wq;
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int img = static_cast<int>(i / (static_cast<size_t>(Hq) * Wq));
    const int rem = static_cast<int>(i - static_cast<size_t>(img) * Hq * Wq);
    const int qy = rem / Wq, qx = rem % Wq;
    const size_t fsz = static_cast<size_t>(H) * W * 3;
    if (!aligned)
        box_means_bytes(src + img * fsz, tgt + img * fsz, W, DS, qy, qx, out + i * 8);
    else if (DS == 8)
        box_means<8>(src + img * fsz, tgt + img * fsz, W, qy, qx, out + i * 8);
    else
        box_means<4>(src + img * fsz, tgt + img * fsz, W, qy, qx, out + i * 8);
}

// The same input built from a guide stack and pairs [first, first + n) of a pair table.
__global__ void prep_input_pairs_kernel(const uint8_t* __restrict__ guides,
                                        const fb::PairDesc* __restrict__ pairs, int first, int n,
                                        int H, int W, int DS, int aligned, bf16* __restrict__ out) {
    const int Hq = H / DS, Wq = W / DS;
    const size_t total = static_cast<size_t>(n) * Hq * Wq;
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int img = static_cast<int>(i / (static_cast<size_t>(Hq) * Wq));
    const int rem = static_cast<int>(i - static_cast<size_t>(img) * Hq * Wq);
    const int qy = rem / Wq, qx = rem % Wq;
    const fb::PairDesc pd = pairs[first + img];
    const size_t fsz = static_cast<size_t>(H) * W * 3;
    const uint8_t* src = guides + static_cast<size_t>(pd.src) * fsz;
    const uint8_t* tgt = guides + static_cast<size_t>(pd.tgt) * fsz;
    if (!aligned)
        box_means_bytes(src, tgt, W, DS, qy, qx, out + i * 8);
    else if (DS == 8)
        box_means<8>(src, tgt, W, qy, qx, out + i * 8);
    else
        box_means<4>(src, tgt, W, qy, qx, out + i * 8);
}

// Training targets from Alg. 1 fields: the mean offset F(x) - x over each DS x DS block,
// with weight 1 where every offset of the block lies within DS/2 pixels of that mean
// (one coherent motion), else 0.
__global__ void nnf_targets_kernel(const int32_t* __restrict__ nnf, int n, int H, int W, int DS,
                                   float* __restrict__ target, float* __restrict__ weight) {
    const int Hq = H / DS, Wq = W / DS;
    const size_t total = static_cast<size_t>(n) * Hq * Wq;
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int img = static_cast<int>(i / (static_cast<size_t>(Hq) * Wq));
    const int rem = static_cast<int>(i - static_cast<size_t>(img) * Hq * Wq);
    const int qy = rem / Wq, qx = rem % Wq;
    float my = 0.f, mx = 0.f;
    for (int j = 0; j < DS * DS; ++j) {
        const int y = DS * qy + j / DS, x = DS * qx + j % DS;
        const size_t p = (static_cast<size_t>(img) * H + y) * W + x;
        my += static_cast<float>(nnf[2 * p] - y);
        mx += static_cast<float>(nnf[2 * p + 1] - x);
    }
    my /= static_cast<float>(DS * DS);
    mx /= static_cast<float>(DS * DS);
    const float tol = 0.5f * DS;
    bool ok = true;
    for (int j = 0; j < DS * DS; ++j) {
        const int y = DS * qy + j / DS, x = DS * qx + j % DS;
        const size_t p = (static_cast<size_t>(img) * H + y) * W + x;
        ok = ok && fabsf(static_cast<float>(nnf[2 * p] - y) - my) <= tol &&
             fabsf(static_cast<float>(nnf[2 * p + 1] - x) - mx) <= tol;
    }
    target[2 * i] = my;
    target[2 * i + 1] = mx;
    if (weight) weight[i] = ok ? 1.f : 0.f;
}

// out[n][2h][2w][C1+C2] = [nearest-upsampled lo, skip]
__global__ void concat_up_kernel(const bf16* __restrict__ lo, int C1, const bf16* __restrict__ skip,
                                 int C2, int n, int H2, int W2, bf16* __restrict__ out) {
    const int C = C1 + C2;
    const size_t total = static_cast<size_t>(n) * H2 * W2 * (C / 8);
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int u = static_cast<int>(i % (C / 8));
    const size_t pix = i / (C / 8);
    const int img = static_cast<int>(pix / (static_cast<size_t>(H2) * W2));
    const int rem = static_cast<int>(pix - static_cast<size_t>(img) * H2 * W2);
    const int y = rem / W2, x = rem % W2;
    const int c = 8 * u;
    uint4 v;
    if (c < C1) {
        const size_t lp = (static_cast<size_t>(img) * (H2 / 2) + y / 2) * (W2 / 2) + x / 2;
        v = *reinterpret_cast<const uint4*>(lo + lp * C1 + c);
    } else {
        v = *reinterpret_cast<const uint4*>(skip + pix * C2 + (c - C1));
    }
    *reinterpret_cast<uint4*>(out + pix * C + c) = v;
}

// Gradient of concat_up: dlo[n][h][w][C1] += sum over the 2x2 block, dskip += its part.
// Gradient of the upsampled part of a concatenation: dlo[p][c] = the sum of the 2 x 2
// block of dout's first C1 channels above p, added to dlo (acc_lo) or written (first
// writer).  The skip part (dout's last C2 channels) is not copied: the ReLU backward of the
// skip tensor's layer adds it where it reads that tensor's gradient.  One thread per 8
// channels of one pixel (C1, C2 multiples of 8), 32-byte accesses; the same sums per value.
__global__ void concat_up_bwd_kernel(const float* __restrict__ dout, int C1, int C2, int n, int H2,
                                     int W2, float* __restrict__ dlo, int acc_lo) {
    const int C = C1 + C2;
    const int H = H2 / 2, W = W2 / 2;
    const size_t units = static_cast<size_t>(n) * H * W * (C1 / 8);
    const size_t u = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (u >= units) return;
    const int c = static_cast<int>(u % (C1 / 8)) * 8;
    const size_t p = u / (C1 / 8);
    const int img = static_cast<int>(p / (static_cast<size_t>(H) * W));
    const int rem = static_cast<int>(p - static_cast<size_t>(img) * H * W);
    const int y = rem / W, x = rem % W;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
            const float4* q = reinterpret_cast<const float4*>(
                dout + ((static_cast<size_t>(img) * H2 + 2 * y + dy) * W2 + 2 * x + dx) * C + c);
            const float4 a = __ldg(q), b = __ldg(q + 1);
            s[0] += a.x; s[1] += a.y; s[2] += a.z; s[3] += a.w;
            s[4] += b.x; s[5] += b.y; s[6] += b.z; s[7] += b.w;
        }
    float4* d = reinterpret_cast<float4*>(dlo + p * C1 + c);
    if (acc_lo) {
        const float4 a = d[0], b = d[1];
        d[0] = make_float4(a.x + s[0], a.y + s[1], a.z + s[2], a.w + s[3]);
        d[1] = make_float4(b.x + s[4], b.y + s[5], b.z + s[6], b.w + s[7]);
    } else {
        d[0] = make_float4(s[0], s[1], s[2], s[3]);
        d[1] = make_float4(s[4], s[5], s[6], s[7]);
    }
}

// dZ = dA * (A > 0) in bf16 (ReLU backward); relu == 0 passes dA through.  With add, the
// gradient is dA + the skip slice of a concatenation's gradient: add[(i / C) * add_stride +
// add_off + i % C] (the skip tensor's other consumer).  One thread per 8 values (C, n,
// add_stride and add_off multiples of 8), 16- and 32-byte accesses; A is read only with relu.
__global__ void relu_bwd_kernel(const float* __restrict__ dA, const bf16* __restrict__ A, size_t n,
                                int relu, bf16* __restrict__ dZ, const float* __restrict__ add, int C,
                                int add_stride, int add_off) {
    const size_t i = (static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 8;
    if (i >= n) return;
    const float4 a0 = __ldg(reinterpret_cast<const float4*>(dA + i));
    const float4 a1 = __ldg(reinterpret_cast<const float4*>(dA + i) + 1);
    float g[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    if (add) {
        const float4* q = reinterpret_cast<const float4*>(add + (i / C) * add_stride + add_off + i % C);
        const float4 b0 = __ldg(q), b1 = __ldg(q + 1);
        g[0] += b0.x; g[1] += b0.y; g[2] += b0.z; g[3] += b0.w;
        g[4] += b1.x; g[5] += b1.y; g[6] += b1.z; g[7] += b1.w;
    }
    __align__(16) bf16 z[8];
    if (relu) {
        __align__(16) bf16 a[8];
        *reinterpret_cast<uint4*>(a) = __ldg(reinterpret_cast<const uint4*>(A + i));
#pragma unroll
        for (int j = 0; j < 8; ++j) z[j] = __float2bfloat16_rn(!(__bfloat162float(a[j]) > 0.f) ? 0.f : g[j]);
    } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) z[j] = __float2bfloat16_rn(g[j]);
    }
    *reinterpret_cast<uint4*>(dZ + i) = *reinterpret_cast<const uint4*>(z);
}

// Partial sums of db[c] = sum over the P pixels of dZ[p][c] (C a multiple of 8, at most
// 128).  Coalesced: a pixel row's C / 8 threads each read 8 channels as one 16-byte load, a
// 512-thread block walks `rows` rows at a time (the largest power of two that fits) over a
// grid-strided range of pixels, adds its rows by a fixed pairwise tree in shared memory
// and stores one partial sum per channel to part[blockIdx.x][c]; split_sum_kernel adds
// the blocks' partials.
constexpr int kBiasBlocks = 512;   // at most
constexpr int kBiasThreads = 512;

__host__ __device__ constexpr int bias_rows(int C) {
    int r = 1;
    while (2 * r * (C / 8) <= kBiasThreads) r *= 2;
    return r;
}

// Blocks of bias_grad_kernel for P pixels of C channels: enough to stream dZ, and few
// enough that the split sum adds at most 8 partials per thread.
int bias_blocks(size_t P, int C) {
    const size_t rows = bias_rows(C), need = (P + rows - 1) / rows;
    int cap = kBiasBlocks, g = 1;
    while (g * 2 * (C / 4) <= 512) g *= 2;
    if (8 * g < cap) cap = 8 * g;
    return static_cast<int>(need < static_cast<size_t>(cap) ? need : cap);
}

__global__ void __launch_bounds__(kBiasThreads) bias_grad_kernel(const bf16* __restrict__ dZ, size_t P, int C,
                                                                 float* __restrict__ part) {
    __shared__ float red[kBiasThreads * 8];
    const int tpp = C / 8, rows = bias_rows(C);
    const int t = static_cast<int>(threadIdx.x), r = t / tpp, u = t - r * tpp;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (r < rows) {
#pragma unroll 4
        for (size_t p = static_cast<size_t>(blockIdx.x) * rows + r; p < P; p += static_cast<size_t>(gridDim.x) * rows) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(dZ + p * C + 8 * u));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                s[2 * j] += __uint_as_float(w[j] << 16);             // low bf16
                s[2 * j + 1] += __uint_as_float(w[j] & 0xFFFF0000u);  // high bf16
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) red[r * C + 8 * u + j] = s[j];
    }
    for (int h = rows / 2; h > 0; h >>= 1) {   // uniform over the block
        __syncthreads();
        if (r < h) {
#pragma unroll
            for (int j = 0; j < 8; ++j) red[r * C + 8 * u + j] += red[(r + h) * C + 8 * u + j];
        }
    }
    __syncthreads();
    if (t < C) part[static_cast<size_t>(blockIdx.x) * C + t] = red[t];
}

// Smooth-L1 (Huber, delta 1 pixel) between 16 * head[..., 0:2] and the target offsets,
// weighted, averaged over the weight sum.  Writes dHead (fp32, 8 channels) and adds the
// loss to *loss.
__global__ void offset_loss_kernel(const float* __restrict__ head, const float* __restrict__ target,
                                   const float* __restrict__ weight, size_t P, float inv_wsum,
                                   float* __restrict__ dhead, float* __restrict__ loss) {
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < P) {
        const float w = weight ? weight[i] : 1.f;
        for (int ch = 0; ch < 8; ++ch) dhead[i * 8 + ch] = 0.f;
        for (int ch = 0; ch < 2; ++ch) {
            const float d = kOffsetScale * head[i * 8 + ch] - target[i * 2 + ch];
            const float ad = fabsf(d);
            l += w * (ad < 1.f ? 0.5f * d * d : ad - 0.5f);
            const float g = ad < 1.f ? d : (d > 0.f ? 1.f : -1.f);
            dhead[i * 8 + ch] = w * g * kOffsetScale * inv_wsum;
        }
    }
    __shared__ float red[256];
    red[threadIdx.x] = l;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (static_cast<int>(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv_wsum);
}

// fp32 master weights [Cout][9][Cin] -> bf16 copy and bf16 transpose [Cin][9][Cout].
__global__ void weights_to_bf16_kernel(const float* __restrict__ w, int Cout, int Cin,
                                       bf16* __restrict__ wb, bf16* __restrict__ wt) {
    const size_t n = static_cast<size_t>(Cout) * 9 * Cin;
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ci = static_cast<int>(i % Cin);
    const int tap = static_cast<int>((i / Cin) % 9);
    const int co = static_cast<int>(i / (9 * static_cast<size_t>(Cin)));
    const bf16 v = __float2bfloat16_rn(w[i]);
    wb[i] = v;
    wt[(static_cast<size_t>(ci) * 9 + tap) * Cout + co] = v;
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Initial NNF from predicted offsets: F0(x) = clamp(x + rint(offset(x / DS))).
__global__ void offsets_to_nnf_kernel(const float* __restrict__ head, int n, int H, int W, int DS,
                                      int32_t* __restrict__ nnf) {
    const size_t total = static_cast<size_t>(n) * H * W;
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int img = static_cast<int>(i / (static_cast<size_t>(H) * W));
    const int rem = static_cast<int>(i - static_cast<size_t>(img) * H * W);
    const int y = rem / W, x = rem % W;
    const int Hq = H / DS, Wq = W / DS;
    const size_t q = (static_cast<size_t>(img) * Hq + min(y / DS, Hq - 1)) * Wq + min(x / DS, Wq - 1);
    const float dy = kOffsetScale * head[q * 8 + 0], dx = kOffsetScale * head[q * 8 + 1];
    const int ry = y + static_cast<int>(rintf(fminf(fmaxf(dy, -32768.f), 32768.f)));
    const int rx = x + static_cast<int>(rintf(fminf(fmaxf(dx, -32768.f), 32768.f)));
    nnf[2 * i] = min(max(ry, 0), H - 1);
    nnf[2 * i + 1] = min(max(rx, 0), W - 1);
}

// ---------------------------------------------------------------------------------
// Network
// ---------------------------------------------------------------------------------
struct LayerDef {
    int cin, cout, stride, relu;
};
// e0a e0b e1a e1b e2a e2b e3a e3b d2 d1 d0 head
constexpr LayerDef kLayers[12] = {
    {8, 32, 1, 1},    {32, 32, 1, 1},   {32, 64, 2, 1},  {64, 64, 1, 1},
    {64, 96, 2, 1},   {96, 96, 1, 1},   {96, 128, 2, 1}, {128, 128, 1, 1},
    {224, 96, 1, 1},  {160, 64, 1, 1},  {96, 32, 1, 1},  {32, 8, 1, 0}};
constexpr int kNumLayers = 12;

size_t layer_weights(int l) { return static_cast<size_t>(kLayers[l].cout) * 9 * kLayers[l].cin; }

}  // namespace
}  // namespace net
}  // namespace fb

using fb::net::bf16;
using fb::net::ConvGeom;
using fb::net::kLayers;
using fb::net::kNumLayers;

struct fb_initnet {
    fb_ctx* ctx = nullptr;
    int device = 0;
    int max_pairs = 0, H = 0, W = 0;
    int ds = 4;                             // guide pixels per network pixel, per axis
    int sms = 0;
    size_t n_params = 0;                    // weights + biases
    size_t w_off[kNumLayers], b_off[kNumLayers];
    float* params = nullptr;                // fp32 master: [w0 b0 w1 b1 ...]
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    bf16* wb = nullptr;                     // bf16 weights, per layer at w_off
    bf16* wt = nullptr;                     // bf16 transposed weights
    // activations (bf16) and gradients (fp32), sized for max_pairs
    bf16* act[16] = {};
    float* dact[16] = {};
    bf16* dz = nullptr;                     // scratch: bf16 dZ of the largest layer
    bf16* dz2 = nullptr;                    // ... and a second one (fused ReLU backward)
    float* wpart = nullptr;                 // per-split weight-gradient slices of one layer
    float* bpart = nullptr;                 // per-block bias-gradient partials of one layer
    float* head = nullptr;                  // fp32 head output [P][8]
    float* loss = nullptr;
    int* status = nullptr;
    uint64_t step = 0;
    char* arena = nullptr;
    std::string err;
};

namespace {

using fb::net::ConvGeom;

int net_fail(fb_initnet* net, int status, const char* msg) {
    if (net) net->err = msg;
    return status;
}

#define NET_CUDA(net, expr)                                                  \
    do {                                                                     \
        cudaError_t e_ = (expr);                                             \
        if (e_ != cudaSuccess) {                                             \
            cudaGetLastError();                                              \
            return net_fail(net, FB_ERR_CUDA, cudaGetErrorString(e_));       \
        }                                                                    \
    } while (0)

// Spatial size (Hq-relative divisor) of each tensor:
//   act[0]=input(1) act[1]=e0a act[2]=e0b(1) act[3]=e1a act[4]=e1b(2) act[5]=e2a
//   act[6]=e2b(4) act[7]=e3a act[8]=e3b(8) act[9]=cat2(4) act[10]=d2(4) act[11]=cat1(2)
//   act[12]=d1(2) act[13]=cat0(1) act[14]=d0(1)
struct Tens {
    int div, ch;
};
constexpr Tens kTens[15] = {{1, 8},   {1, 32},  {1, 32},  {2, 64},  {2, 64},
                            {4, 96},  {4, 96},  {8, 128}, {8, 128}, {4, 224},
                            {4, 96},  {2, 160}, {2, 64},  {1, 96},  {1, 32}};
// layer l: input tensor, output tensor
constexpr int kIn[12] = {0, 1, 2, 3, 4, 5, 6, 7, 9, 11, 13, 14};
constexpr int kOut[12] = {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, -1};

ConvGeom geom(const fb_initnet* net, int l, int n) {
    const int Hq = net->H / net->ds, Wq = net->W / net->ds;
    const fb::net::LayerDef& d = kLayers[l];
    const int hin = Hq / kTens[kIn[l]].div, win = Wq / kTens[kIn[l]].div;
    ConvGeom g;
    g.n = n;
    g.H = hin;
    g.W = win;
    g.Cin = d.cin;
    g.stride = d.stride;
    g.Ho = (hin + d.stride - 1) / d.stride;
    g.Wo = (win + d.stride - 1) / d.stride;
    g.Cout = d.cout;
    return g;
}

size_t tens_elems(const fb_initnet* net, int t, int n) {
    const int Hq = net->H / net->ds, Wq = net->W / net->ds;
    return static_cast<size_t>(n) * (Hq / kTens[t].div) * (Wq / kTens[t].div) * kTens[t].ch;
}

int net_layers(fb_initnet* net, int n, cudaStream_t st);

int net_forward(fb_initnet* net, const uint8_t* src, const uint8_t* tgt, int n, cudaStream_t st) {
    using namespace fb::net;
    const size_t Pq = static_cast<size_t>(n) * (net->H / net->ds) * (net->W / net->ds);
    // 8-byte aligned stacks (every frame then is: W is a multiple of 64) take vector loads
    const int aligned = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(tgt)) & 7) == 0;
    prep_input_kernel<<<blocks(Pq), 256, 0, st>>>(src, tgt, n, net->H, net->W, net->ds, aligned, net->act[0]);
    NET_CUDA(net, cudaGetLastError());
    return net_layers(net, n, st);
}

// The twelve layers on the input already in act[0].
int net_layers(fb_initnet* net, int n, cudaStream_t st) {
    using namespace fb::net;
    for (int l = 0; l < kNumLayers; ++l) {
        if (l == 8 || l == 9 || l == 10) {  // build the decoder's concatenated input
            const int lo = l == 8 ? 8 : (l == 9 ? 10 : 12);
            const int skip = l == 8 ? 6 : (l == 9 ? 4 : 2);
            const int cat = kIn[l];
            const int H2 = (net->H / net->ds) / kTens[cat].div, W2 = (net->W / net->ds) / kTens[cat].div;
            const size_t units = static_cast<size_t>(n) * H2 * W2 * (kTens[cat].ch / 8);
            concat_up_kernel<<<blocks(units), 256, 0, st>>>(net->act[lo], kTens[lo].ch, net->act[skip],
                                                             kTens[skip].ch, n, H2, W2, net->act[cat]);
            NET_CUDA(net, cudaGetLastError());
        }
        const ConvGeom g = geom(net, l, n);
        const bool head = kOut[l] < 0;
        NET_CUDA(net, conv_forward(g, net->act[kIn[l]], net->wb + net->w_off[l], net->params + net->b_off[l],
                                   kLayers[l].relu, head ? nullptr : net->act[kOut[l]],
                                   head ? net->head : nullptr, net->status, st));
    }
    return FB_OK;
}

int refresh_bf16(fb_initnet* net, cudaStream_t st) {
    using namespace fb::net;
    for (int l = 0; l < kNumLayers; ++l) {
        const size_t nw = layer_weights(l);
        weights_to_bf16_kernel<<<blocks(nw), 256, 0, st>>>(net->params + net->w_off[l], kLayers[l].cout,
                                                            kLayers[l].cin, net->wb + net->w_off[l],
                                                            net->wt + net->w_off[l]);
        NET_CUDA(net, cudaGetLastError());
    }
    return FB_OK;
}

}  // namespace

namespace fb {

int initnet_init_pairs(::fb_initnet* net, const uint8_t* guides, const PairDesc* pairs, int first,
                       int n, int32_t* nnf_out, cudaStream_t st) {
    using namespace fb::net;
    if (n < 1 || n > net->max_pairs) return FB_ERR_ARG;
    const size_t Pq = static_cast<size_t>(n) * (net->H / net->ds) * (net->W / net->ds);
    prep_input_pairs_kernel<<<blocks(Pq), 256, 0, st>>>(guides, pairs, first, n, net->H, net->W,
                                                        net->ds, (reinterpret_cast<uintptr_t>(guides) & 7) == 0, net->act[0]);
    NET_CUDA(net, cudaGetLastError());
    int rc = net_layers(net, n, st);
    if (rc) return rc;
    const size_t total = static_cast<size_t>(n) * net->H * net->W;
    offsets_to_nnf_kernel<<<blocks(total), 256, 0, st>>>(net->head, n, net->H, net->W, net->ds, nnf_out);
    NET_CUDA(net, cudaGetLastError());
    return FB_OK;
}

int initnet_max_pairs(const ::fb_initnet* net) { return net->max_pairs; }

void initnet_dims(const ::fb_initnet* net, int* H, int* W) {
    *H = net->H;
    *W = net->W;
}

}  // namespace fb

extern "C" {

int fb_initnet_targets(const int32_t* nnf, int n, int H, int W, int downscale, float* target,
                       float* weight, void* stream) {
    if (!nnf || !target || n < 1 || (downscale != 4 && downscale != 8) || H % downscale || W % downscale)
        return FB_ERR_ARG;
    const size_t total = static_cast<size_t>(n) * (H / downscale) * (W / downscale);
    fb::net::nnf_targets_kernel<<<fb::net::blocks(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        nnf, n, H, W, downscale, target, weight);
    return cudaGetLastError() == cudaSuccess ? FB_OK : FB_ERR_CUDA;
}

int fb_initnet_create(fb_ctx* ctx, fb_initnet** out, int max_pairs, int H, int W, int downscale) {
    if (!ctx || !out) return FB_ERR_ARG;
    *out = nullptr;
    if (downscale != 4 && downscale != 8) return FB_ERR_ARG;
    const int unit = 8 * downscale;  // three stride-2 levels below the network resolution
    if (max_pairs < 1 || H < unit || W < unit || H % unit || W % unit || H > 32767 || W > 32767)
        return FB_ERR_ARG;
    fb_initnet* net = new fb_initnet();
    net->ds = downscale;
    net->ctx = ctx;
    cudaGetDevice(&net->device);
    net->max_pairs = max_pairs;
    net->H = H;
    net->W = W;
    cudaDeviceGetAttribute(&net->sms, cudaDevAttrMultiProcessorCount, net->device);
    size_t off = 0;
    for (int l = 0; l < kNumLayers; ++l) {
        net->w_off[l] = off;
        off += fb::net::layer_weights(l);
        net->b_off[l] = off;
        off += kLayers[l].cout;
    }
    net->n_params = off;
    // one arena
    size_t bytes = 0;
    auto take = [&](size_t nbytes) {
        const size_t o = bytes;
        bytes += (nbytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_p = take(off * 4), o_g = take(off * 4), o_m = take(off * 4), o_v = take(off * 4);
    const size_t o_wb = take(off * 2), o_wt = take(off * 2);
    size_t o_act[15], o_dact[15], max_t = 0;
    for (int t = 0; t < 15; ++t) {
        const size_t e = tens_elems(net, t, max_pairs);
        max_t = e > max_t ? e : max_t;
        o_act[t] = take(e * 2);
        o_dact[t] = take(e * 4);
    }
    const size_t Pq = static_cast<size_t>(max_pairs) * (H / downscale) * (W / downscale);
    const size_t o_dz = take(max_t * 2), o_dz2 = take(max_t * 2), o_head = take(Pq * 8 * 4),
                 o_dhead = take(Pq * 8 * 4);
    const size_t o_loss = take(4), o_status = take(4);
    size_t wpart = 0;
    for (int l = 0; l < kNumLayers; ++l) {
        const size_t f = fb::net::wgrad_part_floats(geom(net, l, max_pairs), net->sms);
        wpart = f > wpart ? f : wpart;
    }
    const size_t o_wpart = take(wpart * 4), o_bpart = take(static_cast<size_t>(fb::net::kBiasBlocks) * 128 * 4);
    if (cudaMalloc(reinterpret_cast<void**>(&net->arena), bytes) != cudaSuccess) {
        cudaGetLastError();
        delete net;
        return FB_ERR_OOM;
    }
    cudaMemset(net->arena, 0, bytes);
    char* a = net->arena;
    net->params = reinterpret_cast<float*>(a + o_p);
    net->grads = reinterpret_cast<float*>(a + o_g);
    net->adam_m = reinterpret_cast<float*>(a + o_m);
    net->adam_v = reinterpret_cast<float*>(a + o_v);
    net->wb = reinterpret_cast<bf16*>(a + o_wb);
    net->wt = reinterpret_cast<bf16*>(a + o_wt);
    for (int t = 0; t < 15; ++t) {
        net->act[t] = reinterpret_cast<bf16*>(a + o_act[t]);
        net->dact[t] = reinterpret_cast<float*>(a + o_dact[t]);
    }
    net->dact[15] = reinterpret_cast<float*>(a + o_dhead);  // gradient of the head output
    net->dz = reinterpret_cast<bf16*>(a + o_dz);
    net->dz2 = reinterpret_cast<bf16*>(a + o_dz2);
    net->wpart = reinterpret_cast<float*>(a + o_wpart);
    net->bpart = reinterpret_cast<float*>(a + o_bpart);
    net->head = reinterpret_cast<float*>(a + o_head);
    net->loss = reinterpret_cast<float*>(a + o_loss);
    net->status = reinterpret_cast<int*>(a + o_status);
    *out = net;
    return FB_OK;
}

int fb_initnet_destroy(fb_initnet* net) {
    if (!net) return FB_OK;
    cudaDeviceSynchronize();
    if (net->arena) cudaFree(net->arena);
    delete net;
    return FB_OK;
}

const char* fb_initnet_last_error(const fb_initnet* net) { return net ? net->err.c_str() : ""; }

size_t fb_initnet_param_count(const fb_initnet* net) { return net ? net->n_params : 0; }

int fb_initnet_get_params(fb_initnet* net, float* host_out) {
    if (!net || !host_out) return FB_ERR_ARG;
    NET_CUDA(net, cudaMemcpy(host_out, net->params, net->n_params * 4, cudaMemcpyDeviceToHost));
    return FB_OK;
}

int fb_initnet_set_params(fb_initnet* net, const float* host_in) {
    if (!net || !host_in) return FB_ERR_ARG;
    NET_CUDA(net, cudaMemcpy(net->params, host_in, net->n_params * 4, cudaMemcpyHostToDevice));
    NET_CUDA(net, cudaMemset(net->adam_m, 0, net->n_params * 4));
    NET_CUDA(net, cudaMemset(net->adam_v, 0, net->n_params * 4));
    net->step = 0;
    return refresh_bf16(net, nullptr);
}

int fb_initnet_get_optimizer(fb_initnet* net, float* m_out, float* v_out, uint64_t* step_out) {
    if (!net || !m_out || !v_out || !step_out) return FB_ERR_ARG;
    NET_CUDA(net, cudaMemcpy(m_out, net->adam_m, net->n_params * 4, cudaMemcpyDeviceToHost));
    NET_CUDA(net, cudaMemcpy(v_out, net->adam_v, net->n_params * 4, cudaMemcpyDeviceToHost));
    *step_out = net->step;
    return FB_OK;
}

int fb_initnet_set_optimizer(fb_initnet* net, const float* m_in, const float* v_in, uint64_t step) {
    if (!net || !m_in || !v_in) return FB_ERR_ARG;
    NET_CUDA(net, cudaMemcpy(net->adam_m, m_in, net->n_params * 4, cudaMemcpyHostToDevice));
    NET_CUDA(net, cudaMemcpy(net->adam_v, v_in, net->n_params * 4, cudaMemcpyHostToDevice));
    net->step = step;
    return FB_OK;
}

int fb_initnet_forward(fb_initnet* net, const uint8_t* src, const uint8_t* tgt, int n,
                       float* head_out, void* stream) {
    if (!net || !src || !tgt || n < 1 || n > net->max_pairs) return FB_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = net_forward(net, src, tgt, n, st);
    if (rc) return rc;
    fb::count_launches(net->ctx, 16);  // input, 3 concatenations, 12 convolutions
    if (head_out) {
        const size_t Pq = static_cast<size_t>(n) * (net->H / net->ds) * (net->W / net->ds);
        NET_CUDA(net, cudaMemcpyAsync(head_out, net->head, Pq * 8 * 4, cudaMemcpyDeviceToDevice, st));
    }
    return FB_OK;
}

int fb_initnet_init_nnf(fb_initnet* net, int n, int32_t* nnf_out, void* stream) {
    if (!net || !nnf_out || n < 1 || n > net->max_pairs) return FB_ERR_ARG;
    const size_t total = static_cast<size_t>(n) * net->H * net->W;
    fb::net::offsets_to_nnf_kernel<<<fb::net::blocks(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        net->head, n, net->H, net->W, net->ds, nnf_out);
    NET_CUDA(net, cudaGetLastError());
    fb::count_launches(net->ctx, 1);
    return FB_OK;
}

int fb_initnet_train_step(fb_initnet* net, const uint8_t* src, const uint8_t* tgt, int n,
                          const float* target, const float* weight, float weight_sum, float lr,
                          float* loss_out, void* stream) {
    using namespace fb::net;
    if (!net || !src || !tgt || !target || n < 1 || n > net->max_pairs || !(weight_sum > 0.f))
        return FB_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = net_forward(net, src, tgt, n, st);
    if (rc) return rc;
    const size_t Pq = static_cast<size_t>(n) * (net->H / net->ds) * (net->W / net->ds);
    NET_CUDA(net, cudaMemsetAsync(net->loss, 0, 4, st));
    int launches = 1;   // the loss
    // Every parameter's gradient is written once per step, by the split sum of its layer,
    // so the gradient buffer needs no clearing and the sums do not depend on timing.
    // Activation gradients need no clearing: the first kernel to reach a tensor writes it
    // and later ones add.  The skip tensors of the stride-2 encoder layers have two
    // consumers; their gradient is written by the next layer's input gradient, and the
    // other contribution -- the skip slice of the concatenation's gradient -- is added by
    // the ReLU backward that reads it (skip_cat: the concatenation, skip_off: its channel).
    bool written[16] = {};
    written[15] = true;   // the head's gradient, written by the loss kernel
    int skip_cat[16], skip_off[16];
    for (int t = 0; t < 16; ++t) skip_cat[t] = skip_off[t] = -1;
    offset_loss_kernel<<<blocks(Pq), 256, 0, st>>>(net->head, target, weight, Pq, 1.f / weight_sum,
                                                   net->dact[15], net->loss);
    NET_CUDA(net, cudaGetLastError());
    // The bf16 operand dZ of a layer's gradients comes from its ReLU backward, or -- when
    // the next layer's input gradient is the only writer of this layer's output gradient
    // (a plain chain link: no concatenation reads or writes it) -- straight from that
    // input gradient's epilogue, into the other of two dZ buffers.
    bf16* dzb[2] = {net->dz, net->dz2};
    int cur = 0;
    bool dz_ready = false;
    auto in_concat = [](int t) { return t == 2 || t == 4 || t == 6 || t == 8 || t == 10 || t == 12; };
    for (int l = kNumLayers - 1; l >= 0; --l) {
        const ConvGeom g = geom(net, l, n);
        bf16* dz = dzb[cur];
        if (!dz_ready) {
            const size_t out_elems = static_cast<size_t>(g.n) * g.Ho * g.Wo * g.Cout;
            const float* dA = kOut[l] < 0 ? net->dact[15] : net->dact[kOut[l]];
            const bf16* A = kOut[l] < 0 ? nullptr : net->act[kOut[l]];
            const int to = kOut[l] < 0 ? 15 : kOut[l];
            if (!written[to]) return FB_ERR_CUDA;  // unreachable: every gradient is written first
            const int cat = skip_cat[to];
            relu_bwd_kernel<<<blocks(out_elems / 8), 256, 0, st>>>(
                dA, A ? A : net->act[0], out_elems, kLayers[l].relu, dz, cat >= 0 ? net->dact[cat] : nullptr,
                g.Cout, cat >= 0 ? kTens[cat].ch : 0, skip_off[to]);
            NET_CUDA(net, cudaGetLastError());
            ++launches;
        }
        dz_ready = false;
        const size_t P = static_cast<size_t>(g.n) * g.Ho * g.Wo;
        const int bg_grid = bias_blocks(P, g.Cout);
        bias_grad_kernel<<<bg_grid, kBiasThreads, 0, st>>>(dz, P, g.Cout, net->bpart);
        NET_CUDA(net, cudaGetLastError());
        int splits = 0;
        NET_CUDA(net, conv_wgrad(g, dz, net->act[kIn[l]], net->wpart, net->sms, net->status, st, &splits));
        NET_CUDA(net, launch_split_sum(split_sum(net->wpart, splits, g.Cout * 9 * g.Cin, net->grads + net->w_off[l]),
                                       split_sum(net->bpart, bg_grid, g.Cout, net->grads + net->b_off[l]), 0, st));
        launches += 3;
        if (l > 0) {
            const int t = kIn[l];
            if (!written[t] && kOut[l - 1] == t && !in_concat(t)) {
                const EpiDgradRelu epi{dzb[cur ^ 1], net->act[t], kTens[t].ch, kLayers[l - 1].relu};
                NET_CUDA(net, conv_dgrad_epi(g, dz, net->wt + net->w_off[l], epi, net->status, st));
                cur ^= 1;
                dz_ready = true;
            } else {
                NET_CUDA(net, conv_dgrad(g, dz, net->wt + net->w_off[l], net->dact[t], written[t] ? 1 : 0,
                                         net->status, st));
            }
            written[t] = true;
            ++launches;
        }
        if (l == 8 || l == 9 || l == 10) {  // split the concatenated input's gradient
            const int lo = l == 8 ? 8 : (l == 9 ? 10 : 12);
            const int skip = l == 8 ? 6 : (l == 9 ? 4 : 2);
            const int cat = kIn[l];
            const int H2 = (net->H / net->ds) / kTens[cat].div, W2 = (net->W / net->ds) / kTens[cat].div;
            const size_t tot = tens_elems(net, lo, n) / 8;
            concat_up_bwd_kernel<<<blocks(tot), 256, 0, st>>>(net->dact[cat], kTens[lo].ch, kTens[skip].ch, n,
                                                              H2, W2, net->dact[lo], written[lo] ? 1 : 0);
            NET_CUDA(net, cudaGetLastError());
            ++launches;
            written[lo] = true;
            skip_cat[skip] = cat;
            skip_off[skip] = kTens[lo].ch;
        }
    }
    if (lr > 0.f) {
        net->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, static_cast<float>(net->step));
        const float c2 = 1.f - std::pow(b2, static_cast<float>(net->step));
        adam_kernel<<<blocks(net->n_params), 256, 0, st>>>(net->params, net->grads, net->adam_m, net->adam_v,
                                                          net->n_params, lr, b1, b2, 1e-8f, c1, c2);
        NET_CUDA(net, cudaGetLastError());
        rc = refresh_bf16(net, st);
        if (rc) return rc;
    }
    if (loss_out) NET_CUDA(net, cudaMemcpyAsync(loss_out, net->loss, 4, cudaMemcpyDeviceToDevice, st));
    // the forward's 16 and the backward's, counted above; with an update Adam 1 and the
    // bf16 refresh 12.
    fb::count_launches(net->ctx, 16 + launches + (lr > 0.f ? 13 : 0));
    return FB_OK;
}

int fb_initnet_get_grads(fb_initnet* net, float* host_out) {
    if (!net || !host_out) return FB_ERR_ARG;
    NET_CUDA(net, cudaMemcpy(host_out, net->grads, net->n_params * 4, cudaMemcpyDeviceToHost));
    return FB_OK;
}

int fb_initnet_status(fb_initnet* net) {
    if (!net) return FB_ERR_ARG;
    int s = 0;
    NET_CUDA(net, cudaMemcpy(&s, net->status, 4, cudaMemcpyDeviceToHost));
    if (s) NET_CUDA(net, cudaMemset(net->status, 0, 4));  // reported once, then cleared
    return s ? FB_ERR_TIMEOUT : FB_OK;
}

int fb_debug_set_wait_limit(int64_t polls) {
    const long v = polls >= 0 ? static_cast<long>(polls) : fb::tc::kWaitLimit;
    if (cudaDeviceSynchronize() != cudaSuccess) return FB_ERR_CUDA;
    if (cudaMemcpyToSymbol(fb::tc::g_progress_wait_limit, &v, sizeof(v)) != cudaSuccess) return FB_ERR_CUDA;
    return cudaDeviceSynchronize() == cudaSuccess ? FB_OK : FB_ERR_CUDA;
}

int fb_conv_gemm_path(int mode, uint64_t* tma_launches) {
    if (mode < -1 || mode > 2) return FB_ERR_ARG;
    if (tma_launches) *tma_launches = fb::net::g_tma_launches.load();
    if (mode >= 0) fb::net::g_gemm_path.store(mode);
    return FB_OK;
}

// Single-layer entry points (used by the gradient checks against the CPU oracle).
int fb_conv3x3_forward(const uint16_t* x, int n, int H, int W, int Cin, const uint16_t* w,
                       const float* bias, int Cout, int stride, int relu, uint16_t* y_bf16,
                       float* y_f32, int* status, void* stream) {
    if (!x || !w || !bias || (!y_bf16 && !y_f32) || Cin % 8 || Cout % 8 || Cout > 128 || Cin > 1024 ||
        (stride != 1 && stride != 2) || n < 1 || H < 1 || W < 1 || !status)
        return FB_ERR_ARG;
    ConvGeom g{n, H, W, Cin, (H + stride - 1) / stride, (W + stride - 1) / stride, Cout, stride};
    cudaError_t e = fb::net::conv_forward(g, reinterpret_cast<const bf16*>(x), reinterpret_cast<const bf16*>(w),
                                          bias, relu, reinterpret_cast<bf16*>(y_bf16), y_f32, status,
                                          static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FB_OK : FB_ERR_CUDA;
}

int fb_conv3x3_backward(const uint16_t* x, int n, int H, int W, int Cin, const uint16_t* wt,
                        int Cout, int stride, const uint16_t* dz, float* dx, float* dw, int* status,
                        void* stream) {
    if (!x || !dz || Cin % 8 || Cout % 8 || Cout > 128 || Cin > 1024 || (stride != 1 && stride != 2) ||
        n < 1 || H < 1 || W < 1 || !status || (dx && !wt))
        return FB_ERR_ARG;
    ConvGeom g{n, H, W, Cin, (H + stride - 1) / stride, (W + stride - 1) / stride, Cout, stride};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (dw) {
        using fb::net::SplitSum;
        float* part = nullptr;
        if (cudaMallocAsync(reinterpret_cast<void**>(&part), fb::net::wgrad_part_floats(g, sms) * 4, st) !=
            cudaSuccess) {
            cudaGetLastError();
            return FB_ERR_OOM;
        }
        int splits = 0;
        cudaError_t e = fb::net::conv_wgrad(g, reinterpret_cast<const bf16*>(dz), reinterpret_cast<const bf16*>(x),
                                            part, sms, status, st, &splits);
        if (e == cudaSuccess)
            e = fb::net::launch_split_sum(fb::net::split_sum(part, splits, Cout * 9 * Cin, dw),
                                          SplitSum{nullptr, 0, 0, nullptr, 1, 1}, 1, st);
        cudaFreeAsync(part, st);
        if (e != cudaSuccess) return FB_ERR_CUDA;
    }
    if (dx) {
        cudaError_t e = fb::net::conv_dgrad(g, reinterpret_cast<const bf16*>(dz), reinterpret_cast<const bf16*>(wt),
                                            dx, 0, status, st);
        if (e != cudaSuccess) return FB_ERR_CUDA;
    }
    return FB_OK;
}

}  // extern "C"
