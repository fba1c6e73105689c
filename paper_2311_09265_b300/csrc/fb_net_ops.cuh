// fb_net_ops.cuh -- 3x3 convolutions (zero padding 1, stride 1 or 2, NHWC bf16) of the
// learned NNF initialiser expressed as gathered tcgen05 GEMMs (fb_tc_gemm.cuh):
//   forward  Y[p][co]  = act(b[co] + sum_{tap,ci} X[p*s + tap - 1][ci] W[co][tap][ci])
//            GEMM M = output pixels, N = Cout, K = 9 Cin
//   dgrad    dX[q][ci] = sum_{tap,co} dZ[(q - tap + 1)/s][co] W[co][tap][ci]
//            GEMM M = input pixels, N = Cin, K = 9 Cout (B = weights transposed)
//   wgrad    dW[co][tap][ci] = sum_p dZ[p][co] X[p*s + tap - 1][ci]
//            GEMM M = Cout, N = 9 Cin, K = output pixels (split over CTAs, fp32 atomics)
// Channel counts are multiples of 8, so one 16-byte gather unit (8 channels) is one
// row of a core matrix.
#pragma once

#include <cuda_bf16.h>

#include "fb_tc_gemm.cuh"

namespace fb {
namespace net {

using bf16 = __nv_bfloat16;

struct ConvGeom {
    int n, H, W, Cin;   // input
    int Ho, Wo, Cout;   // output
    int stride;
};

__device__ __forceinline__ uint4 zero4() { return make_uint4(0u, 0u, 0u, 0u); }

__device__ __forceinline__ void store_unit(unsigned char* tile, int row, int k, uint4 v) {
    *reinterpret_cast<uint4*>(tile + tc::tile_off(row, k)) = v;
}

// ---- forward ---------------------------------------------------------------------
template <int BN>
struct GatherFwd {
    const bf16* X;   // [n][H][W][Cin]
    const bf16* Wt;  // [Cout][9*Cin]
    ConvGeom g;
    int M, K;
    __device__ __forceinline__ void load(unsigned char* sa, unsigned char* sb, int k0, int m0,
                                         int n0) const {
        const int t = threadIdx.x;
        const int m = m0 + t;
        int img = 0, oy = 0, ox = 0;
        if (m < M) {
            img = m / (g.Ho * g.Wo);
            const int rem = m - img * g.Ho * g.Wo;
            oy = rem / g.Wo;
            ox = rem - oy * g.Wo;
        }
#pragma unroll
        for (int u = 0; u < tc::BK / 8; ++u) {
            const int k = k0 + 8 * u;
            uint4 v = zero4();
            if (m < M && k < K) {
                const int tap = k / g.Cin, ci = k - tap * g.Cin;
                const int iy = oy * g.stride + tap / 3 - 1, ix = ox * g.stride + tap % 3 - 1;
                if (iy >= 0 && iy < g.H && ix >= 0 && ix < g.W)
                    v = __ldg(reinterpret_cast<const uint4*>(
                        X + ((static_cast<size_t>(img) * g.H + iy) * g.W + ix) * g.Cin + ci));
            }
            store_unit(sa, t, 8 * u, v);
        }
        for (int idx = t; idx < BN * (tc::BK / 8); idx += 128) {
            const int row = idx / (tc::BK / 8), u = idx % (tc::BK / 8);
            const int n = n0 + row, k = k0 + 8 * u;
            uint4 v = zero4();
            if (n < g.Cout && k < K)
                v = __ldg(reinterpret_cast<const uint4*>(Wt + static_cast<size_t>(n) * K + k));
            store_unit(sb, row, 8 * u, v);
        }
    }
    // Pipelined path (tc_gemm_async_kernel): K is walked tap-major in blocks of 64
    // input channels, chunk c = (tap, channel block), so a chunk is 8 contiguous 16-byte
    // copies per output pixel and the pixel is decoded once per thread.
    int ncb;  // channel blocks: (Cin + 63) / 64
    struct State {
        long long base;  // element offset of the pixel's top-left tap (may be negative)
        uint32_t ok;     // bits 0-2: tap rows inside the image, bits 3-5: tap columns
    };
    __device__ __forceinline__ State thread_state(int m0) const {
        State st{0, 0u};
        const int m = m0 + static_cast<int>(threadIdx.x);
        if (m < M) {
            const int img = m / (g.Ho * g.Wo);
            const int rem = m - img * g.Ho * g.Wo;
            const int oy = rem / g.Wo, ox = rem - (rem / g.Wo) * g.Wo;
            const int y0 = oy * g.stride - 1, x0 = ox * g.stride - 1;
            st.base = ((static_cast<long long>(img) * g.H + y0) * g.W + x0) * g.Cin;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (y0 + d >= 0 && y0 + d < g.H) st.ok |= 1u << d;
                if (x0 + d >= 0 && x0 + d < g.W) st.ok |= 1u << (3 + d);
            }
        }
        return st;
    }
    __device__ __forceinline__ int chunks() const { return 9 * ncb; }
    __device__ __forceinline__ int k_steps(int c) const {
        const int cb = c - (c / ncb) * ncb;
        return (min(64, g.Cin - 64 * cb) + 15) / 16;
    }
    __device__ __forceinline__ void load_async(const State& st, uint32_t sa, uint32_t sb, int c,
                                               int n0) const {
        const int t = threadIdx.x;
        const int tap = c / ncb, cb = c - tap * ncb;
        const int dy = (tap * 11) >> 5, dx = tap - 3 * dy;  // tap / 3, tap % 3 for tap < 9
        const int c0 = 64 * cb;
        const bool pix = ((st.ok >> dy) & (st.ok >> (3 + dx)) & 1u) != 0u;
        const long long off = st.base + (static_cast<long long>(dy) * g.W + dx) * g.Cin + c0;
#pragma unroll
        for (int u = 0; u < tc::BK / 8; ++u) {
            const bool v = pix && c0 + 8 * u < g.Cin;
            tc::cp_async16(sa + tc::tile_off(t, 8 * u), v ? X + off + 8 * u : X, v ? 16u : 0u);
        }
        for (int idx = t; idx < BN * (tc::BK / 8); idx += 128) {
            const int row = idx >> 3, u = idx & 7;
            const int n = n0 + row, ci = c0 + 8 * u;
            const bool v = n < g.Cout && ci < g.Cin;
            tc::cp_async16(sb + tc::tile_off(row, 8 * u),
                           v ? Wt + static_cast<size_t>(n) * K + tap * g.Cin + ci : Wt, v ? 16u : 0u);
        }
    }
};

// bias + optional ReLU, bf16 output [M][Cout] (or fp32 output when Yf is set).
struct EpiFwd {
    bf16* Y;
    float* Yf;
    const float* bias;
    int Cout;
    int relu;
    __device__ __forceinline__ void store(int row, int col0, const float (&v)[16]) const {
        if (Yf) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (col0 + j < Cout) Yf[static_cast<size_t>(row) * Cout + col0 + j] = v[j] + bias[col0 + j];
            return;
        }
        if (col0 + 16 <= Cout) {
            __align__(16) bf16 o[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                float x = v[j] + bias[col0 + j];
                o[j] = __float2bfloat16_rn(relu ? fmaxf(x, 0.f) : x);
            }
            uint4* d = reinterpret_cast<uint4*>(Y + static_cast<size_t>(row) * Cout + col0);
            d[0] = *reinterpret_cast<const uint4*>(&o[0]);
            d[1] = *reinterpret_cast<const uint4*>(&o[8]);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                if (col0 + j >= Cout) break;
                const float x = v[j] + bias[col0 + j];
                Y[static_cast<size_t>(row) * Cout + col0 + j] = __float2bfloat16_rn(relu ? fmaxf(x, 0.f) : x);
            }
        }
    }
};

// ---- input gradient ----------------------------------------------------------------
template <int BN>
struct GatherDgrad {
    const bf16* dZ;  // [n][Ho][Wo][Cout]
    const bf16* WT;  // [Cin][9*Cout]
    ConvGeom g;
    int M, K;        // M = n*H*W, K = 9*Cout
    __device__ __forceinline__ void load(unsigned char* sa, unsigned char* sb, int k0, int m0,
                                         int n0) const {
        const int t = threadIdx.x;
        const int m = m0 + t;
        int img = 0, y = 0, x = 0;
        if (m < M) {
            img = m / (g.H * g.W);
            const int rem = m - img * g.H * g.W;
            y = rem / g.W;
            x = rem - y * g.W;
        }
#pragma unroll
        for (int u = 0; u < tc::BK / 8; ++u) {
            const int k = k0 + 8 * u;
            uint4 v = zero4();
            if (m < M && k < K) {
                const int tap = k / g.Cout, co = k - tap * g.Cout;
                const int ty = y - tap / 3 + 1, tx = x - tap % 3 + 1;  // = output pixel * stride
                if (ty >= 0 && tx >= 0 && ty % g.stride == 0 && tx % g.stride == 0) {
                    const int oy = ty / g.stride, ox = tx / g.stride;
                    if (oy < g.Ho && ox < g.Wo)
                        v = __ldg(reinterpret_cast<const uint4*>(
                            dZ + ((static_cast<size_t>(img) * g.Ho + oy) * g.Wo + ox) * g.Cout + co));
                }
            }
            store_unit(sa, t, 8 * u, v);
        }
        for (int idx = t; idx < BN * (tc::BK / 8); idx += 128) {
            const int row = idx / (tc::BK / 8), u = idx % (tc::BK / 8);
            const int n = n0 + row, k = k0 + 8 * u;
            uint4 v = zero4();
            if (n < g.Cin && k < K)
                v = __ldg(reinterpret_cast<const uint4*>(WT + static_cast<size_t>(n) * K + k));
            store_unit(sb, row, 8 * u, v);
        }
    }
    // Pipelined path: K walked tap-major in blocks of 64 output channels, as in GatherFwd.
    int ncb;  // (Cout + 63) / 64
    struct State {
        int img, y1, x1;  // input pixel (y + 1, x + 1); img < 0 past the end
    };
    __device__ __forceinline__ State thread_state(int m0) const {
        State st{-1, 0, 0};
        const int m = m0 + static_cast<int>(threadIdx.x);
        if (m < M) {
            st.img = m / (g.H * g.W);
            const int rem = m - st.img * g.H * g.W;
            st.y1 = rem / g.W + 1;
            st.x1 = rem - (rem / g.W) * g.W + 1;
        }
        return st;
    }
    __device__ __forceinline__ int chunks() const { return 9 * ncb; }
    __device__ __forceinline__ int k_steps(int c) const {
        const int cb = c - (c / ncb) * ncb;
        return (min(64, g.Cout - 64 * cb) + 15) / 16;
    }
    __device__ __forceinline__ void load_async(const State& st, uint32_t sa, uint32_t sb, int c,
                                               int n0) const {
        const int t = threadIdx.x;
        const int tap = c / ncb, cb = c - tap * ncb;
        const int dy = (tap * 11) >> 5, dx = tap - 3 * dy;
        const int c0 = 64 * cb;
        // output pixel (ty, tx) / stride feeds input pixel (y, x) through tap (dy, dx)
        const int ty = st.y1 - dy, tx = st.x1 - dx;
        bool pix = st.img >= 0 && ty >= 0 && tx >= 0;
        int oy = ty, ox = tx;
        if (g.stride == 2) {
            pix = pix && ((ty | tx) & 1) == 0;
            oy = ty >> 1;
            ox = tx >> 1;
        }
        pix = pix && oy < g.Ho && ox < g.Wo;
        const size_t off = pix ? ((static_cast<size_t>(st.img) * g.Ho + oy) * g.Wo + ox) * g.Cout + c0 : 0;
#pragma unroll
        for (int u = 0; u < tc::BK / 8; ++u) {
            const bool v = pix && c0 + 8 * u < g.Cout;
            tc::cp_async16(sa + tc::tile_off(t, 8 * u), v ? dZ + off + 8 * u : dZ, v ? 16u : 0u);
        }
        for (int idx = t; idx < BN * (tc::BK / 8); idx += 128) {
            const int row = idx >> 3, u = idx & 7;
            const int n = n0 + row, co = c0 + 8 * u;
            const bool v = n < g.Cin && co < g.Cout;
            tc::cp_async16(sb + tc::tile_off(row, 8 * u),
                           v ? WT + static_cast<size_t>(n) * K + tap * g.Cout + co : WT, v ? 16u : 0u);
        }
    }
};

// fp32 input gradient [M][Cin], written or added; 16-byte vectors where the 16 columns lie
// inside the row (Cin % 8 == 0 keeps them aligned).
struct EpiDgrad {
    float* dX;
    int Cin;
    int accumulate;
    __device__ __forceinline__ void store(int row, int col0, const float (&v)[16]) const {
        float* d = dX + static_cast<size_t>(row) * Cin + col0;
        if (col0 + 16 <= Cin && (Cin & 3) == 0) {
            float4* d4 = reinterpret_cast<float4*>(d);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float4 o = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                if (accumulate) {
                    const float4 a = d4[q];
                    o = make_float4(a.x + o.x, a.y + o.y, a.z + o.z, a.w + o.w);
                }
                d4[q] = o;
            }
            return;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (col0 + j >= Cin) break;
            d[j] = accumulate ? d[j] + v[j] : v[j];
        }
    }
};

// Input gradient fused with the ReLU backward of the layer whose output it is: the kernel
// is the only writer of that gradient, so its value v goes straight to the bf16 operand of
// that layer's own gradients, dZ = bf16(relu && !(A > 0) ? 0 : v) -- the relu_bwd_kernel
// result -- and the fp32 gradient is never stored.
struct EpiDgradRelu {
    bf16* dZ;        // [rows][C]
    const bf16* A;   // the layer's output activation [rows][C]
    int C;
    int relu;
    __device__ __forceinline__ void store(int row, int col0, const float (&v)[16]) const {
        const size_t o = static_cast<size_t>(row) * C + col0;
        if (col0 + 16 <= C && (C & 7) == 0) {
            __align__(16) bf16 a[16], z[16];
            *reinterpret_cast<uint4*>(&a[0]) = __ldg(reinterpret_cast<const uint4*>(A + o));
            *reinterpret_cast<uint4*>(&a[8]) = __ldg(reinterpret_cast<const uint4*>(A + o + 8));
#pragma unroll
            for (int j = 0; j < 16; ++j)
                z[j] = __float2bfloat16_rn(relu && !(__bfloat162float(a[j]) > 0.f) ? 0.f : v[j]);
            uint4* d = reinterpret_cast<uint4*>(dZ + o);
            d[0] = *reinterpret_cast<const uint4*>(&z[0]);
            d[1] = *reinterpret_cast<const uint4*>(&z[8]);
            return;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (col0 + j >= C) break;
            dZ[o + j] = __float2bfloat16_rn(relu && !(__bfloat162float(A[o + j]) > 0.f) ? 0.f : v[j]);
        }
    }
};

// ---- weight gradient ---------------------------------------------------------------
template <int BN>
struct GatherWgrad {
    const bf16* dZ;  // [P][Cout], P = n*Ho*Wo
    const bf16* X;   // [n][H][W][Cin]
    ConvGeom g;
    int P;           // K of the GEMM
    __device__ __forceinline__ void load(unsigned char* sa, unsigned char* sb, int k0, int m0,
                                         int n0) const {
        const int t = threadIdx.x;
        (void)m0;  // M = Cout <= 128: one tile
        // A[co][p] = dZ[p][co]: each unit (8 channels of one pixel) scatters to 8 rows.
        const int groups_a = (g.Cout + 7) / 8;
        for (int idx = t; idx < tc::BK * groups_a; idx += 128) {
            const int j = idx / groups_a, gr = idx - j * groups_a;
            const int p = k0 + j;
            uint4 v = zero4();
            if (p < P)
                v = __ldg(reinterpret_cast<const uint4*>(dZ + static_cast<size_t>(p) * g.Cout + 8 * gr));
            const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                *reinterpret_cast<bf16*>(sa + tc::tile_off(8 * gr + q, j)) = e[q];
        }
        // B[tap*Cin + ci][p] = X[p*s + tap - 1][ci]
        constexpr int groups_b = BN / 8;
        for (int idx = t; idx < tc::BK * groups_b; idx += 128) {
            const int j = idx / groups_b, gr = idx - j * groups_b;
            const int p = k0 + j, n = n0 + 8 * gr;
            uint4 v = zero4();
            if (p < P && n < 9 * g.Cin) {
                const int tap = n / g.Cin, ci = n - tap * g.Cin;
                const int img = p / (g.Ho * g.Wo);
                const int rem = p - img * g.Ho * g.Wo;
                const int oy = rem / g.Wo, ox = rem - oy * g.Wo;
                const int iy = oy * g.stride + tap / 3 - 1, ix = ox * g.stride + tap % 3 - 1;
                if (iy >= 0 && iy < g.H && ix >= 0 && ix < g.W)
                    v = __ldg(reinterpret_cast<const uint4*>(
                        X + ((static_cast<size_t>(img) * g.H + iy) * g.W + ix) * g.Cin + ci));
            }
            const bf16* e = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                *reinterpret_cast<bf16*>(sb + tc::tile_off(8 * gr + q, j)) = e[q];
        }
    }
};

// The K split blockIdx.z stores its partial sums to its own slice of part (each slice laid
// out like dW); a separate reduction adds the slices in split order.
struct EpiWgrad {
    float* part;  // [splits][Cout][9*Cin]
    int N;        // 9*Cin
    size_t MN;    // Cout * 9*Cin: floats per slice
    __device__ __forceinline__ void store(int row, int col0, const float (&v)[16]) const {
        float* slice = part + blockIdx.z * MN + static_cast<size_t>(row) * N;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (col0 + j < N) slice[col0 + j] = v[j];
    }
};

}  // namespace net
}  // namespace fb
