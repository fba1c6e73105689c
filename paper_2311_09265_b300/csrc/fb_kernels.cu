// fb_kernels.cu -- sm_103a kernels of the FastBlend hot path (arXiv 2311.09265).
//
//   prep_guides   guide frame -> row-patch layout (Eq. 1 operands)
//   downsample    one pyramid step (Alg. 1, "resize images")
//   style_rgbx    style frame -> 4-byte pixels for single-load gathers
//   nnf_init      random / upsampled / user initial field and its Eq. 1 error
//   nnf_iter      one Jacobi iteration of Alg. 1: propagation + random search
//   combine       Alg. 2 remap of every pair of an output frame, fused with the
//                 Eq. 2 window sum (or the Sec. 3.5.2 keyframe weights) and the
//                 final division
//
// Everything on the NNF path is integer: Eq. 1 is evaluated one patch row at a time as
// |s|^2 + |t|^2 - 2 <s, t> with dp4a, which is exactly the clamp-to-edge sum of squared
// byte differences; a candidate stops loading rows once its running sum reaches the
// incumbent's error.
#include "fb_internal.h"

namespace fb {
namespace {

#ifndef FB_ITER_MIN_BLOCKS
#define FB_ITER_MIN_BLOCKS 5  // resident 256-thread blocks per SM the k=5 iteration kernel is built for
#endif
#ifndef FB_TILE_H
#define FB_TILE_H 8
#endif

constexpr int TILE_W = 32;
constexpr int TILE_H = FB_TILE_H;
constexpr int TILE_THREADS = TILE_W * TILE_H;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }
__device__ __forceinline__ uint32_t pack_rc(int r, int c) {
    return (static_cast<uint32_t>(r) << 16) | static_cast<uint32_t>(c);
}
__device__ __forceinline__ int row_of(uint32_t f) { return static_cast<int>(f >> 16); }
__device__ __forceinline__ int col_of(uint32_t f) { return static_cast<int>(f & 0xFFFFu); }

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplies whose halves are recombined with the round key; the key advances by
// the two Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 v, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo_a = 0xD2511F53u * v.x, hi_a = __umulhi(0xD2511F53u, v.x);
        const uint32_t lo_b = 0xCD9E8D57u * v.z, hi_b = __umulhi(0xCD9E8D57u, v.z);
        v = make_uint4(hi_b ^ v.y ^ k0, lo_b, hi_a ^ v.w ^ k1, lo_a);
    }
    return v;
}

template <int K>
struct Geo {
    static constexpr int P = K / 2;
    static constexpr int NW = (3 * K + 3) / 4;    // 32-bit words holding one 3K-byte patch row
    static constexpr int RPW = (NW + 3) / 4 * 4;  // row-patch slot stride: 16-byte aligned
};

// ---------------------------------------------------------------------------------
// Guide preparation: "row patches".  Slot (r, c) holds the k pixels
// (r, clamp(c-p .. c+p)) as 3k bytes in RPW words (zero padded), so one patch row of
// Eq. 1 is one aligned 16- or 32-byte load and row clamping is an index clamp.
// ---------------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(256) prep_guides_kernel(const uint8_t* __restrict__ frames,
                                                          int H, int W,
                                                          uint32_t* __restrict__ rp) {
    using G = Geo<K>;
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t pix = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (pix >= npx) return;
    const size_t f = blockIdx.y;
    const int r = static_cast<int>(pix / W), c = static_cast<int>(pix % W);
    const uint8_t* img = frames + f * npx * 3;
    uint32_t words[G::RPW];
#pragma unroll
    for (int w = 0; w < G::RPW; ++w) words[w] = 0;
#pragma unroll
    for (int m = 0; m < K; ++m) {
        const int cc = clampi(c - G::P + m, 0, W - 1);
        const uint8_t* q = img + (static_cast<size_t>(r) * W + cc) * 3;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const int idx = 3 * m + ch;
            words[idx >> 2] |= static_cast<uint32_t>(q[ch]) << (8 * (idx & 3));
        }
    }
    uint4* dst = reinterpret_cast<uint4*>(rp + (f * npx + pix) * G::RPW);
#pragma unroll
    for (int v = 0; v < G::RPW / 4; ++v)
        dst[v] = make_uint4(words[4 * v], words[4 * v + 1], words[4 * v + 2], words[4 * v + 3]);
}

__global__ void __launch_bounds__(256) downsample_kernel(const uint8_t* __restrict__ in, int H,
                                                         int W, uint8_t* __restrict__ out) {
    const int h2 = (H + 1) / 2, w2 = (W + 1) / 2;
    const size_t n2 = static_cast<size_t>(h2) * w2;
    const size_t pix = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (pix >= n2) return;
    const size_t f = blockIdx.y;
    const int r = static_cast<int>(pix / w2), c = static_cast<int>(pix % w2);
    const uint8_t* img = in + f * static_cast<size_t>(H) * W * 3;
    const int r0 = 2 * r, r1 = min(2 * r + 1, H - 1), c0 = 2 * c, c1 = min(2 * c + 1, W - 1);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const int s = img[(static_cast<size_t>(r0) * W + c0) * 3 + ch] +
                      img[(static_cast<size_t>(r0) * W + c1) * 3 + ch] +
                      img[(static_cast<size_t>(r1) * W + c0) * 3 + ch] +
                      img[(static_cast<size_t>(r1) * W + c1) * 3 + ch];
        out[(f * n2 + pix) * 3 + ch] = static_cast<uint8_t>((s + 2) >> 2);
    }
}

__global__ void __launch_bounds__(256) style_rgbx_kernel(const uint8_t* __restrict__ in,
                                                         size_t n_px,
                                                         uint32_t* __restrict__ out) {
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_px) return;
    const uint8_t* q = in + 3 * i;
    out[i] = static_cast<uint32_t>(q[0]) | (static_cast<uint32_t>(q[1]) << 8) |
             (static_cast<uint32_t>(q[2]) << 16);
}

// ---------------------------------------------------------------------------------
// Patch distance (Eq. 1)
// ---------------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void load_row(const uint32_t* __restrict__ p,
                                         uint32_t (&out)[Geo<K>::NW]) {
    constexpr int NW = Geo<K>::NW;
    const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int v = 0; v < NW / 4; ++v) {
        const uint4 t = __ldg(q + v);
        out[4 * v] = t.x;
        out[4 * v + 1] = t.y;
        out[4 * v + 2] = t.z;
        out[4 * v + 3] = t.w;
    }
    constexpr int rem = NW % 4;
    if constexpr (rem == 2) {
        const uint2 t = __ldg(reinterpret_cast<const uint2*>(p + NW - 2));
        out[NW - 2] = t.x;
        out[NW - 1] = t.y;
    } else if constexpr (rem == 3) {
        const uint4 t = __ldg(q + NW / 4);
        out[NW - 3] = t.x;
        out[NW - 2] = t.y;
        out[NW - 1] = t.z;
    } else if constexpr (rem == 1) {
        out[NW - 1] = __ldg(p + NW - 1);
    }
}

template <int K>
struct TargetPatch {
    uint32_t w[K][Geo<K>::NW];  // the k rows of the target patch
    uint32_t row_e[K];          // sum of squares of each row
};

template <int K>
__device__ __forceinline__ void load_target(const uint32_t* __restrict__ rpt, int H, int W,
                                            int r, int c, TargetPatch<K>& t) {
    using G = Geo<K>;
#pragma unroll
    for (int a = 0; a < K; ++a) {
        const int rr = clampi(r - G::P + a, 0, H - 1);
        load_row<K>(rpt + (static_cast<size_t>(rr) * W + c) * G::RPW, t.w[a]);
        uint32_t e = 0;
#pragma unroll
        for (int w = 0; w < G::NW; ++w) e = __dp4a(t.w[a][w], t.w[a][w], e);
        t.row_e[a] = e;
    }
}

// Eq. 1 error of source patch u = (ur, uc) against target t, accumulated row by row as
// the exact non-negative terms |s_a|^2 + |t_a|^2 - 2 <s_a, t_a> (dp4a, four byte pairs
// per instruction).  Once the running sum reaches `bound` the candidate cannot be
// strictly better than the incumbent and its remaining rows are not loaded (returns
// false).  Otherwise returns true with the full error in *e.
template <int K>
__device__ __forceinline__ bool patch_error_below(const uint32_t* __restrict__ rps, int H, int W,
                                                  int ur, int uc, const TargetPatch<K>& t,
                                                  uint32_t bound, uint32_t* e) {
    using G = Geo<K>;
    uint32_t acc = 0;
#pragma unroll
    for (int a = 0; a < K; ++a) {
        const int rr = clampi(ur - G::P + a, 0, H - 1);
        uint32_t s[G::NW];
        load_row<K>(rps + (static_cast<size_t>(rr) * W + uc) * G::RPW, s);
        uint32_t dot = 0, ss = 0;
#pragma unroll
        for (int w = 0; w < G::NW; ++w) {
            dot = __dp4a(s[w], t.w[a][w], dot);
            ss = __dp4a(s[w], s[w], ss);
        }
        acc += ss + t.row_e[a] - 2u * dot;
        if (acc >= bound) return false;
    }
    *e = acc;
    return true;
}

struct TileCoord {
    int r, c;
};
__device__ __forceinline__ TileCoord tile_coord(int W) {
    const int tiles_x = (W + TILE_W - 1) / TILE_W;
    TileCoord t;
    t.c = static_cast<int>(blockIdx.x % tiles_x) * TILE_W + threadIdx.x;
    t.r = static_cast<int>(blockIdx.x / tiles_x) * TILE_H + threadIdx.y;
    return t;
}

// ---------------------------------------------------------------------------------
// Alg. 1: initial field and its error
// ---------------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(TILE_THREADS)
    nnf_init_kernel(const PairDesc* __restrict__ pairs, int pair0, int H, int W,
                    const uint32_t* __restrict__ rp, int mode,
                    const uint32_t* __restrict__ coarse_F, int Hc, int Wc,
                    const int32_t* __restrict__ user_init, uint32_t key0, uint32_t key1,
                    uint32_t level_word, uint32_t* __restrict__ F, uint32_t* __restrict__ E) {
    using G = Geo<K>;
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const int pl = blockIdx.y;
    const PairDesc pd = pairs[pair0 + pl];
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t x = static_cast<size_t>(tc.r) * W + tc.c;

    int ur, uc;
    if (mode == 0) {
        const uint4 u = philox4x32_10(make_uint4(static_cast<uint32_t>(x), pd.tag, level_word, 0u),
                                      key0, key1);
        ur = static_cast<int>(__umulhi(u.x, static_cast<uint32_t>(H)));
        uc = static_cast<int>(__umulhi(u.y, static_cast<uint32_t>(W)));
    } else if (mode == 1) {
        const uint32_t fc = coarse_F[static_cast<size_t>(pl) * Hc * Wc +
                                     static_cast<size_t>(tc.r >> 1) * Wc + (tc.c >> 1)];
        ur = clampi(2 * row_of(fc) + (tc.r & 1), 0, H - 1);
        uc = clampi(2 * col_of(fc) + (tc.c & 1), 0, W - 1);
    } else {
        ur = clampi(user_init[2 * x], 0, H - 1);
        uc = clampi(user_init[2 * x + 1], 0, W - 1);
    }
    TargetPatch<K> t;
    load_target<K>(rp + static_cast<size_t>(pd.tgt) * npx * G::RPW, H, W, tc.r, tc.c, t);
    uint32_t e = 0;
    patch_error_below<K>(rp + static_cast<size_t>(pd.src) * npx * G::RPW, H, W, ur, uc, t,
                         0xFFFFFFFFu, &e);
    F[static_cast<size_t>(pl) * npx + x] = pack_rc(ur, uc);
    E[static_cast<size_t>(pl) * npx + x] = e;
}

// Resident 256-thread blocks per SM the iteration kernel is compiled for: larger
// patches hold more target words in registers.
template <int K>
struct IterOccupancy {
    static constexpr int value = K <= 3 ? 6 : K <= 5 ? FB_ITER_MIN_BLOCKS : K <= 7 ? 3 : 2;
};

// ---------------------------------------------------------------------------------
// Alg. 1: one Jacobi iteration (Sec. 3.2 parallel update).  Reads the snapshot
// (Fp, Ep), writes (Fn, En).  Per pixel: propagation from the four neighbours in the
// order (-1,0), (1,0), (0,-1), (0,1), then random search around the running best with
// radius r0 >> t; strict improvement only.  A candidate equal to the running best is
// skipped: its error equals the incumbent's, so it could not win.
// ---------------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(TILE_THREADS, IterOccupancy<K>::value * 256 / TILE_THREADS)
    nnf_iter_kernel(const PairDesc* __restrict__ pairs, int pair0, int H, int W,
                    const uint32_t* __restrict__ rp, int r0,
                    uint32_t key0, uint32_t key1, uint32_t ctr_word,
                    const uint32_t* __restrict__ Fp, const uint32_t* __restrict__ Ep,
                    uint32_t* __restrict__ Fn, uint32_t* __restrict__ En) {
    using G = Geo<K>;
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const int r = tc.r, c = tc.c;
    const int pl = blockIdx.y;
    const PairDesc pd = pairs[pair0 + pl];
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t x = static_cast<size_t>(r) * W + c;
    const uint32_t* __restrict__ rps = rp + static_cast<size_t>(pd.src) * npx * G::RPW;
    const uint32_t* __restrict__ Fpp = Fp + static_cast<size_t>(pl) * npx;

    TargetPatch<K> t;
    load_target<K>(rp + static_cast<size_t>(pd.tgt) * npx * G::RPW, H, W, r, c, t);

    uint32_t bf = Fpp[x];
    uint32_t be = Ep[static_cast<size_t>(pl) * npx + x];

    auto consider = [&](int cr, int cc) {
        const uint32_t f = pack_rc(cr, cc);
        if (f == bf) return;
        uint32_t e;
        if (patch_error_below<K>(rps, H, W, cr, cc, t, be, &e)) {
            be = e;
            bf = f;
        }
    };

    // Propagation: F'(x) = F(x + d) - d.
    if (r > 0) {
        const uint32_t f = Fpp[x - W];
        consider(min(row_of(f) + 1, H - 1), col_of(f));
    }
    if (r < H - 1) {
        const uint32_t f = Fpp[x + W];
        consider(max(row_of(f) - 1, 0), col_of(f));
    }
    if (c > 0) {
        const uint32_t f = Fpp[x - 1];
        consider(row_of(f), min(col_of(f) + 1, W - 1));
    }
    if (c < W - 1) {
        const uint32_t f = Fpp[x + 1];
        consider(row_of(f), max(col_of(f) - 1, 0));
    }

    // Random search: F'(x) = F(x) + U[-r, r]^2, r = r0 >> t, t = 0, 1, ... while r >= 1.
    uint4 u = make_uint4(0u, 0u, 0u, 0u);
    for (int tt = 0; (r0 >> tt) >= 1; ++tt) {
        const int rad = r0 >> tt;
        if ((tt & 1) == 0)
            u = philox4x32_10(make_uint4(static_cast<uint32_t>(x), pd.tag,
                                         ctr_word | static_cast<uint32_t>(tt >> 1), 0u),
                              key0, key1);
        const uint32_t span = static_cast<uint32_t>(2 * rad + 1);
        const int dr = static_cast<int>(__umulhi((tt & 1) ? u.z : u.x, span)) - rad;
        const int dc = static_cast<int>(__umulhi((tt & 1) ? u.w : u.y, span)) - rad;
        consider(clampi(row_of(bf) + dr, 0, H - 1), clampi(col_of(bf) + dc, 0, W - 1));
    }

    Fn[static_cast<size_t>(pl) * npx + x] = bf;
    En[static_cast<size_t>(pl) * npx + x] = be;
}

__global__ void __launch_bounds__(256) nnf_unpack_kernel(const uint32_t* __restrict__ F,
                                                         const uint32_t* __restrict__ E,
                                                         size_t npx, int32_t* __restrict__ nnf,
                                                         uint32_t* __restrict__ err) {
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= npx) return;
    const uint32_t f = F[i];
    nnf[2 * i] = row_of(f);
    nnf[2 * i + 1] = col_of(f);
    if (err) err[i] = E[i];
}

__global__ void __launch_bounds__(256) nnf_pack_kernel(const int32_t* __restrict__ nnf, int H,
                                                       int W, uint32_t* __restrict__ F) {
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= npx) return;
    F[i] = pack_rc(clampi(nnf[2 * i], 0, H - 1), clampi(nnf[2 * i + 1], 0, W - 1));
}

// ---------------------------------------------------------------------------------
// Alg. 2 remap fused with the output combination.  For output frame i:
//   num(x) = self_w * k^2 * S_self(x) + sum_pairs weight * V_pair(x)
//   V(x)   = sum_{q in k x k around x} S(clamp(F(q^) - (q^ - x))),  q^ = clamp(q)
//   out(x) = num(x) / den        (one IEEE division per channel)
// ---------------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(TILE_THREADS)
    combine_kernel(const JobDesc* __restrict__ jobs, int job0, const PairDesc* __restrict__ pairs,
                   int pair0, const uint32_t* __restrict__ F, const uint32_t* __restrict__ styles,
                   int H, int W, float* __restrict__ out) {
    constexpr int P = K / 2;
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const int r = tc.r, c = tc.c;
    const JobDesc job = jobs[job0 + blockIdx.y];
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t x = static_cast<size_t>(r) * W + c;

    uint32_t a0 = 0, a1 = 0, a2 = 0;
    if (job.self_style >= 0) {
        const uint32_t s = __ldg(styles + static_cast<size_t>(job.self_style) * npx + x);
        const uint32_t w = job.self_w * static_cast<uint32_t>(K * K);
        a0 = w * (s & 0xFFu);
        a1 = w * ((s >> 8) & 0xFFu);
        a2 = w * ((s >> 16) & 0xFFu);
    }
    for (int p = 0; p < job.n_pairs; ++p) {
        const int gp = job.first_pair + p;
        const PairDesc pd = pairs[gp];
        const uint32_t* __restrict__ Fq = F + static_cast<size_t>(gp - pair0) * npx;
        const uint32_t* __restrict__ S = styles + static_cast<size_t>(pd.style) * npx;
        uint32_t v0 = 0, v1 = 0, v2 = 0;
#pragma unroll
        for (int a = -P; a <= P; ++a) {
            const int qr = clampi(r + a, 0, H - 1);
#pragma unroll
            for (int b = -P; b <= P; ++b) {
                const int qc = clampi(c + b, 0, W - 1);
                const uint32_t f = __ldg(Fq + static_cast<size_t>(qr) * W + qc);
                const int sr = clampi(row_of(f) - (qr - r), 0, H - 1);
                const int sc = clampi(col_of(f) - (qc - c), 0, W - 1);
                const uint32_t s = __ldg(S + static_cast<size_t>(sr) * W + sc);
                v0 += s & 0xFFu;
                v1 += (s >> 8) & 0xFFu;
                v2 += (s >> 16) & 0xFFu;
            }
        }
        a0 += pd.weight * v0;
        a1 += pd.weight * v1;
        a2 += pd.weight * v2;
    }
    const float den = __uint2float_rn(job.den);
    float* o = out + (static_cast<size_t>(job.out_frame) * npx + x) * 3;
    o[0] = __fdiv_rn(__uint2float_rn(a0), den);
    o[1] = __fdiv_rn(__uint2float_rn(a1), den);
    o[2] = __fdiv_rn(__uint2float_rn(a2), den);
}

inline dim3 tile_grid(int H, int W, int n) {
    const unsigned tiles = static_cast<unsigned>(((W + TILE_W - 1) / TILE_W) *
                                                 ((H + TILE_H - 1) / TILE_H));
    return dim3(tiles, static_cast<unsigned>(n), 1);
}
inline unsigned blocks_for(size_t n, unsigned per) {
    return static_cast<unsigned>((n + per - 1) / per);
}

#define FB_DISPATCH_K(k, CALL)                \
    switch (k) {                              \
        case 3: { constexpr int KK = 3; CALL; } break; \
        case 5: { constexpr int KK = 5; CALL; } break; \
        case 7: { constexpr int KK = 7; CALL; } break; \
        case 9: { constexpr int KK = 9; CALL; } break; \
        default: return cudaErrorInvalidValue;         \
    }

}  // namespace

cudaError_t launch_prep_guides(int k, const uint8_t* frames, int n_frames, int H, int W,
                               uint32_t* rp, cudaStream_t st) {
    if (n_frames <= 0) return cudaSuccess;
    const dim3 grid(blocks_for(static_cast<size_t>(H) * W, 256), static_cast<unsigned>(n_frames));
    FB_DISPATCH_K(k, (prep_guides_kernel<KK><<<grid, 256, 0, st>>>(frames, H, W, rp)));
    return cudaGetLastError();
}

cudaError_t launch_downsample(const uint8_t* in, int n_frames, int H, int W, uint8_t* out,
                              cudaStream_t st) {
    if (n_frames <= 0) return cudaSuccess;
    const size_t n2 = static_cast<size_t>((H + 1) / 2) * ((W + 1) / 2);
    downsample_kernel<<<dim3(blocks_for(n2, 256), static_cast<unsigned>(n_frames)), 256, 0, st>>>(
        in, H, W, out);
    return cudaGetLastError();
}

cudaError_t launch_style_rgbx(const uint8_t* in, size_t n_px, uint32_t* out, cudaStream_t st) {
    if (n_px == 0) return cudaSuccess;
    style_rgbx_kernel<<<blocks_for(n_px, 256), 256, 0, st>>>(in, n_px, out);
    return cudaGetLastError();
}

cudaError_t launch_nnf_init(int k, const PairDesc* pairs, int pair0, int n_pairs,
                            const LevelGeom& g, int mode, const uint32_t* coarse_F, int Hc,
                            int Wc, const int32_t* user_init, uint64_t seed, int level,
                            uint32_t* F, uint32_t* E, cudaStream_t st) {
    if (n_pairs <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(g.H, g.W, n_pairs);
    const dim3 block(TILE_W, TILE_H);
    const uint32_t level_word = static_cast<uint32_t>(level) << 24;
    FB_DISPATCH_K(k, (nnf_init_kernel<KK><<<grid, block, 0, st>>>(
                         pairs, pair0, g.H, g.W, g.rp, mode, coarse_F, Hc, Wc, user_init,
                         static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32),
                         level_word, F, E)));
    return cudaGetLastError();
}

cudaError_t launch_nnf_iter(int k, const PairDesc* pairs, int pair0, int n_pairs,
                            const LevelGeom& g, int r0, uint64_t seed, int level, int it,
                            const uint32_t* Fp, const uint32_t* Ep, uint32_t* Fn, uint32_t* En,
                            cudaStream_t st) {
    if (n_pairs <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(g.H, g.W, n_pairs);
    const dim3 block(TILE_W, TILE_H);
    const uint32_t ctr_word = (static_cast<uint32_t>(level) << 24) |
                              (static_cast<uint32_t>(it + 1) << 8);
    FB_DISPATCH_K(k, (nnf_iter_kernel<KK><<<grid, block, 0, st>>>(
                         pairs, pair0, g.H, g.W, g.rp, r0,
                         static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32),
                         ctr_word, Fp, Ep, Fn, En)));
    return cudaGetLastError();
}

cudaError_t launch_nnf_unpack(const uint32_t* F, const uint32_t* E, size_t npx, int32_t* nnf_out,
                              uint32_t* err_out, cudaStream_t st) {
    nnf_unpack_kernel<<<blocks_for(npx, 256), 256, 0, st>>>(F, E, npx, nnf_out, err_out);
    return cudaGetLastError();
}

cudaError_t launch_nnf_pack(const int32_t* nnf, int H, int W, uint32_t* F, cudaStream_t st) {
    nnf_pack_kernel<<<blocks_for(static_cast<size_t>(H) * W, 256), 256, 0, st>>>(nnf, H, W, F);
    return cudaGetLastError();
}

cudaError_t launch_combine(int k, const JobDesc* jobs, int job0, int n_jobs,
                           const PairDesc* pairs, int pair0, const uint32_t* F,
                           const uint32_t* styles, int H, int W, float* out, cudaStream_t st) {
    if (n_jobs <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(H, W, n_jobs);
    const dim3 block(TILE_W, TILE_H);
    FB_DISPATCH_K(k, (combine_kernel<KK><<<grid, block, 0, st>>>(jobs, job0, pairs, pair0, F,
                                                                 styles, H, W, out)));
    return cudaGetLastError();
}

}  // namespace fb
