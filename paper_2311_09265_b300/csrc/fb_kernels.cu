// fb_kernels.cu -- sm_103a kernels of the FastBlend hot path (arXiv 2311.09265).
//
//   prep_guides   guide frame -> one patch record per pixel (Eq. 1 operands)
//   downsample    one pyramid step (Alg. 1, "resize images")
//   style_rgbx    style frame -> 4-byte pixels for single-load gathers
//   nnf_init      random / upsampled / user initial field and its Eq. 1 error
//   nnf_iter      one Jacobi iteration of Alg. 1: propagation + random search
//   combine       Alg. 2 remap of every pair of an output frame, fused with the
//                 Eq. 2 window sum (or the Sec. 3.5.2 keyframe weights) and the
//                 final division
//
// Everything on the NNF path is integer: Eq. 1 is evaluated one 32-byte sector of the
// candidate's patch record at a time as |s|^2 + |t|^2 - 2 <s, t> with dp4a, which is
// exactly the clamp-to-edge sum of squared byte differences; a candidate stops loading
// once an exact lower bound or its running sum reaches the incumbent's error.
#include "fb_internal.h"

namespace fb {
namespace {

#ifndef FB_ITER_MIN_BLOCKS
#define FB_ITER_MIN_BLOCKS 5  // resident 256-thread blocks per SM the iteration kernel is built for
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

// Patch record of a guide pixel u (the acceleration structure of the NNF search):
//   word 0      sum of channel 0 | sum of channel 1 << 16 over the clamped k x k patch
//   word 1      sum of channel 2
//   words 2..   the 3k^2 bytes of the clamped patch, row-major, RGB, zero padded
// padded to whole 32-byte sectors, so that one 256-bit load fetches one sector.
template <int K>
struct Rec {
    static constexpr int P = K / 2;
    static constexpr int PATCH_BYTES = 3 * K * K;
    static constexpr int PATCH_WORDS = (PATCH_BYTES + 3) / 4;
    static constexpr int HEAD = 2;
    static constexpr int WORDS = (HEAD + PATCH_WORDS + 7) / 8 * 8;
    static constexpr int SECTORS = WORDS / 8;
};

__device__ __forceinline__ void ld256_nc(const uint32_t* p, uint32_t (&w)[8]) {
    asm volatile("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                   "=r"(w[6]), "=r"(w[7])
                 : "l"(p));
}

// ---------------------------------------------------------------------------------
// Guide preparation: one patch record per pixel.
// ---------------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(256) prep_guides_kernel(const uint8_t* __restrict__ frames,
                                                          int H, int W,
                                                          uint32_t* __restrict__ rec) {
    using R = Rec<K>;
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t pix = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (pix >= npx) return;
    const size_t f = blockIdx.y;
    const int r = static_cast<int>(pix / W), c = static_cast<int>(pix % W);
    const uint8_t* img = frames + f * npx * 3;

    uint32_t words[R::WORDS];
#pragma unroll
    for (int w = 0; w < R::WORDS; ++w) words[w] = 0;
    uint32_t sum[3] = {0u, 0u, 0u};
#pragma unroll
    for (int a = 0; a < K; ++a) {
        const int rr = clampi(r - R::P + a, 0, H - 1);
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const int cc = clampi(c - R::P + b, 0, W - 1);
            const uint8_t* q = img + (static_cast<size_t>(rr) * W + cc) * 3;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const uint32_t v = q[ch];
                const int idx = 3 * (a * K + b) + ch;
                words[R::HEAD + (idx >> 2)] |= v << (8 * (idx & 3));
                sum[ch] += v;
            }
        }
    }
    words[0] = sum[0] | (sum[1] << 16);
    words[1] = sum[2];
    uint4* dst = reinterpret_cast<uint4*>(rec + (f * npx + pix) * R::WORDS);
#pragma unroll
    for (int v = 0; v < R::WORDS / 4; ++v)
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
// Patch distance (Eq. 1) against a target record held in shared memory
// ---------------------------------------------------------------------------------
// Each thread keeps its own target record in shared memory (registers stay free for
// occupancy): sector s as two 16-byte halves, plane-major so a warp's accesses are
// contiguous, plus each sector's sum of squares over its patch words.
template <int K>
struct TargetSmem {
    uint4* w;      // [SECTORS][2][TILE_THREADS]
    uint32_t* e;   // [SECTORS][TILE_THREADS]
    int tid;
    uint32_t sum01, sum2;  // channel sums of the target patch
    __device__ __forceinline__ uint4 half(int s, int h) const {
        return w[(s * 2 + h) * TILE_THREADS + tid];
    }
    __device__ __forceinline__ uint32_t energy(int s) const { return e[s * TILE_THREADS + tid]; }
};

template <int K>
constexpr size_t target_smem_bytes() {
    return static_cast<size_t>(Rec<K>::SECTORS) * TILE_THREADS * (2 * sizeof(uint4) + sizeof(uint32_t));
}

template <int K>
__device__ __forceinline__ TargetSmem<K> stage_target(const uint32_t* __restrict__ rec_t,
                                                      size_t xpix, unsigned char* smem) {
    using R = Rec<K>;
    TargetSmem<K> t;
    t.w = reinterpret_cast<uint4*>(smem);
    t.e = reinterpret_cast<uint32_t*>(smem + static_cast<size_t>(R::SECTORS) * 2 * TILE_THREADS * sizeof(uint4));
    t.tid = threadIdx.y * TILE_W + threadIdx.x;
    const uint32_t* p = rec_t + xpix * R::WORDS;
#pragma unroll
    for (int s = 0; s < R::SECTORS; ++s) {
        uint32_t w[8];
        ld256_nc(p + 8 * s, w);
        if (s == 0) {
            t.sum01 = w[0];
            t.sum2 = w[1];
        }
        uint32_t e = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int wi = 8 * s + q;
            if (wi >= R::HEAD && wi < R::HEAD + R::PATCH_WORDS) e = __dp4a(w[q], w[q], e);
        }
        t.w[(s * 2 + 0) * TILE_THREADS + t.tid] = make_uint4(w[0], w[1], w[2], w[3]);
        t.w[(s * 2 + 1) * TILE_THREADS + t.tid] = make_uint4(w[4], w[5], w[6], w[7]);
        t.e[s * TILE_THREADS + t.tid] = e;
    }
    return t;
}

// Eq. 1 error of the source patch whose record starts at `src`, against target t.
// The error is accumulated one 32-byte sector at a time as the exact non-negative sum
// |s|^2 + |t|^2 - 2 <s, t> over that sector's patch bytes (dp4a, four byte pairs per
// instruction).  Rejection is exact and only skips work:
//   * with `use_bound`, the first sector's channel sums give the Cauchy-Schwarz bound
//     k^2 * SSD >= sum_ch (sum_s,ch - sum_t,ch)^2, so a candidate whose bound reaches
//     `bound` cannot be strictly better than the incumbent;
//   * after each sector, a running sum that reaches `bound` stops the work.
// The loads of CHUNK consecutive sectors are issued together before any is used:
// CHUNK = 1 saves bytes for candidates that are usually rejected at once, a larger
// CHUNK saves dependent round trips for candidates that usually need every sector.
// Returns true, with the full error in *e, only when the error is below `bound`.
template <int K, int CHUNK>
__device__ __forceinline__ bool patch_error_below(const uint32_t* __restrict__ src,
                                                  const TargetSmem<K>& t, uint32_t bound,
                                                  bool use_bound, uint32_t* e) {
    using R = Rec<K>;
    uint32_t acc = 0;
#pragma unroll
    for (int s0 = 0; s0 < R::SECTORS; s0 += CHUNK) {
        uint32_t w[CHUNK][8];
#pragma unroll
        for (int j = 0; j < CHUNK; ++j)
            if (s0 + j < R::SECTORS) ld256_nc(src + 8 * (s0 + j), w[j]);
#pragma unroll
        for (int j = 0; j < CHUNK; ++j) {
            const int s = s0 + j;
            if (s >= R::SECTORS) break;
            if (s == 0 && use_bound) {
                const int d0 = static_cast<int>(w[j][0] & 0xFFFFu) - static_cast<int>(t.sum01 & 0xFFFFu);
                const int d1 = static_cast<int>(w[j][0] >> 16) - static_cast<int>(t.sum01 >> 16);
                const int d2 = static_cast<int>(w[j][1]) - static_cast<int>(t.sum2);
                const uint64_t lb = static_cast<uint64_t>(d0 * d0) + static_cast<uint64_t>(d1 * d1) +
                                    static_cast<uint64_t>(d2 * d2);
                if (lb >= static_cast<uint64_t>(bound) * (K * K)) return false;
            }
            const uint4 ta = t.half(s, 0), tb = t.half(s, 1);
            const uint32_t tv[8] = {ta.x, ta.y, ta.z, ta.w, tb.x, tb.y, tb.z, tb.w};
            uint32_t dot = 0, ss = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int wi = 8 * s + q;
                if (wi >= R::HEAD && wi < R::HEAD + R::PATCH_WORDS) {
                    dot = __dp4a(w[j][q], tv[q], dot);
                    ss = __dp4a(w[j][q], w[j][q], ss);
                }
            }
            acc += ss + t.energy(s) - 2u * dot;
            if (acc >= bound) return false;
        }
    }
    *e = acc;
    return true;
}

#ifndef FB_PROP_CHUNK
#define FB_PROP_CHUNK 4       // sectors loaded together for propagation candidates
#endif
#ifndef FB_NEAR_CHUNK
#define FB_NEAR_CHUNK 4       // ... for random-search candidates with radius <= FB_NEAR_RADIUS
#endif
#ifndef FB_FAR_CHUNK
#define FB_FAR_CHUNK 1        // ... for random-search candidates with a larger radius
#endif
#ifndef FB_NEAR_RADIUS
#define FB_NEAR_RADIUS 16
#endif
template <int K, int C>
struct Chunk {
    static constexpr int value = C < Rec<K>::SECTORS ? C : Rec<K>::SECTORS;
};

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
                    const uint32_t* __restrict__ rec, int mode,
                    const uint32_t* __restrict__ coarse_F, int Hc, int Wc,
                    const int32_t* __restrict__ user_init, uint32_t key0, uint32_t key1,
                    uint32_t level_word, uint32_t* __restrict__ F, uint32_t* __restrict__ E) {
    using R = Rec<K>;
    extern __shared__ __align__(16) unsigned char smem[];
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const int pl = blockIdx.y;
    const PairDesc pd = pairs[pair0 + pl];
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t x = static_cast<size_t>(tc.r) * W + tc.c;
    const TargetSmem<K> t =
        stage_target<K>(rec + static_cast<size_t>(pd.tgt) * npx * R::WORDS, x, smem);

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
    const uint32_t* recs = rec + static_cast<size_t>(pd.src) * npx * R::WORDS;
    uint32_t e = 0;
    patch_error_below<K, Chunk<K, 4>::value>(recs + (static_cast<size_t>(ur) * W + uc) * R::WORDS,
                                             t, 0xFFFFFFFFu, false, &e);
    F[static_cast<size_t>(pl) * npx + x] = pack_rc(ur, uc);
    E[static_cast<size_t>(pl) * npx + x] = e;
}

// ---------------------------------------------------------------------------------
// Alg. 1: one Jacobi iteration (Sec. 3.2 parallel update).  Reads the snapshot
// (Fp, Ep), writes (Fn, En).  Per pixel: propagation from the four neighbours in the
// order (-1,0), (1,0), (0,-1), (0,1), then random search around the running best with
// radius r0 >> t; strict improvement only.  A candidate equal to the running best is
// skipped: its error equals the incumbent's, so it could not win.
// ---------------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(TILE_THREADS, FB_ITER_MIN_BLOCKS * 256 / TILE_THREADS)
    nnf_iter_kernel(const PairDesc* __restrict__ pairs, int pair0, int H, int W,
                    const uint32_t* __restrict__ rec, int r0,
                    uint32_t key0, uint32_t key1, uint32_t ctr_word,
                    const uint32_t* __restrict__ Fp, const uint32_t* __restrict__ Ep,
                    uint32_t* __restrict__ Fn, uint32_t* __restrict__ En) {
    using R = Rec<K>;
    extern __shared__ __align__(16) unsigned char smem[];
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const int r = tc.r, c = tc.c;
    const int pl = blockIdx.y;
    const PairDesc pd = pairs[pair0 + pl];
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t x = static_cast<size_t>(r) * W + c;
    const uint32_t* __restrict__ recs = rec + static_cast<size_t>(pd.src) * npx * R::WORDS;
    const uint32_t* __restrict__ Fpp = Fp + static_cast<size_t>(pl) * npx;
    const TargetSmem<K> t =
        stage_target<K>(rec + static_cast<size_t>(pd.tgt) * npx * R::WORDS, x, smem);

    uint32_t bf = Fpp[x];
    uint32_t be = Ep[static_cast<size_t>(pl) * npx + x];

    auto consider = [&](int cr, int cc, auto chunk) {
        const uint32_t f = pack_rc(cr, cc);
        if (f == bf) return;
        uint32_t e;
        if (patch_error_below<K, decltype(chunk)::value>(
                recs + (static_cast<size_t>(cr) * W + cc) * R::WORDS, t, be, true, &e)) {
            be = e;
            bf = f;
        }
    };
    const Chunk<K, FB_PROP_CHUNK> prop_chunk;
    const Chunk<K, FB_NEAR_CHUNK> near_chunk;
    const Chunk<K, FB_FAR_CHUNK> far_chunk;

    // Propagation: F'(x) = F(x + d) - d.
    if (r > 0) {
        const uint32_t f = Fpp[x - W];
        consider(min(row_of(f) + 1, H - 1), col_of(f), prop_chunk);
    }
    if (r < H - 1) {
        const uint32_t f = Fpp[x + W];
        consider(max(row_of(f) - 1, 0), col_of(f), prop_chunk);
    }
    if (c > 0) {
        const uint32_t f = Fpp[x - 1];
        consider(row_of(f), min(col_of(f) + 1, W - 1), prop_chunk);
    }
    if (c < W - 1) {
        const uint32_t f = Fpp[x + 1];
        consider(row_of(f), max(col_of(f) - 1, 0), prop_chunk);
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
        const int cr = clampi(row_of(bf) + dr, 0, H - 1), cc = clampi(col_of(bf) + dc, 0, W - 1);
        if (rad <= FB_NEAR_RADIUS)
            consider(cr, cc, near_chunk);
        else
            consider(cr, cc, far_chunk);
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

// Opt a kernel in to the dynamic shared memory it needs (once per kernel).
template <class Kernel>
inline void prepare_smem(Kernel kernel, size_t bytes) {
    if (bytes > 48 * 1024)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(bytes));
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
                               uint32_t* rec, cudaStream_t st) {
    if (n_frames <= 0) return cudaSuccess;
    const dim3 grid(blocks_for(static_cast<size_t>(H) * W, 256), static_cast<unsigned>(n_frames));
    FB_DISPATCH_K(k, (prep_guides_kernel<KK><<<grid, 256, 0, st>>>(frames, H, W, rec)));
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
    FB_DISPATCH_K(k, (prepare_smem(nnf_init_kernel<KK>, target_smem_bytes<KK>()),
                      nnf_init_kernel<KK><<<grid, block, target_smem_bytes<KK>(), st>>>(
                         pairs, pair0, g.H, g.W, g.rec, mode, coarse_F, Hc, Wc, user_init,
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
    FB_DISPATCH_K(k, (prepare_smem(nnf_iter_kernel<KK>, target_smem_bytes<KK>()),
                      nnf_iter_kernel<KK><<<grid, block, target_smem_bytes<KK>(), st>>>(
                         pairs, pair0, g.H, g.W, g.rec, r0,
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
