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
#include "fb_device.cuh"

namespace fb {
namespace {

using namespace dev;

#ifndef FB_TILE_H
#define FB_TILE_H 4
#endif

#ifndef FB_TILE_W
#define FB_TILE_W 32
#endif
constexpr int TILE_W = FB_TILE_W;
constexpr int TILE_H = FB_TILE_H;
constexpr int TILE_THREADS = TILE_W * TILE_H;

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

// The paired k = 5 layout: thread (q, c) of frame f writes the 32-byte slot holding the
// row patches of rows clamp(2q - 2) and clamp(2q - 1) at column c.
__global__ void __launch_bounds__(256) prep_guides_paired_kernel(const uint8_t* __restrict__ frames,
                                                                 int H, int W,
                                                                 uint32_t* __restrict__ rp) {
    constexpr int K = 5, P = 2;
    const size_t n_slots = static_cast<size_t>(rowpatch_pair_rows(H)) * W;
    const size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= n_slots) return;
    const size_t f = blockIdx.y;
    const int q = static_cast<int>(idx / W), c = static_cast<int>(idx % W);
    const uint8_t* img = frames + f * static_cast<size_t>(H) * W * 3;
    uint32_t words[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) words[w] = 0;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int r = clampi(2 * q - 2 + half, 0, H - 1);
#pragma unroll
        for (int m = 0; m < K; ++m) {
            const int cc = clampi(c - P + m, 0, W - 1);
            const uint8_t* px = img + (static_cast<size_t>(r) * W + cc) * 3;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const int b = 3 * m + ch;
                words[4 * half + (b >> 2)] |= static_cast<uint32_t>(px[ch]) << (8 * (b & 3));
            }
        }
    }
    uint4* dst = reinterpret_cast<uint4*>(rp + f * rowpatch_frame_words(K, H, W) + idx * 8);
    dst[0] = make_uint4(words[0], words[1], words[2], words[3]);
    dst[1] = make_uint4(words[4], words[5], words[6], words[7]);
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
// ---------------------------------------------------------------------------------
// Per-call kernels (one pair table / job table per call)
// ---------------------------------------------------------------------------------
struct TileCoord {
    int r, c;
};
// Checked builds: pair index q (relative to the launch's first pair) of a chain neighbour
// or partner of launch pair pl is one of the launch's gridDim.y pairs.
__device__ __forceinline__ bool in_launch(int q, int pl) {
    return FB_CHECK(q >= 0 && q < static_cast<int>(gridDim.y), FB_CHECK_TABLE, pl, q);
}

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
    init_pixel<K>(frame_rows<K>(rp, pd.src, H, W), frame_rows<K>(rp, pd.tgt, H, W), H, W, tc.r,
                  tc.c, pd.tag, mode,
                  coarse_F ? coarse_F + static_cast<size_t>(pl) * Hc * Wc : nullptr, Hc, Wc,
                  user_init ? user_init + static_cast<size_t>(pl) * npx * 2 : nullptr, key0, key1,
                  level_word, F + static_cast<size_t>(pl) * npx, E + static_cast<size_t>(pl) * npx);
}

// Resident warps per SM the iteration kernels are compiled for (launch bounds: that many
// warps in blocks of TILE_THREADS).  Larger patches hold more target words in registers
// (k = 7: 28 warps fit 72 registers without spilling; 24 warps at 80 are slower, 32 at 64
// spill).
#ifndef FB_ITER_WARPS5
#define FB_ITER_WARPS5 40
#endif
#ifndef FB_ITER_WARPS7
#define FB_ITER_WARPS7 28
#endif
template <int K>
struct IterWarps {
    static constexpr int value = K <= 3 ? 48 : K <= 5 ? FB_ITER_WARPS5 : K <= 7 ? FB_ITER_WARPS7 : 16;
};
// Blocks of TILE_THREADS threads that hold `warps` warps.
template <int warps>
struct MinBlocks {
    static constexpr int value = warps * 32 / TILE_THREADS > 0 ? warps * 32 / TILE_THREADS : 1;
};

// ---------------------------------------------------------------------------------
// Alg. 1: one Jacobi iteration (Sec. 3.2 parallel update).  Reads the snapshot
// (Fp, Ep), writes (Fn, En).  Per pixel: propagation from the four neighbours in the
// order (-1,0), (1,0), (0,-1), (0,1), then random search around the running best with
// radius r0 >> t; strict improvement only.  A candidate equal to the running best is
// skipped: its error equals the incumbent's, so it could not win.
// ---------------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(TILE_THREADS, MinBlocks<IterWarps<K>::value>::value)
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
    const uint32_t* __restrict__ rps = frame_rows<K>(rp, pd.src, H, W);
    const uint32_t* __restrict__ Fpp = Fp + static_cast<size_t>(pl) * npx;

    iterate_pixel<K>(rps, frame_rows<K>(rp, pd.tgt, H, W), H, W, r, c, pd.tag, r0,
                     key0, key1, ctr_word, Fpp, Ep + static_cast<size_t>(pl) * npx,
                     Fn + static_cast<size_t>(pl) * npx, En + static_cast<size_t>(pl) * npx);
}

// Tracking (Sec. 3.5.1): as nnf_iter_kernel, plus the matches of the pair's chain
// neighbours (pairs pad[0] / pad[1] of the launch, -1 for none) at the same pixel.
template <int K>
__global__ void __launch_bounds__(TILE_THREADS, MinBlocks<IterWarps<K>::value>::value)
    nnf_iter_track_kernel(const PairDesc* __restrict__ pairs, int pair0, int H, int W,
                          const uint32_t* __restrict__ rp, int r0, uint32_t key0, uint32_t key1,
                          uint32_t ctr_word, const uint32_t* __restrict__ Fp,
                          const uint32_t* __restrict__ Ep, uint32_t* __restrict__ Fn,
                          uint32_t* __restrict__ En) {
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const int pl = blockIdx.y;
    const PairDesc pd = pairs[pair0 + pl];
    const size_t npx = static_cast<size_t>(H) * W;
    const uint32_t* prev = pd.pad[0] >= 0 && in_launch(pd.pad[0] - pair0, pl)
                               ? Fp + static_cast<size_t>(pd.pad[0] - pair0) * npx : nullptr;
    const uint32_t* next = pd.pad[1] >= 0 && in_launch(pd.pad[1] - pair0, pl)
                               ? Fp + static_cast<size_t>(pd.pad[1] - pair0) * npx : nullptr;
    iterate_pixel_tracking<K>(frame_rows<K>(rp, pd.src, H, W), frame_rows<K>(rp, pd.tgt, H, W), H, W, tc.r,
                              tc.c, pd.tag, r0, key0, key1, ctr_word, Fp + static_cast<size_t>(pl) * npx,
                              Ep + static_cast<size_t>(pl) * npx, prev, next,
                              Fn + static_cast<size_t>(pl) * npx, En + static_cast<size_t>(pl) * npx);
}

// ---------------------------------------------------------------------------------
// Improved loss of Sec. 3.4 ("balanced mode").  Per iteration: S^ of every pair from its
// current field (shat_kernel, then the guide row-patch layout), the incumbent's loss
// against the new S^ (energy_balanced_kernel), then the Jacobi step under that loss.
// ---------------------------------------------------------------------------------
// S^(x) = the Alg. 2 remap of the pair's source style through F, rounded half up to 8 bits.
template <int K>
__global__ void __launch_bounds__(TILE_THREADS)
    shat_kernel(const PairDesc* __restrict__ pairs, int pair0, int H, int W,
                const uint32_t* __restrict__ F, const uint32_t* __restrict__ styles,
                uint8_t* __restrict__ shat) {
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const int pl = blockIdx.y;
    const PairDesc pd = pairs[pair0 + pl];
    const size_t npx = static_cast<size_t>(H) * W;
    uint32_t v0, v1, v2;
    remap_votes<K>(F + static_cast<size_t>(pl) * npx, styles + static_cast<size_t>(pd.style) * npx, H,
                   W, tc.r, tc.c, v0, v1, v2);
    constexpr uint32_t kk = static_cast<uint32_t>(K * K);
    uint8_t* o = shat + (static_cast<size_t>(pl) * npx + static_cast<size_t>(tc.r) * W + tc.c) * 3;
    o[0] = static_cast<uint8_t>((v0 + kk / 2) / kk);
    o[1] = static_cast<uint8_t>((v1 + kk / 2) / kk);
    o[2] = static_cast<uint8_t>((v2 + kk / 2) / kk);
}

// Accurate mode of Sec. 3.4: Tbar of output frame job.out_frame = the Eq. 2 numerator of
// the current fields (k^2 S_self + sum of the pairs' votes) over k^2 c, rounded half up.
template <int K>
__global__ void __launch_bounds__(TILE_THREADS)
    tbar_kernel(const JobDesc* __restrict__ jobs, int job0, const PairDesc* __restrict__ pairs,
                int pair0, const uint32_t* __restrict__ F, const uint32_t* __restrict__ styles, int H,
                int W, uint8_t* __restrict__ out) {
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const JobDesc job = jobs[job0 + blockIdx.y];
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t x = static_cast<size_t>(tc.r) * W + tc.c;
    constexpr uint32_t kk = static_cast<uint32_t>(K * K);
    const uint32_t s = __ldg(styles + static_cast<size_t>(job.self_style) * npx + x);
    uint32_t a0 = kk * (s & 0xFFu), a1 = kk * ((s >> 8) & 0xFFu), a2 = kk * ((s >> 16) & 0xFFu);
    for (int p = 0; p < job.n_pairs; ++p) {
        const int gp = job.first_pair + p;
        const PairDesc pd = pairs[gp];
        uint32_t v0, v1, v2;
        remap_votes<K, false>(F + static_cast<size_t>(gp - pair0) * npx, styles + static_cast<size_t>(pd.style) * npx,
                              H, W, tc.r, tc.c, v0, v1, v2);
        a0 += v0;
        a1 += v1;
        a2 += v2;
    }
    const uint32_t den = job.den / 255u;  // k^2 c
    uint8_t* o = out + (static_cast<size_t>(blockIdx.y) * npx + x) * 3;
    o[0] = static_cast<uint8_t>((a0 + den / 2) / den);
    o[1] = static_cast<uint8_t>((a1 + den / 2) / den);
    o[2] = static_cast<uint8_t>((a2 + den / 2) / den);
}

// E(x) = the improved loss of the pair's current match against its current S^.
template <int K>
__global__ void __launch_bounds__(TILE_THREADS)
    energy_balanced_kernel(const PairDesc* __restrict__ pairs, int pair0, int H, int W,
                           const uint32_t* __restrict__ rp, const uint32_t* __restrict__ srp,
                           const uint32_t* __restrict__ shat_rp, int slot_by_target, int target0,
                           uint32_t alpha, const uint32_t* __restrict__ F, uint32_t* __restrict__ E) {
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const int pl = blockIdx.y;
    const PairDesc pd = pairs[pair0 + pl];
    const size_t x = static_cast<size_t>(tc.r) * W + tc.c;
    const size_t npx = static_cast<size_t>(H) * W;
    TargetPatch<K> tg, ts;
    load_target<K>(frame_rows<K>(rp, pd.tgt, H, W), H, W, tc.r, tc.c, tg);
    load_target<K>(frame_rows<K>(shat_rp, slot_by_target ? pd.tgt - target0 : pl, H, W), H, W, tc.r, tc.c, ts);
    const uint32_t f = F[static_cast<size_t>(pl) * npx + x];
    uint32_t e = 0;
    balanced_error_below<K>(frame_rows<K>(rp, pd.src, H, W), frame_rows<K>(srp, pd.style, H, W), H, W,
                            row_of(f), col_of(f), tg, ts, alpha, 0xFFFFFFFFu, &e);
    E[static_cast<size_t>(pl) * npx + x] = e;
}

// Two target patches per thread: fewer resident warps than the plain kernel.
#ifndef FB_BAL_WARPS5
#define FB_BAL_WARPS5 24
#endif
#ifndef FB_BAL_WARPS7
#define FB_BAL_WARPS7 16
#endif
template <int K>
struct BalancedWarps {
    static constexpr int value = K <= 3 ? 32 : K <= 5 ? FB_BAL_WARPS5 : K <= 7 ? FB_BAL_WARPS7 : 8;
};

template <int K>
__global__ void __launch_bounds__(TILE_THREADS, MinBlocks<BalancedWarps<K>::value>::value)
    nnf_iter_balanced_kernel(const PairDesc* __restrict__ pairs, int pair0, int H, int W,
                             const uint32_t* __restrict__ rp, const uint32_t* __restrict__ srp,
                             const uint32_t* __restrict__ shat_rp, int slot_by_target, int target0,
                             uint32_t alpha, int r0, uint32_t key0, uint32_t key1, uint32_t ctr_word,
                             const uint32_t* __restrict__ Fp, uint32_t* __restrict__ Fn,
                             uint32_t* __restrict__ En) {
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const int pl = blockIdx.y;
    const PairDesc pd = pairs[pair0 + pl];
    const size_t npx = static_cast<size_t>(H) * W;
    iterate_pixel_balanced<K>(frame_rows<K>(rp, pd.src, H, W), frame_rows<K>(srp, pd.style, H, W),
                              frame_rows<K>(rp, pd.tgt, H, W),
                              frame_rows<K>(shat_rp, slot_by_target ? pd.tgt - target0 : pl, H, W), alpha,
                              H, W, tc.r, tc.c, pd.tag, r0, key0, key1, ctr_word,
                              Fp + static_cast<size_t>(pl) * npx, Fn + static_cast<size_t>(pl) * npx,
                              En + static_cast<size_t>(pl) * npx);
}

// Alignment of Sec. 3.5.2 (Eq. 10), optionally with tracking: a pair with a partner
// (pd.pad[2], the other key's pair to the same frame, in this launch) takes the coupled
// loss against the partner's snapshot; a pair without one (a frame outside the key range)
// the plain loss.  The branch is uniform per block (one pair per grid row).
template <int K, bool TRACK>
__global__ void __launch_bounds__(TILE_THREADS, MinBlocks<BalancedWarps<K>::value>::value)
    nnf_iter_align_kernel(const PairDesc* __restrict__ pairs, int pair0, int H, int W,
                          const uint32_t* __restrict__ rp, const uint32_t* __restrict__ srp,
                          uint32_t alpha, int r0, uint32_t key0, uint32_t key1, uint32_t ctr_word,
                          const uint32_t* __restrict__ Fp, const uint32_t* __restrict__ Ep,
                          uint32_t* __restrict__ Fn, uint32_t* __restrict__ En) {
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const int pl = blockIdx.y;
    const PairDesc pd = pairs[pair0 + pl];
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t x = static_cast<size_t>(tc.r) * W + tc.c;
    const uint32_t* Fpp = Fp + static_cast<size_t>(pl) * npx;
    const uint32_t* prev = TRACK && pd.pad[0] >= 0 && in_launch(pd.pad[0] - pair0, pl)
                               ? Fp + static_cast<size_t>(pd.pad[0] - pair0) * npx + x : nullptr;
    const uint32_t* next = TRACK && pd.pad[1] >= 0 && in_launch(pd.pad[1] - pair0, pl)
                               ? Fp + static_cast<size_t>(pd.pad[1] - pair0) * npx + x : nullptr;
    const TrackNeighbours extra{prev, next};
    if (pd.pad[2] < 0 || !in_launch(pd.pad[2] - pair0, pl)) {
        TargetPatch<K> t;
        load_target<K>(frame_rows<K>(rp, pd.tgt, H, W), H, W, tc.r, tc.c, t);
        search_pixel<K>(PlainError<K>{frame_rows<K>(rp, pd.src, H, W), H, W, t}, H, W, tc.r, tc.c, pd.tag, r0,
                        key0, key1, ctr_word, Fpp, Fpp[x], Ep[static_cast<size_t>(pl) * npx + x],
                        Fn + static_cast<size_t>(pl) * npx, En + static_cast<size_t>(pl) * npx, extra);
        return;
    }
    const PairDesc po = pairs[pd.pad[2]];
    uint32_t fo = Fp[static_cast<size_t>(pd.pad[2] - pair0) * npx + x];
    if (!FB_CHECK(match_inside(fo, H, W), FB_CHECK_SNAPSHOT, row_of(fo), col_of(fo))) fo = 0u;
    iterate_pixel_aligned<K>(frame_rows<K>(rp, pd.src, H, W), frame_rows<K>(srp, pd.style, H, W),
                             frame_rows<K>(rp, pd.tgt, H, W), frame_rows<K>(srp, po.style, H, W), fo, alpha, H,
                             W, tc.r, tc.c, pd.tag, r0, key0, key1, ctr_word, Fpp,
                             Fn + static_cast<size_t>(pl) * npx, En + static_cast<size_t>(pl) * npx, extra);
}

// ---------------------------------------------------------------------------------
// Fast mode of Sec. 3.4: blending-table entries (Algs. 3-4) and the interval queries of
// the output frames (Alg. 5 + the split identity), exact integer sums.
// ---------------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(TILE_THREADS)
    fast_table_kernel(const FastEntry* __restrict__ entries, const int32_t* __restrict__ src_pairs,
                      const PairDesc* __restrict__ pairs, const uint32_t* __restrict__ F,
                      const uint32_t* __restrict__ styles, int H, int W, uint4* __restrict__ out) {
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const FastEntry e = entries[blockIdx.y];
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t x = static_cast<size_t>(tc.r) * W + tc.c;
    const uint32_t s = __ldg(styles + static_cast<size_t>(e.frame) * npx + x);
    constexpr uint32_t kk = static_cast<uint32_t>(K * K);
    uint32_t a0 = kk * (s & 0xFFu), a1 = kk * ((s >> 8) & 0xFFu), a2 = kk * ((s >> 16) & 0xFFu);
    for (int q = 0; q < e.n_src; ++q) {
        const int p = src_pairs[e.first_src + q];
        const PairDesc pd = pairs[p];
        uint32_t v0, v1, v2;
        remap_votes<K, false>(F + static_cast<size_t>(p) * npx, styles + static_cast<size_t>(pd.style) * npx, H,
                              W, tc.r, tc.c, v0, v1, v2);
        a0 += v0;
        a1 += v1;
        a2 += v2;
    }
    out[static_cast<size_t>(blockIdx.y) * npx + x] = make_uint4(a0, a1, a2, 0u);
}

template <int K>
__global__ void __launch_bounds__(TILE_THREADS)
    fast_combine_kernel(const FastJob* __restrict__ jobs, const int2* __restrict__ pieces,
                        const uint32_t* __restrict__ F, const uint4* __restrict__ entries,
                        const uint32_t* __restrict__ styles, int H, int W, float* __restrict__ out) {
    const TileCoord tc = tile_coord(W);
    if (tc.r >= H || tc.c >= W) return;
    const FastJob job = jobs[blockIdx.y];
    const size_t npx = static_cast<size_t>(H) * W;
    const size_t x = static_cast<size_t>(tc.r) * W + tc.c;
    constexpr uint32_t kk = static_cast<uint32_t>(K * K);
    uint32_t a0 = 0, a1 = 0, a2 = 0;
    for (int q = 0; q < job.n_pieces; ++q) {
        const int2 pc = pieces[job.first_piece + q];
        const uint4* T = entries + static_cast<size_t>(pc.x) * npx;
        if (pc.y < 0) {  // the piece ends at the output frame: identity remap
            const uint4 t = __ldg(T + x);
            a0 += kk * t.x;
            a1 += kk * t.y;
            a2 += kk * t.z;
        } else {
            uint32_t v0, v1, v2;
            remap_votes_u4<K>(F + static_cast<size_t>(pc.y) * npx, T, H, W, tc.r, tc.c, v0, v1, v2);
            a0 += v0;
            a1 += v1;
            a2 += v2;
        }
    }
    const uint32_t s = __ldg(styles + static_cast<size_t>(job.frame) * npx + x);
    constexpr uint32_t k4 = kk * kk;  // S_frame is in both the left and the right query
    a0 -= k4 * (s & 0xFFu);
    a1 -= k4 * ((s >> 8) & 0xFFu);
    a2 -= k4 * ((s >> 16) & 0xFFu);
    const double den = 255.0 * static_cast<double>(k4) * static_cast<double>(job.count);
    write_output_d(out + (static_cast<size_t>(job.frame) * npx + x) * 3, a0, a1, a2, den);
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
        uint32_t v0, v1, v2;
        remap_votes<K>(F + static_cast<size_t>(gp - pair0) * npx,
                       styles + static_cast<size_t>(pd.style) * npx, H, W, r, c, v0, v1, v2);
        a0 += pd.weight * v0;
        a1 += pd.weight * v1;
        a2 += pd.weight * v2;
    }
    write_output(out + (static_cast<size_t>(job.out_frame) * npx + x) * 3, a0, a1, a2, job.den);
}

// Sum of the Eq. 1 errors of n_elems values (double accumulator).
__global__ void __launch_bounds__(256) energy_sum_kernel(const uint32_t* __restrict__ E, size_t n,
                                                         double* __restrict__ acc) {
    double s = 0.0;
    for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        s += E[i];
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (static_cast<int>(threadIdx.x) < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(acc, red[0]);
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
    if (rowpatch_paired(k)) {
        const size_t n_slots = static_cast<size_t>(rowpatch_pair_rows(H)) * W;
        prep_guides_paired_kernel<<<dim3(blocks_for(n_slots, 256), static_cast<unsigned>(n_frames)), 256,
                                    0, st>>>(frames, H, W, rp);
        return cudaGetLastError();
    }
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

cudaError_t launch_shat(int k, const PairDesc* pairs, int pair0, int n_pairs, int H, int W,
                       const uint32_t* F, const uint32_t* styles, uint8_t* shat, cudaStream_t st) {
    if (n_pairs <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(H, W, n_pairs);
    const dim3 block(TILE_W, TILE_H);
    FB_DISPATCH_K(k, (shat_kernel<KK><<<grid, block, 0, st>>>(pairs, pair0, H, W, F, styles, shat)));
    return cudaGetLastError();
}

cudaError_t launch_energy_balanced(int k, const PairDesc* pairs, int pair0, int n_pairs,
                                   const LevelGeom& g, const uint32_t* srp, const uint32_t* shat_rp,
                                   int slot_by_target, int target0, uint32_t alpha, const uint32_t* F,
                                   uint32_t* E, cudaStream_t st) {
    if (n_pairs <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(g.H, g.W, n_pairs);
    const dim3 block(TILE_W, TILE_H);
    FB_DISPATCH_K(k, (energy_balanced_kernel<KK><<<grid, block, 0, st>>>(pairs, pair0, g.H, g.W, g.rp, srp,
                                                                       shat_rp, slot_by_target, target0,
                                                                       alpha, F, E)));
    return cudaGetLastError();
}

cudaError_t launch_tbar(int k, const JobDesc* jobs, int job0, int n_jobs, const PairDesc* pairs, int pair0,
                        const uint32_t* F, const uint32_t* styles, int H, int W, uint8_t* out,
                        cudaStream_t st) {
    if (n_jobs <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(H, W, n_jobs);
    const dim3 block(TILE_W, TILE_H);
    FB_DISPATCH_K(k, (tbar_kernel<KK><<<grid, block, 0, st>>>(jobs, job0, pairs, pair0, F, styles, H, W, out)));
    return cudaGetLastError();
}

cudaError_t launch_nnf_iter_balanced(int k, const PairDesc* pairs, int pair0, int n_pairs,
                                     const LevelGeom& g, const uint32_t* srp, const uint32_t* shat_rp,
                                     int slot_by_target, int target0, uint32_t alpha, int r0,
                                     uint64_t seed, int it, const uint32_t* Fp, uint32_t* Fn,
                                     uint32_t* En, cudaStream_t st) {
    if (n_pairs <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(g.H, g.W, n_pairs);
    const dim3 block(TILE_W, TILE_H);
    const uint32_t ctr_word = static_cast<uint32_t>(it + 1) << 8;  // level 0
    FB_DISPATCH_K(k, (nnf_iter_balanced_kernel<KK><<<grid, block, 0, st>>>(
                         pairs, pair0, g.H, g.W, g.rp, srp, shat_rp, slot_by_target, target0, alpha, r0,
                         static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32), ctr_word,
                         Fp, Fn, En)));
    return cudaGetLastError();
}

cudaError_t launch_fast_table(int k, const FastEntry* entries, int n_entries, const int32_t* src_pairs,
                              const PairDesc* pairs, const uint32_t* F, const uint32_t* styles, int H,
                              int W, uint4* out, cudaStream_t st) {
    if (n_entries <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(H, W, n_entries);
    const dim3 block(TILE_W, TILE_H);
    FB_DISPATCH_K(k, (fast_table_kernel<KK><<<grid, block, 0, st>>>(entries, src_pairs, pairs, F, styles, H,
                                                                   W, out)));
    return cudaGetLastError();
}

cudaError_t launch_fast_combine(int k, const FastJob* jobs, int n_jobs, const int2* pieces,
                                const uint32_t* F, const uint4* entries, const uint32_t* styles, int H,
                                int W, float* out, cudaStream_t st) {
    if (n_jobs <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(H, W, n_jobs);
    const dim3 block(TILE_W, TILE_H);
    FB_DISPATCH_K(k, (fast_combine_kernel<KK><<<grid, block, 0, st>>>(jobs, pieces, F, entries, styles, H, W,
                                                                     out)));
    return cudaGetLastError();
}

cudaError_t launch_nnf_iter_track(int k, const PairDesc* pairs, int pair0, int n_pairs, const LevelGeom& g,
                                  int r0, uint64_t seed, int it, const uint32_t* Fp, const uint32_t* Ep,
                                  uint32_t* Fn, uint32_t* En, cudaStream_t st) {
    if (n_pairs <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(g.H, g.W, n_pairs);
    const dim3 block(TILE_W, TILE_H);
    const uint32_t ctr_word = static_cast<uint32_t>(it + 1) << 8;  // level 0
    FB_DISPATCH_K(k, (nnf_iter_track_kernel<KK><<<grid, block, 0, st>>>(
                         pairs, pair0, g.H, g.W, g.rp, r0, static_cast<uint32_t>(seed),
                         static_cast<uint32_t>(seed >> 32), ctr_word, Fp, Ep, Fn, En)));
    return cudaGetLastError();
}

cudaError_t launch_nnf_iter_align(int k, const PairDesc* pairs, int pair0, int n_pairs, const LevelGeom& g,
                                  const uint32_t* srp, uint32_t alpha, bool tracking, int r0, uint64_t seed,
                                  int it, const uint32_t* Fp, const uint32_t* Ep, uint32_t* Fn, uint32_t* En,
                                  cudaStream_t st) {
    if (n_pairs <= 0) return cudaSuccess;
    const dim3 grid = tile_grid(g.H, g.W, n_pairs);
    const dim3 block(TILE_W, TILE_H);
    const uint32_t ctr_word = static_cast<uint32_t>(it + 1) << 8;  // level 0
    const uint32_t key0 = static_cast<uint32_t>(seed), key1 = static_cast<uint32_t>(seed >> 32);
    if (tracking) {
        FB_DISPATCH_K(k, (nnf_iter_align_kernel<KK, true><<<grid, block, 0, st>>>(
                             pairs, pair0, g.H, g.W, g.rp, srp, alpha, r0, key0, key1, ctr_word, Fp, Ep, Fn, En)));
    } else {
        FB_DISPATCH_K(k, (nnf_iter_align_kernel<KK, false><<<grid, block, 0, st>>>(
                             pairs, pair0, g.H, g.W, g.rp, srp, alpha, r0, key0, key1, ctr_word, Fp, Ep, Fn, En)));
    }
    return cudaGetLastError();
}

cudaError_t launch_energy_sum(const uint32_t* E, size_t n, double* acc, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    energy_sum_kernel<<<1184, 256, 0, st>>>(E, n, acc);
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

#ifdef FB_CHECKED
namespace fb {
cudaError_t check_read_kernels(unsigned long long out[3], bool reset) {
    return dev::check_read_unit(out, reset);
}
}  // namespace fb
#endif

// Debug counter of considered candidates (see fb_device.cuh); the product build reports
// FB_ERR_UNSUPPORTED.
extern "C" int fb_debug_candidates_considered(uint64_t* count, int reset) {
#ifdef FB_COUNT_EVALS
    if (!count) return FB_ERR_ARG;
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, fb::dev::g_candidates_considered, sizeof(v)) != cudaSuccess) {
        cudaGetLastError();
        return FB_ERR_CUDA;
    }
    *count = v;
    if (reset) {
        const unsigned long long zero = 0;
        if (cudaMemcpyToSymbol(fb::dev::g_candidates_considered, &zero, sizeof(zero)) != cudaSuccess) {
            cudaGetLastError();
            return FB_ERR_CUDA;
        }
    }
    return FB_OK;
#else
    (void)count;
    (void)reset;
    return FB_ERR_UNSUPPORTED;
#endif
}
