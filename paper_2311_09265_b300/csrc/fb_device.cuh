// fb_device.cuh -- per-pixel device code of the FastBlend hot path, shared by the
// per-call kernels (fb_kernels.cu) and the batched persistent kernels (fb_batch.cu).
#pragma once

#include <cstdint>

#include "fb_check.cuh"
#include "fb_internal.h"

namespace fb {
namespace dev {

// Debug builds (-DFB_COUNT_EVALS, libfb_debug.so) count every candidate a pixel
// considers -- the initial match, each propagation neighbour inside the image and each
// random-search radius, duplicates included -- so a test can hold the count against its
// closed form.  Product builds compile the counting away.
#ifdef FB_COUNT_EVALS
static __device__ unsigned long long g_candidates_considered;
#define FB_COUNT_CANDIDATES(n) atomicAdd(&::fb::dev::g_candidates_considered, (unsigned long long)(n))
#else
#define FB_COUNT_CANDIDATES(n) ((void)0)
#endif

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
    static constexpr bool PAIRED = rowpatch_paired(K);  // k = 5: two rows per 32-byte slot
};

// Checked builds: the slots the patch at (r, c) reads lie inside the guide frame -- for
// the paired layout slot rows r/2 .. r/2 + 2 of rowpatch_pair_rows(H), otherwise column c
// of the (clamped) rows.  Always true in product builds.
template <int K>
__device__ __forceinline__ bool slots_inside(int r, int c, int H, int W) {
    if constexpr (Geo<K>::PAIRED)
        return FB_CHECK(r >= 0 && c >= 0 && c < W && (r >> 1) + 2 < rowpatch_pair_rows(H), FB_CHECK_SLOT,
                        (r >> 1) + 2, rowpatch_pair_rows(H));
    else
        return FB_CHECK(c >= 0 && c < W, FB_CHECK_SLOT, c, W);
}

// One 32-byte slot of the paired layout (two row patches of 4 words).  A 256-bit load
// is one request, like a 16-byte one, so the pair costs what one row did.  volatile:
// the load must stay behind the early-exit test that guards it.
__device__ __forceinline__ void load_slot(const uint32_t* __restrict__ p, uint32_t (&w)[8]) {
    asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
                   "=r"(w[6]), "=r"(w[7])
                 : "l"(p));
}

__device__ __forceinline__ void load_half_slot(const uint32_t* __restrict__ p, uint32_t (&w)[4]) {
    asm volatile("ld.global.nc.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3])
                 : "l"(p));
}

// Frame f of a guide stack laid out by prep_guides.
template <int K>
__device__ __forceinline__ const uint32_t* frame_rows(const uint32_t* rp, int f, int H, int W) {
    return rp + static_cast<size_t>(f) * rowpatch_frame_words(K, H, W);
}

template <int K>
__device__ __forceinline__ void load_row(const uint32_t* __restrict__ p,
                                         uint32_t (&out)[Geo<K>::NW]) {
    constexpr int NW = Geo<K>::NW;
    if constexpr (Geo<K>::RPW == 8 && NW > 4) {
        // k = 7, 9: the row sits in a 32-byte slot; one 256-bit load is one L1 request
        // (a 16- plus an 8- or 16-byte load would be two for the same sector).
        uint32_t w[8];
        load_slot(p, w);
#pragma unroll
        for (int i = 0; i < NW; ++i) out[i] = w[i];
        return;
    }
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

// The target patch, held in registers for all of a pixel's candidates.  |t_a|^2 of each
// row is recomputed per candidate row (one dp4a per word) rather than held: the k
// registers it would take cost more, as spills or as resident warps, than the dp4a issue.
template <int K>
struct TargetPatch {
    uint32_t w[K][Geo<K>::NW];  // the k rows of the target patch
};

template <int K>
__device__ __forceinline__ void load_target(const uint32_t* __restrict__ rpt, int H, int W,
                                            int r, int c, TargetPatch<K>& t) {
    using G = Geo<K>;
    if (!slots_inside<K>(r, c, H, W)) {  // checked builds only: an all-zero patch instead
#pragma unroll
        for (int a = 0; a < K; ++a) {
#pragma unroll
            for (int w = 0; w < G::NW; ++w) t.w[a][w] = 0;
        }
        return;
    }
    if constexpr (G::PAIRED) {
        // Rows r-2 .. r+2 are the clamped rows 2q-2 .. 2q-1 of slots q = r/2 + 0, 1, 2:
        // for even r they are halves 0..4 of the three slots, for odd r halves 1..5.
        const int odd = r & 1;
        const size_t stride = static_cast<size_t>(W) * 8;
        const uint32_t* base = rpt + (static_cast<size_t>(r >> 1) * W + c) * 8;
        uint32_t h[3][8];
#pragma unroll
        for (int L = 0; L < 3; ++L) load_slot(base + L * stride, h[L]);
#pragma unroll
        for (int a = 0; a < K; ++a) {
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint32_t ev = h[a >> 1][4 * (a & 1) + w];
                const uint32_t od = h[(a + 1) >> 1][4 * ((a + 1) & 1) + w];
                t.w[a][w] = odd ? od : ev;
            }
        }
    } else {
#pragma unroll
        for (int a = 0; a < K; ++a) {
            const int rr = clampi(r - G::P + a, 0, H - 1);
            load_row<K>(rpt + (static_cast<size_t>(rr) * W + c) * G::RPW, t.w[a]);
        }
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
    if (!slots_inside<K>(ur, uc, H, W)) return false;
    uint32_t acc = 0;
    if constexpr (G::PAIRED) {
        // Source rows ur-2 .. ur+2 sit in slots q = ur/2 + L (L = 0, 1, 2), whose halves
        // are patch rows a = 2L - odd and 2L - odd + 1 (a outside 0..4 is not part of the
        // patch).  The two slots holding two patch rows are read first -- L = 1, then
        // L = 0 for even ur or L = 2 for odd ur -- and the slot holding one row last, as a
        // 16-byte half: the early exit then has four of the five rows after two loads for
        // either parity.  Addresses and target rows differ by parity through selects, not
        // branches, so a warp's lanes stay converged.
        const int odd = ur & 1;
        const size_t stride = static_cast<size_t>(W) * 8;
        const uint32_t* base = rps + (static_cast<size_t>(ur >> 1) * W + uc) * 8;
        {   // L = 1: rows a = 2, 3 (even) or 1, 2 (odd)
            uint32_t s[8];
            load_slot(base + stride, s);
            uint32_t dot = 0, ss = 0, te = 0;
#pragma unroll
            for (int half = 0; half < 2; ++half)
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const uint32_t tw = odd ? t.w[1 + half][w] : t.w[2 + half][w];
                    const uint32_t sw = s[4 * half + w];
                    dot = __dp4a(sw, tw, dot);
                    ss = __dp4a(sw, sw, ss);
                    te = __dp4a(tw, tw, te);  // |t|^2 recomputed: five fewer live registers
                }
            acc += ss + te - 2u * dot;
            if (acc >= bound) return false;
        }
        {   // L = 0 (even: rows 0, 1) or L = 2 (odd: rows 3, 4)
            uint32_t s[8];
            load_slot(base + (odd ? 2 * stride : 0), s);
            uint32_t dot = 0, ss = 0, te = 0;
#pragma unroll
            for (int half = 0; half < 2; ++half)
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const uint32_t tw = odd ? t.w[3 + half][w] : t.w[half][w];
                    const uint32_t sw = s[4 * half + w];
                    dot = __dp4a(sw, tw, dot);
                    ss = __dp4a(sw, sw, ss);
                    te = __dp4a(tw, tw, te);
                }
            acc += ss + te - 2u * dot;
            if (acc >= bound) return false;
        }
        {   // the remaining row: L = 2 first half (even: row 4) or L = 0 second half (odd: row 0)
            uint32_t s[4];
            load_half_slot(base + (odd ? 4 : 2 * stride), s);
            uint32_t dot = 0, ss = 0, te = 0;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint32_t tw = odd ? t.w[0][w] : t.w[4][w];
                dot = __dp4a(s[w], tw, dot);
                ss = __dp4a(s[w], s[w], ss);
                te = __dp4a(tw, tw, te);
            }
            acc += ss + te - 2u * dot;
            if (acc >= bound) return false;
        }
        *e = acc;
        return true;
    } else {
#pragma unroll
        for (int a = 0; a < K; ++a) {
            const int rr = clampi(ur - G::P + a, 0, H - 1);
            uint32_t s[G::NW];
            load_row<K>(rps + (static_cast<size_t>(rr) * W + uc) * G::RPW, s);
            uint32_t dot = 0, ss = 0, te = 0;
#pragma unroll
            for (int w = 0; w < G::NW; ++w) {
                dot = __dp4a(s[w], t.w[a][w], dot);
                ss = __dp4a(s[w], s[w], ss);
                te = __dp4a(t.w[a][w], t.w[a][w], te);
            }
            acc += ss + te - 2u * dot;
            if (acc >= bound) return false;
        }
        *e = acc;
        return true;
    }
}

// Improved loss of Sec. 3.4 for candidate u = (ur, uc):
//   alpha * Eq.1(G_src at u, G_tgt at x) + Eq.1(S_src at u, S^ at x),
// accumulated per row (per paired slot for k = 5) with the same exact early exit as
// patch_error_below.  tg / ts: target guide and S^ patches of x; rpg / rpss: source
// guide and style row patches.  alpha <= 255 keeps every partial sum in uint32.
template <int K>
__device__ __forceinline__ bool balanced_error_below(const uint32_t* __restrict__ rpg,
                                                     const uint32_t* __restrict__ rpss, int H,
                                                     int W, int ur, int uc,
                                                     const TargetPatch<K>& tg,
                                                     const TargetPatch<K>& ts, uint32_t alpha,
                                                     uint32_t bound, uint32_t* e) {
    using G = Geo<K>;
    if (!slots_inside<K>(ur, uc, H, W)) return false;
    uint32_t acc = 0;
    if constexpr (G::PAIRED) {
        // Slot order and row selection as patch_error_below: the two two-row slots first
        // (L = 1, then L = 0 for even ur or L = 2 for odd ur), the one-row slot last as
        // 16-byte halves; the guide and style loads of a slot are issued together.
        const int odd = ur & 1;
        const size_t stride = static_cast<size_t>(W) * 8;
        const size_t off = (static_cast<size_t>(ur >> 1) * W + uc) * 8;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const size_t so = off + (i == 0 ? stride : (odd ? 2 * stride : 0));
            uint32_t sg[8], sst[8];
            load_slot(rpg + so, sg);
            load_slot(rpss + so, sst);
            uint32_t gd = 0, gs = 0, gt = 0, sd = 0, ss = 0, st = 0;
#pragma unroll
            for (int half = 0; half < 2; ++half)
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    // i = 0: rows 2, 3 (even) / 1, 2 (odd); i = 1: rows 0, 1 / 3, 4
                    const int ae = i == 0 ? 2 + half : half, ao = i == 0 ? 1 + half : 3 + half;
                    const uint32_t tgw = odd ? tg.w[ao][w] : tg.w[ae][w];
                    const uint32_t tsw = odd ? ts.w[ao][w] : ts.w[ae][w];
                    const uint32_t a = sg[4 * half + w], b = sst[4 * half + w];
                    gd = __dp4a(a, tgw, gd);
                    gs = __dp4a(a, a, gs);
                    gt = __dp4a(tgw, tgw, gt);
                    sd = __dp4a(b, tsw, sd);
                    ss = __dp4a(b, b, ss);
                    st = __dp4a(tsw, tsw, st);
                }
            acc += alpha * (gs + gt - 2u * gd) + (ss + st - 2u * sd);
            if (acc >= bound) return false;
        }
        {   // the remaining row: L = 2 first half (even: row 4) or L = 0 second half (odd: row 0)
            const size_t so = off + (odd ? 4 : 2 * stride);
            uint32_t sg[4], sst[4];
            load_half_slot(rpg + so, sg);
            load_half_slot(rpss + so, sst);
            uint32_t gd = 0, gs = 0, gt = 0, sd = 0, ss = 0, st = 0;
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const uint32_t tgw = odd ? tg.w[0][w] : tg.w[4][w];
                const uint32_t tsw = odd ? ts.w[0][w] : ts.w[4][w];
                gd = __dp4a(sg[w], tgw, gd);
                gs = __dp4a(sg[w], sg[w], gs);
                gt = __dp4a(tgw, tgw, gt);
                sd = __dp4a(sst[w], tsw, sd);
                ss = __dp4a(sst[w], sst[w], ss);
                st = __dp4a(tsw, tsw, st);
            }
            acc += alpha * (gs + gt - 2u * gd) + (ss + st - 2u * sd);
            if (acc >= bound) return false;
        }
    } else {
#pragma unroll
        for (int a = 0; a < K; ++a) {
            const int rr = clampi(ur - G::P + a, 0, H - 1);
            uint32_t sg[G::NW], sst[G::NW];
            load_row<K>(rpg + (static_cast<size_t>(rr) * W + uc) * G::RPW, sg);
            load_row<K>(rpss + (static_cast<size_t>(rr) * W + uc) * G::RPW, sst);
            // |t|^2 of both target rows recomputed per candidate: two held row energies per
            // row would cost 2k registers, which the two target patches cannot spare.
            uint32_t gd = 0, gs = 0, gt = 0, sd = 0, ss = 0, st = 0;
#pragma unroll
            for (int w = 0; w < G::NW; ++w) {
                gd = __dp4a(sg[w], tg.w[a][w], gd);
                gs = __dp4a(sg[w], sg[w], gs);
                gt = __dp4a(tg.w[a][w], tg.w[a][w], gt);
                sd = __dp4a(sst[w], ts.w[a][w], sd);
                ss = __dp4a(sst[w], sst[w], ss);
                st = __dp4a(ts.w[a][w], ts.w[a][w], st);
            }
            acc += alpha * (gs + gt - 2u * gd) + (ss + st - 2u * sd);
            if (acc >= bound) return false;
        }
    }
    *e = acc;
    return true;
}

// Candidate-error functors of the two losses (bound: the incumbent's error).
template <int K>
struct PlainError {
    const uint32_t* rps;
    int H, W;
    const TargetPatch<K>& t;
    __device__ __forceinline__ bool operator()(int ur, int uc, uint32_t bound, uint32_t* e) const {
        return patch_error_below<K>(rps, H, W, ur, uc, t, bound, e);
    }
};

template <int K>
struct BalancedError {
    const uint32_t* rpg;
    const uint32_t* rpss;
    int H, W;
    const TargetPatch<K>& tg;
    const TargetPatch<K>& ts;
    uint32_t alpha;
    __device__ __forceinline__ bool operator()(int ur, int uc, uint32_t bound, uint32_t* e) const {
        return balanced_error_below<K>(rpg, rpss, H, W, ur, uc, tg, ts, alpha, bound, e);
    }
};

// One Jacobi iteration of Alg. 1 (Sec. 3.2 parallel update) for target pixel (r, c) of
// one pair under the candidate error `err`: reads the pair's snapshot (Fp, Ep), writes
// (Fn, En).  Propagation from the four neighbours in the order (-1,0), (1,0), (0,-1),
// (0,1), then random search around the running best with radius r0 >> t; strict
// improvement only.  A candidate equal to the running best is skipped: its error equals
// the incumbent's, so it could not win.
// Extra candidates tried after propagation: none, or (tracking, Sec. 3.5.1) the matches
// of the chain neighbours at the same pixel.
struct NoExtra {
    template <class F>
    __device__ __forceinline__ void operator()(F&) const {}
};
struct TrackNeighbours {
    const uint32_t* prev;  // snapshot of the pair to target i - 1 at this pixel, or null
    const uint32_t* next;  // ... to target i + 1
    template <class F>
    __device__ __forceinline__ void operator()(F& consider) const {
        if (prev) {
            const uint32_t f = *prev;
            consider(row_of(f), col_of(f));
        }
        if (next) {
            const uint32_t f = *next;
            consider(row_of(f), col_of(f));
        }
    }
};

// (bf, be): the incumbent match and its error under `err`.
template <int K, class Err, class Extra = NoExtra>
__device__ __forceinline__ void search_pixel(const Err& err, int H, int W, int r, int c,
                                             uint32_t tag, int r0, uint32_t key0, uint32_t key1,
                                             uint32_t ctr_word, const uint32_t* __restrict__ Fpp,
                                             uint32_t bf, uint32_t be,
                                             uint32_t* __restrict__ Fnp,
                                             uint32_t* __restrict__ Enp, const Extra& extra = Extra{}) {
    const size_t x = static_cast<size_t>(r) * W + c;

#ifdef FB_COUNT_EVALS
    uint32_t n_considered = 0;
#endif
    auto consider = [&](int cr, int cc) {
#ifdef FB_COUNT_EVALS
        ++n_considered;
#endif
        if (!FB_CHECK(cr >= 0 && cr < H && cc >= 0 && cc < W, FB_CHECK_CANDIDATE, cr, cc)) return;
        const uint32_t f = pack_rc(cr, cc);
        if (f == bf) return;
        uint32_t e;
        if (err(cr, cc, be, &e)) {
            be = e;
            bf = f;
        }
    };

#ifdef FB_CHECKED
    // The snapshot invariant: the incumbent lies in the image and be is its loss.
    if (FB_CHECK(match_inside(bf, H, W), FB_CHECK_SNAPSHOT, row_of(bf), col_of(bf))) {
        uint32_t e = 0;
        err(row_of(bf), col_of(bf), 0xFFFFFFFFu, &e);
        (void)FB_CHECK(e == be, FB_CHECK_ENERGY, be, e);
    }
    FB_CHECK_TALLY(1);
#endif
    // A neighbour's snapshot match outside the image (checked builds) is no candidate.
    auto inside = [&](uint32_t f) {
        return FB_CHECK(match_inside(f, H, W), FB_CHECK_SNAPSHOT, row_of(f), col_of(f));
    };

    // Propagation: F'(x) = F(x + d) - d.
    if (r > 0) {
        const uint32_t f = Fpp[x - W];
        if (inside(f)) consider(min(row_of(f) + 1, H - 1), col_of(f));
    }
    if (r < H - 1) {
        const uint32_t f = Fpp[x + W];
        if (inside(f)) consider(max(row_of(f) - 1, 0), col_of(f));
    }
    if (c > 0) {
        const uint32_t f = Fpp[x - 1];
        if (inside(f)) consider(row_of(f), min(col_of(f) + 1, W - 1));
    }
    if (c < W - 1) {
        const uint32_t f = Fpp[x + 1];
        if (inside(f)) consider(row_of(f), max(col_of(f) - 1, 0));
    }

    extra(consider);

    // Random search: F'(x) = F(x) + U[-r, r]^2, r = r0 >> t, t = 0, 1, ... while r >= 1.
    uint4 u = make_uint4(0u, 0u, 0u, 0u);
    for (int tt = 0; (r0 >> tt) >= 1; ++tt) {
        const int rad = r0 >> tt;
        if ((tt & 1) == 0)
            u = philox4x32_10(make_uint4(static_cast<uint32_t>(x), tag,
                                         ctr_word | static_cast<uint32_t>(tt >> 1), 0u),
                              key0, key1);
        const uint32_t span = static_cast<uint32_t>(2 * rad + 1);
        const int dr = static_cast<int>(__umulhi((tt & 1) ? u.z : u.x, span)) - rad;
        const int dc = static_cast<int>(__umulhi((tt & 1) ? u.w : u.y, span)) - rad;
        consider(clampi(row_of(bf) + dr, 0, H - 1), clampi(col_of(bf) + dc, 0, W - 1));
    }

    Fnp[x] = bf;
    Enp[x] = be;
#ifdef FB_COUNT_EVALS
    FB_COUNT_CANDIDATES(n_considered);
#endif
}

// The plain method: Eq. 1 on the guides.
template <int K>
__device__ __forceinline__ void iterate_pixel(const uint32_t* __restrict__ rps,
                                              const uint32_t* __restrict__ rpt, int H, int W,
                                              int r, int c, uint32_t tag, int r0, uint32_t key0,
                                              uint32_t key1, uint32_t ctr_word,
                                              const uint32_t* __restrict__ Fpp,
                                              const uint32_t* __restrict__ Epp,
                                              uint32_t* __restrict__ Fnp,
                                              uint32_t* __restrict__ Enp) {
    TargetPatch<K> t;
    load_target<K>(rpt, H, W, r, c, t);
    const size_t x = static_cast<size_t>(r) * W + c;
    search_pixel<K>(PlainError<K>{rps, H, W, t}, H, W, r, c, tag, r0, key0, key1, ctr_word, Fpp,
                    Fpp[x], Epp[x], Fnp, Enp);
}

// Tracking (Sec. 3.5.1): the plain loss with the chain neighbours' matches as candidates.
template <int K>
__device__ __forceinline__ void iterate_pixel_tracking(
    const uint32_t* __restrict__ rps, const uint32_t* __restrict__ rpt, int H, int W, int r, int c,
    uint32_t tag, int r0, uint32_t key0, uint32_t key1, uint32_t ctr_word,
    const uint32_t* __restrict__ Fpp, const uint32_t* __restrict__ Epp,
    const uint32_t* __restrict__ Fprev, const uint32_t* __restrict__ Fnext, uint32_t* __restrict__ Fnp,
    uint32_t* __restrict__ Enp) {
    TargetPatch<K> t;
    load_target<K>(rpt, H, W, r, c, t);
    const size_t x = static_cast<size_t>(r) * W + c;
    search_pixel<K>(PlainError<K>{rps, H, W, t}, H, W, r, c, tag, r0, key0, key1, ctr_word, Fpp,
                    Fpp[x], Epp[x], Fnp, Enp,
                    TrackNeighbours{Fprev ? Fprev + x : nullptr, Fnext ? Fnext + x : nullptr});
}

// The improved loss of Sec. 3.4: the pair's S^ (rpshat, refreshed before the iteration)
// is the style target; the incumbent's loss is evaluated here against that S^.
template <int K>
__device__ __forceinline__ void iterate_pixel_balanced(
    const uint32_t* __restrict__ rpg_src, const uint32_t* __restrict__ rps_src,
    const uint32_t* __restrict__ rpg_tgt, const uint32_t* __restrict__ rpshat, uint32_t alpha,
    int H, int W, int r, int c, uint32_t tag, int r0, uint32_t key0, uint32_t key1,
    uint32_t ctr_word, const uint32_t* __restrict__ Fpp, uint32_t* __restrict__ Fnp,
    uint32_t* __restrict__ Enp) {
    TargetPatch<K> tg, ts;
    load_target<K>(rpg_tgt, H, W, r, c, tg);
    load_target<K>(rpshat, H, W, r, c, ts);
    const BalancedError<K> err{rpg_src, rps_src, H, W, tg, ts, alpha};
    const uint32_t bf = Fpp[static_cast<size_t>(r) * W + c];
    uint32_t be = 0;
    err(row_of(bf), col_of(bf), 0xFFFFFFFFu, &be);
    search_pixel<K>(err, H, W, r, c, tag, r0, key0, key1, ctr_word, Fpp, bf, be, Fnp, Enp);
}

// Alignment loss of Sec. 3.5.2 (Eq. 10) for a pair with a partner (the other key's pair
// to the same frame): alpha * Eq.1(guides) + Eq.1(own key style at u, partner key style at
// the partner's snapshot match fo of this pixel) -- the pairwise patch error, a patch of
// one keyframe against a patch of the other.  The incumbent is re-evaluated here against
// the partner's snapshot.  Extra: tracking candidates, or none.
template <int K, class Extra>
__device__ __forceinline__ void iterate_pixel_aligned(
    const uint32_t* __restrict__ rpg_src, const uint32_t* __restrict__ rps_src,
    const uint32_t* __restrict__ rpg_tgt, const uint32_t* __restrict__ rps_partner, uint32_t fo,
    uint32_t alpha, int H, int W, int r, int c, uint32_t tag, int r0, uint32_t key0, uint32_t key1,
    uint32_t ctr_word, const uint32_t* __restrict__ Fpp, uint32_t* __restrict__ Fnp,
    uint32_t* __restrict__ Enp, const Extra& extra) {
    TargetPatch<K> tg, ts;
    load_target<K>(rpg_tgt, H, W, r, c, tg);
    load_target<K>(rps_partner, H, W, row_of(fo), col_of(fo), ts);
    const BalancedError<K> err{rpg_src, rps_src, H, W, tg, ts, alpha};
    const uint32_t bf = Fpp[static_cast<size_t>(r) * W + c];
    uint32_t be = 0;
    err(row_of(bf), col_of(bf), 0xFFFFFFFFu, &be);
    search_pixel<K>(err, H, W, r, c, tag, r0, key0, key1, ctr_word, Fpp, bf, be, Fnp, Enp, extra);
}

// Initial field of Alg. 1 for target pixel (r, c) of one pair and its Eq. 1 error.
// mode 0: Philox random match; 1: the coarse level's match, doubled, plus the pixel's
// parity; 2: the caller's field (clamped into the image).
template <int K>
__device__ __forceinline__ void init_pixel(const uint32_t* __restrict__ rps,
                                           const uint32_t* __restrict__ rpt, int H, int W, int r,
                                           int c, uint32_t tag, int mode,
                                           const uint32_t* __restrict__ coarse_Fp, int Hc, int Wc,
                                           const int32_t* __restrict__ user_init, uint32_t key0,
                                           uint32_t key1, uint32_t level_word,
                                           uint32_t* __restrict__ Fp, uint32_t* __restrict__ Ep) {
    const size_t x = static_cast<size_t>(r) * W + c;
    int ur, uc;
    if (mode == 0) {
        const uint4 u = philox4x32_10(make_uint4(static_cast<uint32_t>(x), tag, level_word, 0u),
                                      key0, key1);
        ur = static_cast<int>(__umulhi(u.x, static_cast<uint32_t>(H)));
        uc = static_cast<int>(__umulhi(u.y, static_cast<uint32_t>(W)));
    } else if (mode == 1) {
        uint32_t fc = coarse_Fp[static_cast<size_t>(r >> 1) * Wc + (c >> 1)];
        if (!FB_CHECK(match_inside(fc, Hc, Wc), FB_CHECK_SNAPSHOT, row_of(fc), col_of(fc))) fc = 0u;
        ur = clampi(2 * row_of(fc) + (r & 1), 0, H - 1);
        uc = clampi(2 * col_of(fc) + (c & 1), 0, W - 1);
    } else {
        ur = clampi(user_init[2 * x], 0, H - 1);
        uc = clampi(user_init[2 * x + 1], 0, W - 1);
    }
    TargetPatch<K> t;
    load_target<K>(rpt, H, W, r, c, t);
    uint32_t e = 0;
    patch_error_below<K>(rps, H, W, ur, uc, t, 0xFFFFFFFFu, &e);
    Fp[x] = pack_rc(ur, uc);
    Ep[x] = e;
    FB_COUNT_CANDIDATES(1);
    FB_CHECK_TALLY(1);
}

// Source pixel of the vote of q^ = clamp(x + d) for target x: clamp(F(q^) - (q^ - x)) per
// coordinate.  F packs (row, col) in the two 16-bit halves of a word, both inside the image,
// so for H, W <= 32760 (no half can leave the signed 16-bit range) one per-halfword
// add-min-max instruction (DPX: max(min(a + b, c), 0)) forms both clamped coordinates, and
// the linear index row * W + col is t + row * (W - 65536); larger frames take the scalar
// clamps.  Both give the same pixel.
__device__ __forceinline__ bool votes_packed(int H, int W) { return H <= 32760 && W <= 32760; }

template <int K, bool PACKED, class Vote>
__device__ __forceinline__ void remap_walk(const uint32_t* __restrict__ Fq, int H, int W, int r, int c,
                                           Vote&& vote) {
    constexpr int P = K / 2;
    if (PACKED && votes_packed(H, W)) {   // uniform over the grid
        const uint32_t hi = (static_cast<uint32_t>(H - 1) << 16) | static_cast<uint32_t>(W - 1);
        const uint32_t wm = static_cast<uint32_t>(W) - 65536u;
#pragma unroll
        for (int a = -P; a <= P; ++a) {
            const int qr = clampi(r + a, 0, H - 1);
            const uint32_t ndr = static_cast<uint32_t>(r - qr) << 16;   // -(qr - r), high half
#pragma unroll
            for (int b = -P; b <= P; ++b) {
                const int qc = clampi(c + b, 0, W - 1);
                const uint32_t f = __ldg(Fq + static_cast<size_t>(qr) * W + qc);
                (void)FB_CHECK(match_inside(f, H, W), FB_CHECK_REMAP, row_of(f), col_of(f));
                const uint32_t t = __viaddmin_s16x2_relu(f, ndr | (static_cast<uint32_t>(c - qc) & 0xFFFFu), hi);
                vote(t + (t >> 16) * wm);
            }
        }
    } else {
#pragma unroll
        for (int a = -P; a <= P; ++a) {
            const int qr = clampi(r + a, 0, H - 1);
#pragma unroll
            for (int b = -P; b <= P; ++b) {
                const int qc = clampi(c + b, 0, W - 1);
                const uint32_t f = __ldg(Fq + static_cast<size_t>(qr) * W + qc);
                (void)FB_CHECK(match_inside(f, H, W), FB_CHECK_REMAP, row_of(f), col_of(f));
                const int sr = clampi(row_of(f) - (qr - r), 0, H - 1);
                const int sc = clampi(col_of(f) - (qc - c), 0, W - 1);
                vote(static_cast<uint32_t>(sr) * static_cast<uint32_t>(W) + static_cast<uint32_t>(sc));
            }
        }
    }
}

// Alg. 2 remap of one pair's style through its NNF at output pixel (r, c): the k^2 votes
// S(clamp(F(q^) - (q^ - x))), q^ = clamp(q), summed per channel.  S: RGBX words of the
// source style frame.  PACKED: the packed clamps where the frame allows them.
template <int K, bool PACKED = true>
__device__ __forceinline__ void remap_votes(const uint32_t* __restrict__ Fq,
                                            const uint32_t* __restrict__ S, int H, int W, int r,
                                            int c, uint32_t& v0, uint32_t& v1, uint32_t& v2) {
    // Channels summed two to a register in 16-bit lanes (R and B; G and the pad byte):
    // a lane holds at most k^2 * 255 <= 20655 for k <= 9, so no lane carries over.
    uint32_t rb = 0, gx = 0;
    remap_walk<K, PACKED>(Fq, H, W, r, c, [&](uint32_t idx) {
        const uint32_t s = __ldg(S + idx);
        rb += s & 0x00FF00FFu;
        gx += (s >> 8) & 0x00FF00FFu;
    });
    v0 = rb & 0xFFFFu;
    v1 = gx & 0xFFFFu;
    v2 = rb >> 16;
    FB_CHECK_TALLY(1);
}

// Alg. 2 vote sums of a fast-mode table entry (three uint32 sums per 16-byte pixel).  The
// scalar clamps: with 16-byte votes the packed form's extra live registers cost more than
// the instructions it saves.
template <int K>
__device__ __forceinline__ void remap_votes_u4(const uint32_t* __restrict__ Fq,
                                               const uint4* __restrict__ T, int H, int W, int r,
                                               int c, uint32_t& v0, uint32_t& v1, uint32_t& v2) {
    v0 = v1 = v2 = 0;
    remap_walk<K, false>(Fq, H, W, r, c, [&](uint32_t idx) {
        const uint4 s = __ldg(T + idx);
        v0 += s.x;
        v1 += s.y;
        v2 += s.z;
    });
    FB_CHECK_TALLY(1);
}

// Fast-mode output: num / den per channel, one IEEE double division rounded once to float.
__device__ __forceinline__ void write_output_d(float* __restrict__ o, uint32_t a0, uint32_t a1,
                                               uint32_t a2, double den) {
    o[0] = __double2float_rn(__ddiv_rn(__uint2double_rn(a0), den));
    o[1] = __double2float_rn(__ddiv_rn(__uint2double_rn(a1), den));
    o[2] = __double2float_rn(__ddiv_rn(__uint2double_rn(a2), den));
}

// Output value of one pixel: num / den per channel with one IEEE division.
__device__ __forceinline__ void write_output(float* __restrict__ o, uint32_t a0, uint32_t a1,
                                             uint32_t a2, uint32_t den_u) {
    const float den = __uint2float_rn(den_u);
    o[0] = __fdiv_rn(__uint2float_rn(a0), den);
    o[1] = __fdiv_rn(__uint2float_rn(a1), den);
    o[2] = __fdiv_rn(__uint2float_rn(a2), den);
}

}  // namespace dev
}  // namespace fb
