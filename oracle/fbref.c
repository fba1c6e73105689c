/*
 * fbref.c -- CPU oracle for the FastBlend hot path (arXiv 2311.09265).
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, the package smoke check and the
 * timed CPU baseline.  Never called by the product path.  Plain loops, integer
 * arithmetic, one IEEE float division per output value; no blocking, fusion or
 * reordering beyond the definitions cited at each function.  OpenMP only splits the
 * independent per-pixel loops (Sec. 3.2 updates every position independently).
 *
 * What pins each part (tests/test_oracle_*.py):
 *   Philox-4x32-10  known-answer vectors of Salmon et al. (tests/golden).
 *   SSD (Eq. 1)     hand-derived values on tiny images (tests/golden), closed forms
 *                   for constant images, brute-force agreement.
 *   NNF (Alg. 1)    brute-force exhaustive NNF on tiny inputs (E_pm >= E_bf, equality
 *                   after many iterations), known-shift fixed points, per-pixel
 *                   monotone energy, propagation fixing a single wrong match.
 *   Remap (Alg. 2)  identity NNF => identity, integer-shift NNF => shifted image,
 *                   a hand-derived border example (tests/golden).
 *   Blend (Eq. 2)   constant style => constant, identical frames => that frame,
 *                   closed form on known-shift clips, linearity, window truncation.
 *   Combine (Sec. 3.5.2)  keys copied, endpoint weights, weights sum to one,
 *                   closed form on known-shift clips.
 *   Improved loss, balanced mode (Sec. 3.4)  constant styles reduce to Eq. 1 scaled by
 *                   alpha, true-field fixed point, S^ rounding and refresh, returned
 *                   error = loss of the returned field, constant blends.
 *   Fast mode (Sec. 3.4, Algs. 3-5)  constants for every window, window one, linearity
 *                   in the styles, known-shift closed form.
 *   Accurate mode (Sec. 3.4)  per-frame constant styles reduce to the plain fields,
 *                   T-bar rounding and refresh, constant blends.
 *   Tracking (Sec. 3.5.1)  runs of one frame reduce to the plain search, a neighbour's
 *                   match handed over, monotone energy, Eq. 9 with constant keys, the
 *                   blend reductions (window 3, no iterations) and its composition.
 *   Alignment (Sec. 3.5.2, Eq. 10)  constant key styles reduce to the plain (or tracked)
 *                   search, brute-force initial loss, side symmetry, monotone coupled
 *                   loss, Eq. 9 with constant keys and its composition.
 * Parity unpinned: none of the functions above; end-to-end visual quality against
 * the paper's human study cannot be pinned (no data).
 */
#include "fbref.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------ */
/* Philox-4x32-10, written from its definition in Salmon, Moraes, Dror and Shaw,   */
/* "Parallel random numbers: as easy as 1, 2, 3" (SC'11): each of the 10 rounds    */
/* multiplies counter words 0 and 2 by two fixed odd constants, swaps the 32-bit   */
/* halves into a new 4-word block xor-ed with the round key and the untouched       */
/* words; the 2-word key is advanced by the Weyl increments between rounds.        */
/* ------------------------------------------------------------------------------ */
#define PHILOX_MUL_A 0xD2511F53u
#define PHILOX_MUL_B 0xCD9E8D57u
#define PHILOX_WEYL_A 0x9E3779B9u
#define PHILOX_WEYL_B 0xBB67AE85u

void fbref_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_WEYL_A;
            k1 += PHILOX_WEYL_B;
        }
        uint64_t pa = (uint64_t)PHILOX_MUL_A * x0;
        uint64_t pb = (uint64_t)PHILOX_MUL_B * x2;
        uint32_t pa_hi = (uint32_t)(pa >> 32), pa_lo = (uint32_t)pa;
        uint32_t pb_hi = (uint32_t)(pb >> 32), pb_lo = (uint32_t)pb;
        uint32_t y0 = pb_hi ^ x1 ^ k0;
        uint32_t y1 = pb_lo;
        uint32_t y2 = pa_hi ^ x3 ^ k1;
        uint32_t y3 = pa_lo;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------------ */
static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static uint8_t px(const uint8_t *img, int W, int r, int c, int ch)
{
    return img[((size_t)r * W + c) * 3 + ch];
}

/* Eq. 1, Sec. 3.2: || S[u] - T[x] ||_2^2 over the (2p+1)^2 RGB patch.  Patch reads
 * outside the image take the nearest edge pixel (clamp-to-edge on both images). */
uint32_t fbref_ssd(const uint8_t *src, const uint8_t *tgt, int H, int W, int k,
                   int ur, int uc, int xr, int xc)
{
    int p = k / 2;
    uint32_t acc = 0;
    for (int a = -p; a <= p; ++a) {
        for (int b = -p; b <= p; ++b) {
            int sr = clampi(ur + a, 0, H - 1), sc = clampi(uc + b, 0, W - 1);
            int tr = clampi(xr + a, 0, H - 1), tc = clampi(xc + b, 0, W - 1);
            for (int ch = 0; ch < 3; ++ch) {
                int d = (int)px(src, W, sr, sc, ch) - (int)px(tgt, W, tr, tc, ch);
                acc += (uint32_t)(d * d);
            }
        }
    }
    return acc;
}

/* Alg. 1, "resize images S, T": one pyramid step, 2x2 box mean, round half up. */
void fbref_downsample(const uint8_t *img, int H, int W, uint8_t *out)
{
    int h2 = (H + 1) / 2, w2 = (W + 1) / 2;
    for (int r = 0; r < h2; ++r) {
        for (int c = 0; c < w2; ++c) {
            int r0 = 2 * r, r1 = clampi(2 * r + 1, 0, H - 1);
            int c0 = 2 * c, c1 = clampi(2 * c + 1, 0, W - 1);
            for (int ch = 0; ch < 3; ++ch) {
                int s = px(img, W, r0, c0, ch) + px(img, W, r0, c1, ch) +
                        px(img, W, r1, c0, ch) + px(img, W, r1, c1, ch);
                out[((size_t)r * w2 + c) * 3 + ch] = (uint8_t)((s + 2) >> 2);
            }
        }
    }
}

uint32_t fbref_pair_tag(int j, int i) { return ((uint32_t)j << 16) | (uint32_t)i; }

int fbref_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void fbref_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Uniform integer in [0, n) from one 32-bit Philox word: floor(u * n / 2^32). */
static int32_t uniform_below(uint32_t u, uint32_t n)
{
    return (int32_t)(((uint64_t)u * n) >> 32);
}

/* Random search, Sec. 3.2: the offset (dr, dc) for radius r, each axis uniform on
 * [-r, r].  Candidates t = 2m and 2m+1 share one Philox block: t even takes words
 * 0,1 and t odd takes words 2,3 of counter (pix, pair_tag, level<<24 | (it+1)<<8 | m, 0). */
void fbref_rs_offset(uint64_t seed, uint32_t pix, uint32_t pair_tag, int level, int it,
                     int t, int r, int32_t *dr, int32_t *dc)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {pix, pair_tag,
                       ((uint32_t)level << 24) | ((uint32_t)(it + 1) << 8) | (uint32_t)(t >> 1),
                       0u};
    uint32_t u[4];
    fbref_philox4x32_10(ctr, key, u);
    int w = 2 * (t & 1);
    *dr = uniform_below(u[w], (uint32_t)(2 * r + 1)) - r;
    *dc = uniform_below(u[w + 1], (uint32_t)(2 * r + 1)) - r;
}

/* Random initialisation of F, Alg. 1 first line: row uniform in [0, H'), column
 * uniform in [0, W') from words 0,1 of counter (pix, pair_tag, level<<24, 0). */
static void random_match(uint64_t seed, uint32_t pix, uint32_t pair_tag, int level, int H,
                         int W, int32_t *r, int32_t *c)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {pix, pair_tag, (uint32_t)level << 24, 0u};
    uint32_t u[4];
    fbref_philox4x32_10(ctr, key, u);
    *r = uniform_below(u[0], (uint32_t)H);
    *c = uniform_below(u[1], (uint32_t)W);
}

static int params_ok(const fbref_params *p, int H, int W)
{
    if (!p) return 0;
    if (p->patch < 3 || p->patch > 9 || (p->patch & 1) == 0) return 0;
    if (p->iters < 0 || p->iters > 65534) return 0;
    if (p->levels < 1 || p->levels > 16) return 0;
    if (p->r0 < 0) return 0;
    if (H < 1 || W < 1 || H > 32767 || W > 32767) return 0;
    return 1;
}

/* Alg. 1 for one ordered pair (source `src`, target `tgt`).  Schedule: Sec. 3.2
 * drops the scan-order update for a parallel one in which all positions are updated
 * independently, so every iteration reads a snapshot (F, E) taken at its start and
 * writes a new (F, E); within one pixel the updating sequence is applied candidate
 * by candidate:
 *   propagation  F'(x) = F(x + d) - d for d = (-1,0), (1,0), (0,-1), (0,1), using the
 *                snapshot, skipping neighbours outside the target, clamping into
 *                the source;
 *   random search F'(x) = F(x) + (dr, dc), centred on the current best, r = r0 >> t
 *                for t = 0, 1, ... while r >= 1 (exponential decay to zero), clamped;
 * a candidate replaces the incumbent only if its error is strictly smaller (the
 * masked update of Alg. 1), so ties keep the earlier match. */
static int nnf_impl(const uint8_t *src, const uint8_t *tgt, int H, int W,
                    const fbref_params *p, uint32_t tag, const int32_t *init,
                    int32_t *nnf_out, uint32_t *err_out, uint32_t *err_trace)
{
    if (!params_ok(p, H, W) || !src || !tgt || !nnf_out) return -1;
    if (init && p->levels != 1) return -1;
    const int k = p->patch, L = p->levels;

    /* Image pyramid (Alg. 1, outer loop): level 0 is full resolution. */
    const uint8_t **ps = (const uint8_t **)calloc((size_t)L, sizeof(*ps));
    const uint8_t **pt = (const uint8_t **)calloc((size_t)L, sizeof(*pt));
    int *hs = (int *)calloc((size_t)L, sizeof(int)), *ws = (int *)calloc((size_t)L, sizeof(int));
    ps[0] = src; pt[0] = tgt; hs[0] = H; ws[0] = W;
    for (int l = 1; l < L; ++l) {
        hs[l] = (hs[l - 1] + 1) / 2;
        ws[l] = (ws[l - 1] + 1) / 2;
        uint8_t *a = (uint8_t *)malloc((size_t)hs[l] * ws[l] * 3);
        uint8_t *b = (uint8_t *)malloc((size_t)hs[l] * ws[l] * 3);
        fbref_downsample(ps[l - 1], hs[l - 1], ws[l - 1], a);
        fbref_downsample(pt[l - 1], hs[l - 1], ws[l - 1], b);
        ps[l] = a; pt[l] = b;
    }

    size_t npx0 = (size_t)H * W;
    int32_t *F = (int32_t *)malloc(npx0 * 2 * sizeof(int32_t));
    int32_t *Fn = (int32_t *)malloc(npx0 * 2 * sizeof(int32_t));
    uint32_t *E = (uint32_t *)malloc(npx0 * sizeof(uint32_t));
    uint32_t *En = (uint32_t *)malloc(npx0 * sizeof(uint32_t));

    for (int l = L - 1; l >= 0; --l) {
        const int h = hs[l], w = ws[l];
        const uint8_t *S = ps[l], *T = pt[l];
        if (l == L - 1) {
            for (int r = 0; r < h; ++r)
                for (int c = 0; c < w; ++c) {
                    size_t x = (size_t)r * w + c;
                    if (init) {
                        F[2 * x] = clampi(init[2 * x], 0, h - 1);
                        F[2 * x + 1] = clampi(init[2 * x + 1], 0, w - 1);
                    } else {
                        random_match(p->seed, (uint32_t)x, tag, l, h, w, &F[2 * x], &F[2 * x + 1]);
                    }
                }
        } else {
            /* Alg. 1, "upsample F": the coarse match of x>>1, doubled, plus x's parity. */
            const int wc = ws[l + 1];
            for (int r = 0; r < h; ++r)
                for (int c = 0; c < w; ++c) {
                    size_t xc = (size_t)(r >> 1) * wc + (c >> 1);
                    size_t x = (size_t)r * w + c;
                    Fn[2 * x] = clampi(2 * F[2 * xc] + (r & 1), 0, h - 1);
                    Fn[2 * x + 1] = clampi(2 * F[2 * xc + 1] + (c & 1), 0, w - 1);
                }
            int32_t *t = F; F = Fn; Fn = t;
        }
        /* Alg. 1, "initialize error matrix E". */
#pragma omp parallel for schedule(static)
        for (int r = 0; r < h; ++r)
            for (int c = 0; c < w; ++c) {
                size_t x = (size_t)r * w + c;
                E[x] = fbref_ssd(S, T, h, w, k, F[2 * x], F[2 * x + 1], r, c);
            }
        if (err_trace && l == 0) memcpy(err_trace, E, npx0 * sizeof(uint32_t));

        const int r0 = p->r0 > 0 ? p->r0 : (h > w ? h : w);
        static const int dirs[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
        for (int it = 0; it < p->iters; ++it) {
#pragma omp parallel for schedule(static)
            for (int r = 0; r < h; ++r) {
                for (int c = 0; c < w; ++c) {
                    size_t x = (size_t)r * w + c;
                    int32_t br = F[2 * x], bc = F[2 * x + 1];
                    uint32_t be = E[x];
                    for (int d = 0; d < 4; ++d) {
                        int nr = r + dirs[d][0], nc = c + dirs[d][1];
                        if (nr < 0 || nr >= h || nc < 0 || nc >= w) continue;
                        size_t n = (size_t)nr * w + nc;
                        int cr = clampi(F[2 * n] - dirs[d][0], 0, h - 1);
                        int cc = clampi(F[2 * n + 1] - dirs[d][1], 0, w - 1);
                        uint32_t e = fbref_ssd(S, T, h, w, k, cr, cc, r, c);
                        if (e < be) { be = e; br = cr; bc = cc; }
                    }
                    for (int t = 0; (r0 >> t) >= 1; ++t) {
                        int rad = r0 >> t;
                        int32_t dr, dc;
                        fbref_rs_offset(p->seed, (uint32_t)x, tag, l, it, t, rad, &dr, &dc);
                        int cr = clampi(br + dr, 0, h - 1);
                        int cc = clampi(bc + dc, 0, w - 1);
                        uint32_t e = fbref_ssd(S, T, h, w, k, cr, cc, r, c);
                        if (e < be) { be = e; br = cr; bc = cc; }
                    }
                    Fn[2 * x] = br; Fn[2 * x + 1] = bc; En[x] = be;
                }
            }
            int32_t *tf = F; F = Fn; Fn = tf;
            uint32_t *te = E; E = En; En = te;
            if (err_trace && l == 0) memcpy(err_trace + (size_t)(it + 1) * npx0, E, npx0 * sizeof(uint32_t));
        }
    }

    memcpy(nnf_out, F, npx0 * 2 * sizeof(int32_t));
    if (err_out) memcpy(err_out, E, npx0 * sizeof(uint32_t));
    free(F); free(Fn); free(E); free(En);
    for (int l = 1; l < L; ++l) { free((void *)ps[l]); free((void *)pt[l]); }
    free(ps); free(pt); free(hs); free(ws);
    return 0;
}

int fbref_nnf(const uint8_t *src, const uint8_t *tgt, int H, int W, const fbref_params *p,
              uint32_t pair_tag, const int32_t *init_nnf, int32_t *nnf_out, uint32_t *err_out)
{
    return nnf_impl(src, tgt, H, W, p, pair_tag, init_nnf, nnf_out, err_out, NULL);
}

int fbref_nnf_trace(const uint8_t *src, const uint8_t *tgt, int H, int W, const fbref_params *p,
                    uint32_t pair_tag, const int32_t *init_nnf, int32_t *nnf_out,
                    uint32_t *err_trace)
{
    return nnf_impl(src, tgt, H, W, p, pair_tag, init_nnf, nnf_out, NULL, err_trace);
}

/* The exact nearest-neighbour field of Eq. 1, by exhaustive search. */
void fbref_nnf_bruteforce(const uint8_t *src, const uint8_t *tgt, int H, int W, int k,
                          int32_t *nnf_out, uint32_t *err_out)
{
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            uint32_t be = 0xFFFFFFFFu;
            int br = 0, bc = 0;
            for (int ur = 0; ur < H; ++ur)
                for (int uc = 0; uc < W; ++uc) {
                    uint32_t e = fbref_ssd(src, tgt, H, W, k, ur, uc, r, c);
                    if (e < be) { be = e; br = ur; bc = uc; }
                }
            size_t x = (size_t)r * W + c;
            nnf_out[2 * x] = br; nnf_out[2 * x + 1] = bc;
            if (err_out) err_out[x] = be;
        }
    }
}

/* Alg. 2 (Sec. 3.3) without the division: for each neighbour q of x in the k x k
 * window, q is first clamped into the image (q^), then the source pixel
 * F(q^) - (q^ - x), clamped into the source, is added.  NNF entries outside the
 * image are clamped into it before use. */
void fbref_remap_sum(const uint8_t *style, const int32_t *nnf, int H, int W, int k,
                     uint32_t *v_out)
{
    int p = k / 2;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            uint32_t acc[3] = {0, 0, 0};
            for (int a = -p; a <= p; ++a) {
                for (int b = -p; b <= p; ++b) {
                    int qr = clampi(r + a, 0, H - 1), qc = clampi(c + b, 0, W - 1);
                    size_t q = (size_t)qr * W + qc;
                    int fr = clampi(nnf[2 * q], 0, H - 1), fc = clampi(nnf[2 * q + 1], 0, W - 1);
                    int sr = clampi(fr - (qr - r), 0, H - 1);
                    int sc = clampi(fc - (qc - c), 0, W - 1);
                    for (int ch = 0; ch < 3; ++ch) acc[ch] += px(style, W, sr, sc, ch);
                }
            }
            size_t x = (size_t)r * W + c;
            for (int ch = 0; ch < 3; ++ch) v_out[3 * x + ch] = acc[ch];
        }
    }
}

void fbref_remap(const uint8_t *style, const int32_t *nnf, int H, int W, int k, float *out)
{
    size_t n = (size_t)H * W * 3;
    uint32_t *v = (uint32_t *)malloc(n * sizeof(uint32_t));
    fbref_remap_sum(style, nnf, H, W, k, v);
    float den = (float)(255 * k * k);
    for (size_t i = 0; i < n; ++i) out[i] = (float)v[i] / den;
    free(v);
}

/* Remap the style frame `style` onto guide frame i through NNF(G_j, G_i), adding
 * weight * V into acc. */
static int add_remapped(const uint8_t *gj, const uint8_t *gi, const uint8_t *style, int H, int W,
                        const fbref_params *p, uint32_t tag, uint32_t weight, uint32_t *acc)
{
    size_t npx = (size_t)H * W;
    int32_t *F = (int32_t *)malloc(npx * 2 * sizeof(int32_t));
    uint32_t *V = (uint32_t *)malloc(npx * 3 * sizeof(uint32_t));
    int rc = fbref_nnf(gj, gi, H, W, p, tag, NULL, F, NULL);
    if (rc == 0) {
        fbref_remap_sum(style, F, H, W, p->patch, V);
        for (size_t t = 0; t < npx * 3; ++t) acc[t] += weight * V[t];
    }
    free(F); free(V);
    return rc;
}

/* Eq. 2 (Sec. 3.4) for output frame i.  The window [i-M, i+M] is truncated to the
 * clip and the sum is divided by the number of frames actually in it; the j = i term
 * is S_i itself (an identity remap).  Result = (k^2 S_i + sum_j V_{j->i}) /
 * (255 k^2 c_i), one IEEE float division per value. */
int fbref_blend_frame(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                      int window, const fbref_params *p, int i, float *out)
{
    if (!params_ok(p, H, W) || N < 1 || N > 65535 || window < 1 || (window & 1) == 0 || i < 0 || i >= N)
        return -1;
    const int k = p->patch, M = (window - 1) / 2;
    size_t npx = (size_t)H * W, fsz = npx * 3;
    uint32_t *acc = (uint32_t *)calloc(fsz, sizeof(uint32_t));
    for (size_t t = 0; t < fsz; ++t) acc[t] = (uint32_t)(k * k) * styles[(size_t)i * fsz + t];
    int lo = i - M < 0 ? 0 : i - M, hi = i + M > N - 1 ? N - 1 : i + M;
    int rc = 0;
    for (int j = lo; j <= hi && rc == 0; ++j) {
        if (j == i) continue;
        rc = add_remapped(guides + (size_t)j * fsz, guides + (size_t)i * fsz,
                          styles + (size_t)j * fsz, H, W, p, fbref_pair_tag(j, i), 1u, acc);
    }
    float den = (float)(255 * k * k * (hi - lo + 1));
    for (size_t t = 0; t < fsz; ++t) out[t] = (float)acc[t] / den;
    free(acc);
    return rc;
}

int fbref_blend_window(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                       int window, const fbref_params *p, float *out)
{
    size_t fsz = (size_t)H * W * 3;
    for (int i = 0; i < N; ++i) {
        int rc = fbref_blend_frame(guides, styles, N, H, W, window, p, i, out + (size_t)i * fsz);
        if (rc) return rc;
    }
    return 0;
}

/* Sec. 3.5.2: between keyframes l < i < r,
 *   S~_i = (r - i)/(r - l) (S_l -> S_i) + (i - l)/(r - l) (S_r -> S_i),
 * computed as ((r-i) V_l + (i-l) V_r) / (255 k^2 (r-l)).  Keyframes are output
 * unchanged (S/255).  Frames before the first or after the last keyframe take the
 * nearest keyframe alone (weight one). */
int fbref_interpolate_frame(const uint8_t *guides, int N, int H, int W, const int32_t *key_idx,
                            const uint8_t *key_styles, int n_keys, const fbref_params *p,
                            int i, float *out)
{
    if (!params_ok(p, H, W) || N < 1 || N > 65535 || n_keys < 1 || i < 0 || i >= N) return -1;
    for (int m = 0; m < n_keys; ++m) {
        if (key_idx[m] < 0 || key_idx[m] >= N) return -1;
        if (m > 0 && key_idx[m] <= key_idx[m - 1]) return -1;
    }
    const int k = p->patch;
    size_t npx = (size_t)H * W, fsz = npx * 3;
    uint32_t *acc = (uint32_t *)calloc(fsz, sizeof(uint32_t));
    uint32_t den_int;
    int rc = 0, key_here = -1, ml = -1, mr = -1;
    for (int m = 0; m < n_keys; ++m) {
        if (key_idx[m] == i) key_here = m;
        if (key_idx[m] < i) ml = m;
        if (key_idx[m] > i && mr < 0) mr = m;
    }
    const uint8_t *gi = guides + (size_t)i * fsz;
    if (key_here >= 0) {
        for (size_t t = 0; t < fsz; ++t) acc[t] = (uint32_t)(k * k) * key_styles[(size_t)key_here * fsz + t];
        den_int = (uint32_t)(255 * k * k);
    } else if (ml >= 0 && mr >= 0) {
        int l = key_idx[ml], r = key_idx[mr];
        rc = add_remapped(guides + (size_t)l * fsz, gi, key_styles + (size_t)ml * fsz, H, W, p,
                          fbref_pair_tag(l, i), (uint32_t)(r - i), acc);
        if (rc == 0)
            rc = add_remapped(guides + (size_t)r * fsz, gi, key_styles + (size_t)mr * fsz, H, W, p,
                              fbref_pair_tag(r, i), (uint32_t)(i - l), acc);
        den_int = (uint32_t)(255 * k * k * (r - l));
    } else {
        int m = ml >= 0 ? ml : mr;
        int l = key_idx[m];
        rc = add_remapped(guides + (size_t)l * fsz, gi, key_styles + (size_t)m * fsz, H, W, p,
                          fbref_pair_tag(l, i), 1u, acc);
        den_int = (uint32_t)(255 * k * k);
    }
    float den = (float)den_int;
    for (size_t t = 0; t < fsz; ++t) out[t] = (float)acc[t] / den;
    free(acc);
    return rc;
}

int fbref_interpolate(const uint8_t *guides, int N, int H, int W, const int32_t *key_idx,
                      const uint8_t *key_styles, int n_keys, const fbref_params *p, float *out)
{
    size_t fsz = (size_t)H * W * 3;
    for (int i = 0; i < N; ++i) {
        int rc = fbref_interpolate_frame(guides, N, H, W, key_idx, key_styles, n_keys, p, i,
                                         out + (size_t)i * fsz);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Sec. 3.4, improved blending loss ("balanced mode"):                               */
/*   L(x) = alpha ||G_j[F(x)] - G_i[x]||^2 + ||S_j[F(x)] - S^_i[x]||^2                */
/* over the k x k RGB patches of Eq. 1 (clamp-to-edge on every image).  S^_i is the  */
/* remap (Alg. 2) of S_j through the current field, rounded to 8-bit values; it is   */
/* refreshed once at the beginning of every iteration, and the incumbent's loss is   */
/* re-evaluated against the refreshed S^_i before the iteration's candidates are     */
/* compared with it.  alpha is an integer weight in [0, 255].                         */
/* ------------------------------------------------------------------------------ */

/* S^ = V / k^2 rounded half up per channel, V the Alg. 2 vote sum. */
void fbref_shat(const uint8_t *style, const int32_t *nnf, int H, int W, int k, uint8_t *shat)
{
    size_t n = (size_t)H * W * 3;
    uint32_t *v = (uint32_t *)malloc(n * sizeof(uint32_t));
    fbref_remap_sum(style, nnf, H, W, k, v);
    uint32_t kk = (uint32_t)(k * k);
    for (size_t t = 0; t < n; ++t) shat[t] = (uint8_t)((v[t] + kk / 2) / kk);
    free(v);
}

static uint32_t balanced_loss(const uint8_t *gs, const uint8_t *gt, const uint8_t *ss,
                              const uint8_t *shat, int H, int W, int k, uint32_t alpha,
                              int ur, int uc, int xr, int xc)
{
    return alpha * fbref_ssd(gs, gt, H, W, k, ur, uc, xr, xc) +
           fbref_ssd(ss, shat, H, W, k, ur, uc, xr, xc);
}

/* Alg. 1 with the loss above, one level: the same Jacobi schedule, candidate order,
 * random streams and strict acceptance as fbref_nnf.  shat_out (nullable) receives the
 * S^ of the last iteration (of the initial field when iters = 0); err_out holds L with
 * respect to it. */
int fbref_nnf_balanced(const uint8_t *src_guide, const uint8_t *tgt_guide,
                       const uint8_t *src_style, int H, int W, const fbref_params *p,
                       uint32_t alpha, uint32_t tag, const int32_t *init, int32_t *nnf_out,
                       uint32_t *err_out, uint8_t *shat_out)
{
    if (!params_ok(p, H, W) || p->levels != 1 || alpha > 255) return -1;
    if (!src_guide || !tgt_guide || !src_style || !nnf_out) return -1;
    const int k = p->patch, h = H, w = W;
    size_t npx = (size_t)H * W;
    int32_t *F = (int32_t *)malloc(npx * 2 * sizeof(int32_t));
    int32_t *Fn = (int32_t *)malloc(npx * 2 * sizeof(int32_t));
    uint32_t *E = (uint32_t *)malloc(npx * sizeof(uint32_t));
    uint32_t *En = (uint32_t *)malloc(npx * sizeof(uint32_t));
    uint8_t *shat = (uint8_t *)malloc(npx * 3);
    for (int r = 0; r < h; ++r)
        for (int c = 0; c < w; ++c) {
            size_t x = (size_t)r * w + c;
            if (init) {
                F[2 * x] = clampi(init[2 * x], 0, h - 1);
                F[2 * x + 1] = clampi(init[2 * x + 1], 0, w - 1);
            } else {
                random_match(p->seed, (uint32_t)x, tag, 0, h, w, &F[2 * x], &F[2 * x + 1]);
            }
        }
    const int r0 = p->r0 > 0 ? p->r0 : (h > w ? h : w);
    static const int dirs[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    const int rounds = p->iters > 0 ? p->iters : 1;
    for (int it = 0; it < rounds; ++it) {
        /* the beginning of the iteration: refresh S^ from the field, re-evaluate E */
        fbref_shat(src_style, F, h, w, k, shat);
#pragma omp parallel for schedule(static)
        for (int r = 0; r < h; ++r)
            for (int c = 0; c < w; ++c) {
                size_t x = (size_t)r * w + c;
                E[x] = balanced_loss(src_guide, tgt_guide, src_style, shat, h, w, k, alpha,
                                     F[2 * x], F[2 * x + 1], r, c);
            }
        if (p->iters == 0) break;
#pragma omp parallel for schedule(static)
        for (int r = 0; r < h; ++r) {
            for (int c = 0; c < w; ++c) {
                size_t x = (size_t)r * w + c;
                int32_t br = F[2 * x], bc = F[2 * x + 1];
                uint32_t be = E[x];
                for (int d = 0; d < 4; ++d) {
                    int nr = r + dirs[d][0], nc = c + dirs[d][1];
                    if (nr < 0 || nr >= h || nc < 0 || nc >= w) continue;
                    size_t n = (size_t)nr * w + nc;
                    int cr = clampi(F[2 * n] - dirs[d][0], 0, h - 1);
                    int cc = clampi(F[2 * n + 1] - dirs[d][1], 0, w - 1);
                    uint32_t e = balanced_loss(src_guide, tgt_guide, src_style, shat, h, w, k,
                                               alpha, cr, cc, r, c);
                    if (e < be) { be = e; br = cr; bc = cc; }
                }
                for (int t = 0; (r0 >> t) >= 1; ++t) {
                    int rad = r0 >> t;
                    int32_t dr, dc;
                    fbref_rs_offset(p->seed, (uint32_t)x, tag, 0, it, t, rad, &dr, &dc);
                    int cr = clampi(br + dr, 0, h - 1);
                    int cc = clampi(bc + dc, 0, w - 1);
                    uint32_t e = balanced_loss(src_guide, tgt_guide, src_style, shat, h, w, k,
                                               alpha, cr, cc, r, c);
                    if (e < be) { be = e; br = cr; bc = cc; }
                }
                Fn[2 * x] = br; Fn[2 * x + 1] = bc; En[x] = be;
            }
        }
        int32_t *tf = F; F = Fn; Fn = tf;
        uint32_t *te = E; E = En; En = te;
    }
    memcpy(nnf_out, F, npx * 2 * sizeof(int32_t));
    if (err_out) memcpy(err_out, E, npx * sizeof(uint32_t));
    if (shat_out) memcpy(shat_out, shat, npx * 3);
    free(F); free(Fn); free(E); free(En); free(shat);
    return 0;
}

/* Eq. 2 with the NNFs of the balanced mode: as fbref_blend_frame. */
int fbref_blend_frame_balanced(const uint8_t *guides, const uint8_t *styles, int N, int H,
                               int W, int window, const fbref_params *p, uint32_t alpha, int i,
                               float *out)
{
    if (!params_ok(p, H, W) || p->levels != 1 || N < 1 || N > 65535 || window < 1 ||
        (window & 1) == 0 || i < 0 || i >= N)
        return -1;
    const int k = p->patch, M = (window - 1) / 2;
    size_t npx = (size_t)H * W, fsz = npx * 3;
    uint32_t *acc = (uint32_t *)calloc(fsz, sizeof(uint32_t));
    int32_t *F = (int32_t *)malloc(npx * 2 * sizeof(int32_t));
    uint32_t *V = (uint32_t *)malloc(fsz * sizeof(uint32_t));
    for (size_t t = 0; t < fsz; ++t) acc[t] = (uint32_t)(k * k) * styles[(size_t)i * fsz + t];
    int lo = i - M < 0 ? 0 : i - M, hi = i + M > N - 1 ? N - 1 : i + M;
    int rc = 0;
    for (int j = lo; j <= hi && rc == 0; ++j) {
        if (j == i) continue;
        rc = fbref_nnf_balanced(guides + (size_t)j * fsz, guides + (size_t)i * fsz,
                                styles + (size_t)j * fsz, H, W, p, alpha, fbref_pair_tag(j, i),
                                NULL, F, NULL, NULL);
        if (rc == 0) {
            fbref_remap_sum(styles + (size_t)j * fsz, F, H, W, k, V);
            for (size_t t = 0; t < fsz; ++t) acc[t] += V[t];
        }
    }
    float den = (float)(255 * k * k * (hi - lo + 1));
    for (size_t t = 0; t < fsz; ++t) out[t] = (float)acc[t] / den;
    free(acc); free(F); free(V);
    return rc;
}

int fbref_blend_window_balanced(const uint8_t *guides, const uint8_t *styles, int N, int H,
                                int W, int window, const fbref_params *p, uint32_t alpha,
                                float *out)
{
    size_t fsz = (size_t)H * W * 3;
    for (int i = 0; i < N; ++i) {
        int rc = fbref_blend_frame_balanced(guides, styles, N, H, W, window, p, alpha, i,
                                            out + (size_t)i * fsz);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Sec. 3.4, fast mode: remapping table (Alg. 3), blending table (Alg. 4) and the    */
/* interval query (Alg. 5) over them, for output frame i.                            */
/*   Alg. 3 adds (S_a -> S_j) to RemappingTable(j, L+1) for j = a | (2^(L+1) - 1)    */
/*   whenever bit L of a is 0, i.e. for the 2^L sources a in [j - 2^(L+1) + 1,        */
/*   j - 2^L]; RemappingTable(j, 0) = S_j.  Alg. 4 takes prefix sums over L, so       */
/*   BlendingTable(j, L) = sum over a in [j - 2^L + 1, j] of (S_a -> S_j) (a = j: S_j). */
/*   Alg. 5 walks i = r, r - 2^L, ... down to l, each time with the largest L whose   */
/*   low L bits of i are set and whose entry stays inside [l, r], and adds            */
/*   (BlendingTable(i, L) -> S_r) through NNF(G_i, G_r) (the identity when i = r).    */
/* The window sum of Eq. 2 is the left query [lo, i] plus the query [i, hi] on the    */
/* reversed clip (the symmetric table) minus S_i (the split identity of Sec. 3.4).   */
/* All sums are exact integers: a remap contributes its k^2 votes, so the table       */
/* entries carry k^2 and the query terms k^4 times the remapped values; the result    */
/* is one division (in double, rounded once to float) by 255 k^4 (hi - lo + 1).       */
/* ------------------------------------------------------------------------------ */

/* Alg. 2 vote sums of a 3-channel uint32 image (an already-summed table entry). */
static void remap_sum_u32(const uint32_t *img, const int32_t *nnf, int H, int W, int k,
                          uint32_t *v_out)
{
    int p = k / 2;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            uint32_t acc[3] = {0, 0, 0};
            for (int a = -p; a <= p; ++a) {
                for (int b = -p; b <= p; ++b) {
                    int qr = clampi(r + a, 0, H - 1), qc = clampi(c + b, 0, W - 1);
                    size_t q = (size_t)qr * W + qc;
                    int fr = clampi(nnf[2 * q], 0, H - 1), fc = clampi(nnf[2 * q + 1], 0, W - 1);
                    int sr = clampi(fr - (qr - r), 0, H - 1);
                    int sc = clampi(fc - (qc - c), 0, W - 1);
                    for (int ch = 0; ch < 3; ++ch) acc[ch] += img[((size_t)sr * W + sc) * 3 + ch];
                }
            }
            size_t x = (size_t)r * W + c;
            for (int ch = 0; ch < 3; ++ch) v_out[3 * x + ch] = acc[ch];
        }
    }
}

/* frame index of position t in the clip order (reversed for the symmetric table) */
static int clip_frame(int t, int N, int rev) { return rev ? N - 1 - t : t; }

/* BlendingTable(j, L) in table order `rev` (k^2-scaled): k^2 S_j plus the remaps
 * (S_a -> S_j) through NNF(G_a, G_j) of the 2^L - 1 earlier positions a. */
static int blending_entry(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                          const fbref_params *p, int rev, int j, int L, uint32_t *out)
{
    const int k = p->patch;
    size_t npx = (size_t)H * W, fsz = npx * 3;
    int fj = clip_frame(j, N, rev);
    for (size_t t = 0; t < fsz; ++t) out[t] = (uint32_t)(k * k) * styles[(size_t)fj * fsz + t];
    int32_t *F = (int32_t *)malloc(npx * 2 * sizeof(int32_t));
    uint32_t *V = (uint32_t *)malloc(fsz * sizeof(uint32_t));
    int rc = 0;
    for (int a = j - (1 << L) + 1; a < j && rc == 0; ++a) {
        int fa = clip_frame(a, N, rev);
        rc = fbref_nnf(guides + (size_t)fa * fsz, guides + (size_t)fj * fsz, H, W, p,
                       fbref_pair_tag(fa, fj), NULL, F, NULL);
        if (rc == 0) {
            fbref_remap_sum(styles + (size_t)fa * fsz, F, H, W, k, V);
            for (size_t t = 0; t < fsz; ++t) out[t] += V[t];
        }
    }
    free(F); free(V);
    return rc;
}

/* Alg. 5 on the table of order `rev`: sum over the interval [l, r] (table positions) of
 * (S_a -> S_r), k^4-scaled, added into acc. */
static int query(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                 const fbref_params *p, int rev, int l, int r, uint32_t *acc)
{
    const int k = p->patch;
    size_t npx = (size_t)H * W, fsz = npx * 3;
    uint32_t *B = (uint32_t *)malloc(fsz * sizeof(uint32_t));
    uint32_t *V = (uint32_t *)malloc(fsz * sizeof(uint32_t));
    int32_t *F = (int32_t *)malloc(npx * 2 * sizeof(int32_t));
    int fr = clip_frame(r, N, rev);
    int rc = 0;
    int i = r;
    while (i >= l && rc == 0) {
        int L = 0;
        while (((i >> L) & 1) && i - (1 << (L + 1)) + 1 >= l) ++L;
        rc = blending_entry(guides, styles, N, H, W, p, rev, i, L, B);
        if (rc) break;
        if (i == r) {
            for (size_t t = 0; t < fsz; ++t) acc[t] += (uint32_t)(k * k) * B[t];  /* identity remap */
        } else {
            int fi = clip_frame(i, N, rev);
            rc = fbref_nnf(guides + (size_t)fi * fsz, guides + (size_t)fr * fsz, H, W, p,
                           fbref_pair_tag(fi, fr), NULL, F, NULL);
            if (rc) break;
            remap_sum_u32(B, F, H, W, k, V);
            for (size_t t = 0; t < fsz; ++t) acc[t] += V[t];
        }
        i -= 1 << L;
    }
    free(B); free(V); free(F);
    return rc;
}

int fbref_blend_frame_fast(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                           int window, const fbref_params *p, int i, float *out)
{
    if (!params_ok(p, H, W) || N < 1 || N > 65535 || window < 1 || (window & 1) == 0 || i < 0 || i >= N)
        return -1;
    const int k = p->patch, M = (window - 1) / 2;
    size_t fsz = (size_t)H * W * 3;
    int lo = i - M < 0 ? 0 : i - M, hi = i + M > N - 1 ? N - 1 : i + M;
    uint32_t *acc = (uint32_t *)calloc(fsz, sizeof(uint32_t));
    int rc = query(guides, styles, N, H, W, p, 0, lo, i, acc);                     /* [lo, i] */
    if (rc == 0)
        rc = query(guides, styles, N, H, W, p, 1, N - 1 - hi, N - 1 - i, acc);    /* [i, hi] */
    const uint32_t k4 = (uint32_t)(k * k * k * k);
    double den = 255.0 * k4 * (double)(hi - lo + 1);
    for (size_t t = 0; t < fsz; ++t) {
        uint32_t num = acc[t] - k4 * styles[(size_t)i * fsz + t];   /* S_i was counted twice */
        out[t] = (float)((double)num / den);
    }
    free(acc);
    return rc;
}

int fbref_blend_window_fast(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                            int window, const fbref_params *p, float *out)
{
    size_t fsz = (size_t)H * W * 3;
    for (int i = 0; i < N; ++i) {
        int rc = fbref_blend_frame_fast(guides, styles, N, H, W, window, p, i, out + (size_t)i * fsz);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Sec. 3.4, quality improvement ("accurate mode"), for output frame i: the NNFs of  */
/* all pairs (j -> i) of the truncated window are computed together.  At the        */
/* beginning of every iteration the mean remapped frame                              */
/*   Tbar_i = (k^2 S_i + sum_j V(S_j through F_j)) / (k^2 c_i)    (rounded half up)    */
/* is refreshed from the current fields and every pair's incumbent is re-evaluated    */
/* under L_j(x) = alpha ||G_j[F_j(x)] - G_i[x]||^2 + ||S_j[F_j(x)] - Tbar_i[x]||^2;    */
/* then each pair takes one Jacobi step (same order, streams, strict acceptance as    */
/* fbref_nnf).  The output is Eq. 2 of the final fields.  One level.                  */
/* ------------------------------------------------------------------------------ */
int fbref_blend_frame_accurate(const uint8_t *guides, const uint8_t *styles, int N, int H,
                               int W, int window, const fbref_params *p, uint32_t alpha, int i,
                               float *out, uint8_t *tbar_out, int32_t *nnf_out)
{
    if (!params_ok(p, H, W) || p->levels != 1 || alpha > 255 || N < 1 || N > 65535 ||
        window < 1 || (window & 1) == 0 || i < 0 || i >= N)
        return -1;
    const int k = p->patch, M = (window - 1) / 2, h = H, w = W;
    size_t npx = (size_t)H * W, fsz = npx * 3;
    int lo = i - M < 0 ? 0 : i - M, hi = i + M > N - 1 ? N - 1 : i + M;
    const int c_i = hi - lo + 1, np = c_i - 1;
    const uint8_t *Gi = guides + (size_t)i * fsz, *Si = styles + (size_t)i * fsz;
    int32_t *F = (int32_t *)malloc((size_t)(np > 0 ? np : 1) * npx * 2 * sizeof(int32_t));
    int32_t *Fn = (int32_t *)malloc((size_t)(np > 0 ? np : 1) * npx * 2 * sizeof(int32_t));
    uint32_t *E = (uint32_t *)malloc((size_t)(np > 0 ? np : 1) * npx * sizeof(uint32_t));
    uint32_t *En = (uint32_t *)malloc((size_t)(np > 0 ? np : 1) * npx * sizeof(uint32_t));
    uint32_t *acc = (uint32_t *)malloc(fsz * sizeof(uint32_t));
    uint32_t *V = (uint32_t *)malloc(fsz * sizeof(uint32_t));
    uint8_t *tbar = (uint8_t *)malloc(fsz);
    int js[65535];
    int q = 0;
    for (int j = lo; j <= hi; ++j)
        if (j != i) js[q++] = j;
    for (int m = 0; m < np; ++m)
        for (int r = 0; r < h; ++r)
            for (int c = 0; c < w; ++c) {
                size_t x = (size_t)r * w + c;
                random_match(p->seed, (uint32_t)x, fbref_pair_tag(js[m], i), 0, h, w,
                             &F[((size_t)m * npx + x) * 2], &F[((size_t)m * npx + x) * 2 + 1]);
            }
    const int r0 = p->r0 > 0 ? p->r0 : (h > w ? h : w);
    static const int dirs[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    const uint32_t kk = (uint32_t)(k * k), den_t = kk * (uint32_t)c_i;
    for (int it = 0; it < p->iters; ++it) {
        /* the beginning of the iteration: Tbar_i from the current fields */
        for (size_t t = 0; t < fsz; ++t) acc[t] = kk * Si[t];
        for (int m = 0; m < np; ++m) {
            fbref_remap_sum(styles + (size_t)js[m] * fsz, F + (size_t)m * npx * 2, h, w, k, V);
            for (size_t t = 0; t < fsz; ++t) acc[t] += V[t];
        }
        for (size_t t = 0; t < fsz; ++t) tbar[t] = (uint8_t)((acc[t] + den_t / 2) / den_t);
        for (int m = 0; m < np; ++m) {
            const uint8_t *Gj = guides + (size_t)js[m] * fsz, *Sj = styles + (size_t)js[m] * fsz;
            const int32_t *Fm = F + (size_t)m * npx * 2;
            int32_t *Fnm = Fn + (size_t)m * npx * 2;
            uint32_t *Em = E + (size_t)m * npx, *Enm = En + (size_t)m * npx;
            const uint32_t tag = fbref_pair_tag(js[m], i);
#pragma omp parallel for schedule(static)
            for (int r = 0; r < h; ++r)
                for (int c = 0; c < w; ++c) {
                    size_t x = (size_t)r * w + c;
                    Em[x] = balanced_loss(Gj, Gi, Sj, tbar, h, w, k, alpha, Fm[2 * x], Fm[2 * x + 1], r, c);
                }
#pragma omp parallel for schedule(static)
            for (int r = 0; r < h; ++r) {
                for (int c = 0; c < w; ++c) {
                    size_t x = (size_t)r * w + c;
                    int32_t br = Fm[2 * x], bc = Fm[2 * x + 1];
                    uint32_t be = Em[x];
                    for (int d = 0; d < 4; ++d) {
                        int nr = r + dirs[d][0], nc = c + dirs[d][1];
                        if (nr < 0 || nr >= h || nc < 0 || nc >= w) continue;
                        size_t n = (size_t)nr * w + nc;
                        int cr = clampi(Fm[2 * n] - dirs[d][0], 0, h - 1);
                        int cc = clampi(Fm[2 * n + 1] - dirs[d][1], 0, w - 1);
                        uint32_t e = balanced_loss(Gj, Gi, Sj, tbar, h, w, k, alpha, cr, cc, r, c);
                        if (e < be) { be = e; br = cr; bc = cc; }
                    }
                    for (int t = 0; (r0 >> t) >= 1; ++t) {
                        int rad = r0 >> t;
                        int32_t dr, dc;
                        fbref_rs_offset(p->seed, (uint32_t)x, tag, 0, it, t, rad, &dr, &dc);
                        int cr = clampi(br + dr, 0, h - 1);
                        int cc = clampi(bc + dc, 0, w - 1);
                        uint32_t e = balanced_loss(Gj, Gi, Sj, tbar, h, w, k, alpha, cr, cc, r, c);
                        if (e < be) { be = e; br = cr; bc = cc; }
                    }
                    Fnm[2 * x] = br; Fnm[2 * x + 1] = bc; Enm[x] = be;
                }
            }
        }
        int32_t *tf = F; F = Fn; Fn = tf;
        uint32_t *te = E; E = En; En = te;
    }
    /* Eq. 2 of the final fields */
    for (size_t t = 0; t < fsz; ++t) acc[t] = kk * Si[t];
    for (int m = 0; m < np; ++m) {
        fbref_remap_sum(styles + (size_t)js[m] * fsz, F + (size_t)m * npx * 2, h, w, k, V);
        for (size_t t = 0; t < fsz; ++t) acc[t] += V[t];
    }
    float den = (float)(255 * k * k * c_i);
    for (size_t t = 0; t < fsz; ++t) out[t] = (float)acc[t] / den;
    if (tbar_out && p->iters > 0) memcpy(tbar_out, tbar, fsz);   /* Tbar of the last iteration */
    if (nnf_out && np > 0) memcpy(nnf_out, F, (size_t)np * npx * 2 * sizeof(int32_t));  /* j ascending */
    free(F); free(Fn); free(E); free(En); free(acc); free(V); free(tbar);
    return 0;
}

int fbref_blend_window_accurate(const uint8_t *guides, const uint8_t *styles, int N, int H,
                                int W, int window, const fbref_params *p, uint32_t alpha,
                                float *out)
{
    size_t fsz = (size_t)H * W * 3;
    for (int i = 0; i < N; ++i) {
        int rc = fbref_blend_frame_accurate(guides, styles, N, H, W, window, p, alpha, i,
                                            out + (size_t)i * fsz, NULL, NULL);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Sec. 3.5.1, tracking: the NNFs from one source frame to n consecutive target      */
/* frames form a chain; in every iteration the updating sequence of NNF(S, T_m) is    */
/* expanded by the matches of NNF(S, T_{m-1}) and NNF(S, T_{m+1}) at the same pixel    */
/* (snapshots of the previous iteration), tried after the four propagation            */
/* candidates and before the random search.  Same streams, order and strict           */
/* acceptance as fbref_nnf otherwise; one level.  init (nullable): n initial fields.   */
/* ------------------------------------------------------------------------------ */
int fbref_nnf_chain(const uint8_t *src, const uint8_t *tgts, int n, int H, int W,
                    const fbref_params *p, const uint32_t *tags, const int32_t *init,
                    int32_t *nnf_out, uint32_t *err_out)
{
    if (!params_ok(p, H, W) || p->levels != 1 || n < 1 || !src || !tgts || !tags || !nnf_out)
        return -1;
    const int k = p->patch, h = H, w = W;
    size_t npx = (size_t)H * W, fsz = npx * 3;
    int32_t *F = (int32_t *)malloc((size_t)n * npx * 2 * sizeof(int32_t));
    int32_t *Fn = (int32_t *)malloc((size_t)n * npx * 2 * sizeof(int32_t));
    uint32_t *E = (uint32_t *)malloc((size_t)n * npx * sizeof(uint32_t));
    uint32_t *En = (uint32_t *)malloc((size_t)n * npx * sizeof(uint32_t));
    for (int m = 0; m < n; ++m) {
        const uint8_t *T = tgts + (size_t)m * fsz;
        for (int r = 0; r < h; ++r)
            for (int c = 0; c < w; ++c) {
                size_t x = (size_t)r * w + c, o = ((size_t)m * npx + x) * 2;
                if (init) {
                    F[o] = clampi(init[o], 0, h - 1);
                    F[o + 1] = clampi(init[o + 1], 0, w - 1);
                } else {
                    random_match(p->seed, (uint32_t)x, tags[m], 0, h, w, &F[o], &F[o + 1]);
                }
                E[(size_t)m * npx + x] = fbref_ssd(src, T, h, w, k, F[o], F[o + 1], r, c);
            }
    }
    const int r0 = p->r0 > 0 ? p->r0 : (h > w ? h : w);
    static const int dirs[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    for (int it = 0; it < p->iters; ++it) {
        for (int m = 0; m < n; ++m) {
            const uint8_t *T = tgts + (size_t)m * fsz;
            const int32_t *Fm = F + (size_t)m * npx * 2;
#pragma omp parallel for schedule(static)
            for (int r = 0; r < h; ++r) {
                for (int c = 0; c < w; ++c) {
                    size_t x = (size_t)r * w + c;
                    int32_t br = Fm[2 * x], bc = Fm[2 * x + 1];
                    uint32_t be = E[(size_t)m * npx + x];
                    for (int d = 0; d < 4; ++d) {
                        int nr = r + dirs[d][0], nc = c + dirs[d][1];
                        if (nr < 0 || nr >= h || nc < 0 || nc >= w) continue;
                        size_t q = (size_t)nr * w + nc;
                        int cr = clampi(Fm[2 * q] - dirs[d][0], 0, h - 1);
                        int cc = clampi(Fm[2 * q + 1] - dirs[d][1], 0, w - 1);
                        uint32_t e = fbref_ssd(src, T, h, w, k, cr, cc, r, c);
                        if (e < be) { be = e; br = cr; bc = cc; }
                    }
                    for (int nb = m - 1; nb <= m + 1; nb += 2) {   /* tracking: T_{m-1}, T_{m+1} */
                        if (nb < 0 || nb >= n) continue;
                        const int32_t *Fb = F + ((size_t)nb * npx + x) * 2;
                        uint32_t e = fbref_ssd(src, T, h, w, k, Fb[0], Fb[1], r, c);
                        if (e < be) { be = e; br = Fb[0]; bc = Fb[1]; }
                    }
                    for (int t = 0; (r0 >> t) >= 1; ++t) {
                        int rad = r0 >> t;
                        int32_t dr, dc;
                        fbref_rs_offset(p->seed, (uint32_t)x, tags[m], 0, it, t, rad, &dr, &dc);
                        int cr = clampi(br + dr, 0, h - 1);
                        int cc = clampi(bc + dc, 0, w - 1);
                        uint32_t e = fbref_ssd(src, T, h, w, k, cr, cc, r, c);
                        if (e < be) { be = e; br = cr; bc = cc; }
                    }
                    Fn[((size_t)m * npx + x) * 2] = br;
                    Fn[((size_t)m * npx + x) * 2 + 1] = bc;
                    En[(size_t)m * npx + x] = be;
                }
            }
        }
        int32_t *tf = F; F = Fn; Fn = tf;
        uint32_t *te = E; E = En; En = te;
    }
    memcpy(nnf_out, F, (size_t)n * npx * 2 * sizeof(int32_t));
    if (err_out) memcpy(err_out, E, (size_t)n * npx * sizeof(uint32_t));
    free(F); free(Fn); free(E); free(En);
    return 0;
}

/* Sec. 3.5.2 with tracking: every keyframe's NNFs to the run of frames on each side of it
 * that it serves are one chain.  Output as fbref_interpolate. */
int fbref_interpolate_tracking(const uint8_t *guides, int N, int H, int W,
                               const int32_t *key_idx, const uint8_t *key_styles, int n_keys,
                               const fbref_params *p, float *out)
{
    if (!params_ok(p, H, W) || p->levels != 1 || N < 1 || N > 65535 || n_keys < 1) return -1;
    for (int m = 0; m < n_keys; ++m) {
        if (key_idx[m] < 0 || key_idx[m] >= N) return -1;
        if (m > 0 && key_idx[m] <= key_idx[m - 1]) return -1;
    }
    const int k = p->patch;
    size_t npx = (size_t)H * W, fsz = npx * 3;
    uint32_t *acc = (uint32_t *)calloc((size_t)N * fsz, sizeof(uint32_t));
    uint32_t *den = (uint32_t *)calloc((size_t)N, sizeof(uint32_t));
    uint32_t *V = (uint32_t *)malloc(fsz * sizeof(uint32_t));
    int rc = 0;
    for (int m = 0; m < n_keys && rc == 0; ++m) {
        const int a = key_idx[m];
        for (size_t t = 0; t < fsz; ++t) acc[(size_t)a * fsz + t] = (uint32_t)(k * k) * key_styles[(size_t)m * fsz + t];
        den[a] = (uint32_t)(255 * k * k);
        /* the frames this key serves: left run (after the previous key, or from 0) and
         * right run (up to the next key, or to N - 1) */
        const int prev = m > 0 ? key_idx[m - 1] : -1, next = m + 1 < n_keys ? key_idx[m + 1] : N;
        const int runs[2][2] = {{prev + 1, a - 1}, {a + 1, next - 1}};
        for (int side = 0; side < 2 && rc == 0; ++side) {
            const int lo = runs[side][0], hi = runs[side][1];
            if (lo > hi) continue;
            const int n = hi - lo + 1;
            uint32_t *tags = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
            int32_t *F = (int32_t *)malloc((size_t)n * npx * 2 * sizeof(int32_t));
            for (int q = 0; q < n; ++q) tags[q] = fbref_pair_tag(a, lo + q);
            rc = fbref_nnf_chain(guides + (size_t)a * fsz, guides + (size_t)lo * fsz, n, H, W, p, tags,
                                 NULL, F, NULL);
            for (int q = 0; q < n && rc == 0; ++q) {
                const int i = lo + q;
                /* Eq. 9 weights: (r - i) for the left key, (i - l) for the right key, over
                 * (r - l); a frame outside the key range takes its one key with weight one */
                uint32_t wgt, dd;
                if (side == 1 && next < N) { wgt = (uint32_t)(next - i); dd = (uint32_t)(next - a); }
                else if (side == 0 && prev >= 0) { wgt = (uint32_t)(i - prev); dd = (uint32_t)(a - prev); }
                else { wgt = 1u; dd = 1u; }
                fbref_remap_sum(key_styles + (size_t)m * fsz, F + (size_t)q * npx * 2, H, W, k, V);
                for (size_t t = 0; t < fsz; ++t) acc[(size_t)i * fsz + t] += wgt * V[t];
                den[i] = (uint32_t)(255 * k * k) * dd;
            }
            free(tags); free(F);
        }
    }
    for (int i = 0; i < N; ++i) {
        float d = (float)den[i];
        for (size_t t = 0; t < fsz; ++t) out[(size_t)i * fsz + t] = (float)acc[(size_t)i * fsz + t] / d;
    }
    free(acc); free(den); free(V);
    return rc;
}

/* ------------------------------------------------------------------------------ */
/* Sec. 3.5.2, alignment (Eq. 10): between keyframes l < r the NNFs F_l = NNF(l -> i) and */
/* F_r = NNF(r -> i) of every frame l < i < r are coupled.  The loss of a candidate u  */
/* of F_l at pixel x is                                                                 */
/*   alpha * Eq.1(G_l at u, G_i at x) + Eq.1(S_l at u, S_r at F_r(x)),                  */
/* the second term a patch difference between the two keyframes' styles (the pairwise  */
/* patch error), and symmetrically for F_r.  F_r(x) is the partner's snapshot of the   */
/* previous iteration (Jacobi), so the incumbent's loss is re-evaluated at the start of */
/* every iteration.  With tracking (Sec. 3.5.1) each side's n NNFs also form a chain.   */
/* Candidate order, random streams (tags_l[m] = tag of (l -> l+1+m), tags_r[m] of      */
/* (r -> l+1+m)) and strict acceptance as fbref_nnf; one level.  Fields and errors are */
/* laid out left chain first (index s * n + m).  With iters = 0, err_out holds the      */
/* coupled loss of the initial fields.                                                  */
/* ------------------------------------------------------------------------------ */
static uint32_t aligned_loss(const uint8_t *gs, const uint8_t *gt, const uint8_t *ss,
                             const uint8_t *so, int H, int W, int k, uint32_t alpha, int ur, int uc,
                             int xr, int xc, int pr, int pc)
{
    return alpha * fbref_ssd(gs, gt, H, W, k, ur, uc, xr, xc) +
           fbref_ssd(ss, so, H, W, k, ur, uc, pr, pc);
}

int fbref_nnf_segment(const uint8_t *guide_l, const uint8_t *guide_r, const uint8_t *style_l,
                      const uint8_t *style_r, const uint8_t *tgts, int n, int H, int W,
                      const fbref_params *p, uint32_t alpha, int tracking, const uint32_t *tags_l,
                      const uint32_t *tags_r, const int32_t *init, int32_t *nnf_out,
                      uint32_t *err_out)
{
    if (!params_ok(p, H, W) || p->levels != 1 || n < 1 || alpha > 255 || !guide_l || !guide_r ||
        !style_l || !style_r || !tgts || !tags_l || !tags_r || !nnf_out)
        return -1;
    const int k = p->patch, h = H, w = W;
    const size_t npx = (size_t)H * W, fsz = npx * 3, nf = (size_t)2 * n;
    const uint8_t *G[2] = {guide_l, guide_r}, *S[2] = {style_l, style_r};
    const uint32_t *tags[2] = {tags_l, tags_r};
    int32_t *F = (int32_t *)malloc(nf * npx * 2 * sizeof(int32_t));
    int32_t *Fn = (int32_t *)malloc(nf * npx * 2 * sizeof(int32_t));
    uint32_t *E = (uint32_t *)malloc(nf * npx * sizeof(uint32_t));
    for (int sd = 0; sd < 2; ++sd)
        for (int m = 0; m < n; ++m)
            for (size_t x = 0; x < npx; ++x) {
                size_t o = (((size_t)sd * n + m) * npx + x) * 2;
                if (init) {
                    F[o] = clampi(init[o], 0, h - 1);
                    F[o + 1] = clampi(init[o + 1], 0, w - 1);
                } else {
                    random_match(p->seed, (uint32_t)x, tags[sd][m], 0, h, w, &F[o], &F[o + 1]);
                }
            }
    const int r0 = p->r0 > 0 ? p->r0 : (h > w ? h : w);
    static const int dirs[4][2] = {{-1, 0}, {1, 0}, {0, -1}, {0, 1}};
    const int rounds = p->iters > 0 ? p->iters : 1;
    for (int it = 0; it < rounds; ++it) {
        for (int sd = 0; sd < 2; ++sd) {
            const uint8_t *Gs = G[sd], *Ss = S[sd], *So = S[1 - sd];
            for (int m = 0; m < n; ++m) {
                const uint8_t *T = tgts + (size_t)m * fsz;
                const int32_t *Fm = F + ((size_t)sd * n + m) * npx * 2;
                const int32_t *Fo = F + ((size_t)(1 - sd) * n + m) * npx * 2;   /* the partner */
                int32_t *Fnm = Fn + ((size_t)sd * n + m) * npx * 2;
                uint32_t *Em = E + ((size_t)sd * n + m) * npx;
#pragma omp parallel for schedule(static)
                for (int r = 0; r < h; ++r) {
                    for (int c = 0; c < w; ++c) {
                        size_t x = (size_t)r * w + c;
                        const int pr = Fo[2 * x], pc = Fo[2 * x + 1];
                        int32_t br = Fm[2 * x], bc = Fm[2 * x + 1];
                        uint32_t be = aligned_loss(Gs, T, Ss, So, h, w, k, alpha, br, bc, r, c, pr, pc);
                        if (p->iters > 0) {
                            for (int d = 0; d < 4; ++d) {
                                int nr = r + dirs[d][0], nc = c + dirs[d][1];
                                if (nr < 0 || nr >= h || nc < 0 || nc >= w) continue;
                                size_t q = (size_t)nr * w + nc;
                                int cr = clampi(Fm[2 * q] - dirs[d][0], 0, h - 1);
                                int cc = clampi(Fm[2 * q + 1] - dirs[d][1], 0, w - 1);
                                uint32_t e = aligned_loss(Gs, T, Ss, So, h, w, k, alpha, cr, cc, r, c, pr, pc);
                                if (e < be) { be = e; br = cr; bc = cc; }
                            }
                            for (int nb = m - 1; tracking && nb <= m + 1; nb += 2) {
                                if (nb < 0 || nb >= n) continue;
                                const int32_t *Fb = F + (((size_t)sd * n + nb) * npx + x) * 2;
                                uint32_t e = aligned_loss(Gs, T, Ss, So, h, w, k, alpha, Fb[0], Fb[1], r, c, pr, pc);
                                if (e < be) { be = e; br = Fb[0]; bc = Fb[1]; }
                            }
                            for (int t = 0; (r0 >> t) >= 1; ++t) {
                                int rad = r0 >> t;
                                int32_t dr, dc;
                                fbref_rs_offset(p->seed, (uint32_t)x, tags[sd][m], 0, it, t, rad, &dr, &dc);
                                int cr = clampi(br + dr, 0, h - 1);
                                int cc = clampi(bc + dc, 0, w - 1);
                                uint32_t e = aligned_loss(Gs, T, Ss, So, h, w, k, alpha, cr, cc, r, c, pr, pc);
                                if (e < be) { be = e; br = cr; bc = cc; }
                            }
                        }
                        Fnm[2 * x] = br;
                        Fnm[2 * x + 1] = bc;
                        Em[x] = be;
                    }
                }
            }
        }
        int32_t *tf = F; F = Fn; Fn = tf;
    }
    memcpy(nnf_out, F, nf * npx * 2 * sizeof(int32_t));
    if (err_out) memcpy(err_out, E, nf * npx * sizeof(uint32_t));
    free(F); free(Fn); free(E);
    return 0;
}

/* Sec. 3.5.2 with the alignment loss of Eq. 10 (alpha the guide weight; tracking
 * optional): the frames between two keys take fbref_nnf_segment's coupled fields; frames
 * before the first key or after the last have one key and no partner, and take the
 * plain loss (fbref_nnf, or a tracked chain).  Output: the Eq. 9 combination exactly as
 * fbref_interpolate. */
int fbref_interpolate_aligned(const uint8_t *guides, int N, int H, int W, const int32_t *key_idx,
                              const uint8_t *key_styles, int n_keys, const fbref_params *p,
                              uint32_t alpha, int tracking, float *out)
{
    if (!params_ok(p, H, W) || p->levels != 1 || alpha > 255 || N < 1 || N > 65535 || n_keys < 1)
        return -1;
    for (int m = 0; m < n_keys; ++m) {
        if (key_idx[m] < 0 || key_idx[m] >= N) return -1;
        if (m > 0 && key_idx[m] <= key_idx[m - 1]) return -1;
    }
    const int k = p->patch;
    const size_t npx = (size_t)H * W, fsz = npx * 3;
    uint32_t *acc = (uint32_t *)calloc((size_t)N * fsz, sizeof(uint32_t));
    uint32_t *den = (uint32_t *)calloc((size_t)N, sizeof(uint32_t));
    uint32_t *V = (uint32_t *)malloc(fsz * sizeof(uint32_t));
    int rc = 0;
    for (int m = 0; m < n_keys; ++m) {
        const int a = key_idx[m];
        for (size_t t = 0; t < fsz; ++t) acc[(size_t)a * fsz + t] = (uint32_t)(k * k) * key_styles[(size_t)m * fsz + t];
        den[a] = (uint32_t)(255 * k * k);
    }
    /* runs served by one key: before the first key (served by key 0) and after the last */
    for (int side = 0; side < 2 && rc == 0; ++side) {
        const int m = side == 0 ? 0 : n_keys - 1, a = key_idx[m];
        const int lo = side == 0 ? 0 : a + 1, hi = side == 0 ? a - 1 : N - 1;
        if (lo > hi) continue;
        const int n = hi - lo + 1;
        int32_t *Fs = (int32_t *)malloc((size_t)n * npx * 2 * sizeof(int32_t));
        uint32_t *tags = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
        for (int q = 0; q < n; ++q) tags[q] = fbref_pair_tag(a, lo + q);
        if (tracking)
            rc = fbref_nnf_chain(guides + (size_t)a * fsz, guides + (size_t)lo * fsz, n, H, W, p, tags, NULL, Fs, NULL);
        for (int q = 0; q < n && rc == 0; ++q) {
            if (!tracking)
                rc = fbref_nnf(guides + (size_t)a * fsz, guides + (size_t)(lo + q) * fsz, H, W, p, tags[q], NULL,
                               Fs + (size_t)q * npx * 2, NULL);
            if (rc) break;
            fbref_remap_sum(key_styles + (size_t)m * fsz, Fs + (size_t)q * npx * 2, H, W, k, V);
            for (size_t t = 0; t < fsz; ++t) acc[(size_t)(lo + q) * fsz + t] += V[t];
            den[lo + q] = (uint32_t)(255 * k * k);
        }
        free(Fs); free(tags);
    }
    /* segments between consecutive keys: coupled fields */
    for (int m = 0; m + 1 < n_keys && rc == 0; ++m) {
        const int l = key_idx[m], r = key_idx[m + 1], n = r - l - 1;
        if (n < 1) continue;
        int32_t *Fs = (int32_t *)malloc((size_t)2 * n * npx * 2 * sizeof(int32_t));
        uint32_t *tl = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
        uint32_t *tr = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
        for (int q = 0; q < n; ++q) {
            tl[q] = fbref_pair_tag(l, l + 1 + q);
            tr[q] = fbref_pair_tag(r, l + 1 + q);
        }
        rc = fbref_nnf_segment(guides + (size_t)l * fsz, guides + (size_t)r * fsz,
                               key_styles + (size_t)m * fsz, key_styles + (size_t)(m + 1) * fsz,
                               guides + (size_t)(l + 1) * fsz, n, H, W, p, alpha, tracking, tl, tr, NULL,
                               Fs, NULL);
        for (int q = 0; q < n && rc == 0; ++q) {
            const int i = l + 1 + q;
            fbref_remap_sum(key_styles + (size_t)m * fsz, Fs + (size_t)q * npx * 2, H, W, k, V);
            for (size_t t = 0; t < fsz; ++t) acc[(size_t)i * fsz + t] += (uint32_t)(r - i) * V[t];
            fbref_remap_sum(key_styles + (size_t)(m + 1) * fsz, Fs + (size_t)(n + q) * npx * 2, H, W, k, V);
            for (size_t t = 0; t < fsz; ++t) acc[(size_t)i * fsz + t] += (uint32_t)(i - l) * V[t];
            den[i] = (uint32_t)(255 * k * k) * (uint32_t)(r - l);
        }
        free(Fs); free(tl); free(tr);
    }
    for (int i = 0; i < N; ++i) {
        float d = (float)den[i];
        for (size_t t = 0; t < fsz; ++t) out[(size_t)i * fsz + t] = (float)acc[(size_t)i * fsz + t] / d;
    }
    free(acc); free(den); free(V);
    return rc;
}

/* Sec. 3.5.1 applied to the Eq. 2 blend (the optional setting the paper mentions): the
 * NNFs from source frame j to the targets of its window form two chains, the targets
 * before j and the targets after j (no NNF(G_j, G_j) is computed, so a chain ends next to
 * its source); each chain is computed with tracking, then every output frame is the Eq. 2
 * mean over its window exactly as in fbref_blend_frame. */
int fbref_blend_window_tracking(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                                int window, const fbref_params *p, float *out)
{
    if (!params_ok(p, H, W) || p->levels != 1 || N < 1 || N > 65535 || window < 1 || (window & 1) == 0)
        return -1;
    const int k = p->patch, M = (window - 1) / 2;
    size_t npx = (size_t)H * W, fsz = npx * 3;
    uint32_t *acc = (uint32_t *)calloc((size_t)N * fsz, sizeof(uint32_t));
    uint32_t *V = (uint32_t *)malloc(fsz * sizeof(uint32_t));
    for (size_t t = 0; t < (size_t)N * fsz; ++t) acc[t] = (uint32_t)(k * k) * styles[t];
    int rc = 0;
    for (int j = 0; j < N && rc == 0; ++j) {
        const int runs[2][2] = {{j - M < 0 ? 0 : j - M, j - 1}, {j + 1, j + M > N - 1 ? N - 1 : j + M}};
        for (int side = 0; side < 2 && rc == 0; ++side) {
            const int lo = runs[side][0], hi = runs[side][1];
            if (lo > hi) continue;
            const int n = hi - lo + 1;
            uint32_t *tags = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
            int32_t *F = (int32_t *)malloc((size_t)n * npx * 2 * sizeof(int32_t));
            for (int q = 0; q < n; ++q) tags[q] = fbref_pair_tag(j, lo + q);
            rc = fbref_nnf_chain(guides + (size_t)j * fsz, guides + (size_t)lo * fsz, n, H, W, p, tags,
                                 NULL, F, NULL);
            for (int q = 0; q < n && rc == 0; ++q) {
                fbref_remap_sum(styles + (size_t)j * fsz, F + (size_t)q * npx * 2, H, W, k, V);
                uint32_t *a = acc + (size_t)(lo + q) * fsz;
                for (size_t t = 0; t < fsz; ++t) a[t] += V[t];
            }
            free(tags); free(F);
        }
    }
    for (int i = 0; i < N; ++i) {
        const int lo = i - M < 0 ? 0 : i - M, hi = i + M > N - 1 ? N - 1 : i + M;
        float den = (float)(255 * k * k * (hi - lo + 1));
        for (size_t t = 0; t < fsz; ++t) out[(size_t)i * fsz + t] = (float)acc[(size_t)i * fsz + t] / den;
    }
    free(acc); free(V);
    return rc;
}
