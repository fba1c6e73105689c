/*
 * fbref.h -- CPU oracle for the FastBlend hot path (arXiv 2311.09265).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously correct restatement
 * of what the paper computes, used to prove the CUDA library right.  Only the test
 * suite, the package smoke check and the timed CPU baseline of bench.py may load it.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * Conventions (the paper's notation, Sec. 3.2):
 *   images  H x W x 3 uint8, row-major, channel-fastest (HWC);
 *   NNF F   H x W x 2 int32, F(x) = (row, col) of the source patch centre matched to
 *           target pixel x = (row, col);  rows index the paper's first coordinate x;
 *   errors  E H x W uint32 (Eq. 1 evaluated at F).
 *
 * Parity status per function is listed in the header comment of fbref.c.
 */
#ifndef FBREF_H
#define FBREF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fbref_params {
    int32_t patch;   /* k = 2p+1, odd, 3..9                                       */
    int32_t iters;   /* n, patch-match iterations per pyramid level (Alg. 1)      */
    int32_t levels;  /* pyramid levels, >= 1 (Alg. 1 outer loop)                  */
    int32_t r0;      /* initial random-search radius; 0 => max(H', W') per level */
    uint64_t seed;   /* Philox key                                                */
} fbref_params;

/* Philox-4x32-10 counter-based generator (Salmon et al., SC'11). */
void fbref_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Eq. 1: squared L2 distance between the source patch centred at u=(ur,uc) and the
 * target patch centred at x=(xr,xc), k x k x 3 bytes, clamp-to-edge reads. */
uint32_t fbref_ssd(const uint8_t *src, const uint8_t *tgt, int H, int W, int k,
                   int ur, int uc, int xr, int xc);

/* Pyramid step of Alg. 1: 2x2 box average with round-half-up, clamped reads.
 * out has ((H+1)/2) x ((W+1)/2) x 3 bytes. */
void fbref_downsample(const uint8_t *img, int H, int W, uint8_t *out);

/* The random-search offset drawn for candidate t (radius r) of pixel `pix` in
 * iteration `it` at pyramid level `level` of the pair with tag `pair_tag`. */
void fbref_rs_offset(uint64_t seed, uint32_t pix, uint32_t pair_tag, int level, int it,
                     int t, int r, int32_t *dr, int32_t *dc);

/* Alg. 1 with the Jacobi schedule of Sec. 3.2.  init_nnf may be NULL (Philox random
 * init); a non-NULL init requires levels == 1.  Returns 0, or -1 on a bad argument. */
int fbref_nnf(const uint8_t *src, const uint8_t *tgt, int H, int W, const fbref_params *p,
              uint32_t pair_tag, const int32_t *init_nnf, int32_t *nnf_out, uint32_t *err_out);

/* Same as fbref_nnf but also records E after every iteration of the finest level:
 * err_trace holds (iters+1) x H x W values (index 0 = after initialisation). */
int fbref_nnf_trace(const uint8_t *src, const uint8_t *tgt, int H, int W, const fbref_params *p,
                    uint32_t pair_tag, const int32_t *init_nnf, int32_t *nnf_out,
                    uint32_t *err_trace);

/* Exhaustive nearest-neighbour field under Eq. 1: for every x the minimising u over the
 * whole source, ties to the smallest row-major index. */
void fbref_nnf_bruteforce(const uint8_t *src, const uint8_t *tgt, int H, int W, int k,
                          int32_t *nnf_out, uint32_t *err_out);

/* Alg. 2 without the final division: integer voting sums V (H x W x 3 uint32). */
void fbref_remap_sum(const uint8_t *style, const int32_t *nnf, int H, int W, int k,
                     uint32_t *v_out);

/* Alg. 2: V / (255 k^2) as float in [0, 1]. */
void fbref_remap(const uint8_t *style, const int32_t *nnf, int H, int W, int k, float *out);

/* Eq. 2 sliding-window blend of all frames.  guides, styles: N x H x W x 3;
 * out: N x H x W x 3 float.  window = 2M+1, odd.  Returns 0 or -1. */
int fbref_blend_window(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                       int window, const fbref_params *p, float *out);

/* Eq. 2 for the single output frame i (out: H x W x 3 float). */
int fbref_blend_frame(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                      int window, const fbref_params *p, int i, float *out);

/* Sec. 3.5.2 two-keyframe combine over all frames.  key_idx: n_keys sorted distinct
 * frame indices; key_styles: n_keys x H x W x 3.  Returns 0 or -1. */
int fbref_interpolate(const uint8_t *guides, int N, int H, int W, const int32_t *key_idx,
                      const uint8_t *key_styles, int n_keys, const fbref_params *p, float *out);

/* The same for the single output frame i. */
int fbref_interpolate_frame(const uint8_t *guides, int N, int H, int W, const int32_t *key_idx,
                            const uint8_t *key_styles, int n_keys, const fbref_params *p,
                            int i, float *out);

/* Tag that identifies the ordered pair (source frame j -> target frame i) in the
 * Philox counter. */
uint32_t fbref_pair_tag(int j, int i);

/* Sec. 3.5.1 tracking (one level): see fbref.c. */
int fbref_nnf_chain(const uint8_t *src, const uint8_t *tgts, int n, int H, int W,
                    const fbref_params *p, const uint32_t *tags, const int32_t *init,
                    int32_t *nnf_out, uint32_t *err_out);
int fbref_interpolate_tracking(const uint8_t *guides, int N, int H, int W,
                               const int32_t *key_idx, const uint8_t *key_styles, int n_keys,
                               const fbref_params *p, float *out);
/* Sec. 3.5.2 alignment (Eq. 10), one level: see fbref.c. */
int fbref_nnf_segment(const uint8_t *guide_l, const uint8_t *guide_r, const uint8_t *style_l,
                      const uint8_t *style_r, const uint8_t *tgts, int n, int H, int W,
                      const fbref_params *p, uint32_t alpha, int tracking, const uint32_t *tags_l,
                      const uint32_t *tags_r, const int32_t *init, int32_t *nnf_out,
                      uint32_t *err_out);
int fbref_interpolate_aligned(const uint8_t *guides, int N, int H, int W, const int32_t *key_idx,
                              const uint8_t *key_styles, int n_keys, const fbref_params *p,
                              uint32_t alpha, int tracking, float *out);
int fbref_blend_window_tracking(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                                int window, const fbref_params *p, float *out);

/* Sec. 3.4 quality improvement ("accurate mode"), one level: see fbref.c. */
int fbref_blend_frame_accurate(const uint8_t *guides, const uint8_t *styles, int N, int H,
                               int W, int window, const fbref_params *p, uint32_t alpha, int i,
                               float *out, uint8_t *tbar_out, int32_t *nnf_out);
int fbref_blend_window_accurate(const uint8_t *guides, const uint8_t *styles, int N, int H,
                                int W, int window, const fbref_params *p, uint32_t alpha,
                                float *out);

/* Sec. 3.4 fast mode (Algs. 3-5 and the split identity): see fbref.c. */
int fbref_blend_frame_fast(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                           int window, const fbref_params *p, int i, float *out);
int fbref_blend_window_fast(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                            int window, const fbref_params *p, float *out);

/* Sec. 3.4 improved loss ("balanced mode"), one level: see fbref.c. */
void fbref_shat(const uint8_t *style, const int32_t *nnf, int H, int W, int k, uint8_t *shat);
int fbref_nnf_balanced(const uint8_t *src_guide, const uint8_t *tgt_guide,
                       const uint8_t *src_style, int H, int W, const fbref_params *p,
                       uint32_t alpha, uint32_t pair_tag, const int32_t *init_nnf,
                       int32_t *nnf_out, uint32_t *err_out, uint8_t *shat_out);
int fbref_blend_frame_balanced(const uint8_t *guides, const uint8_t *styles, int N, int H,
                               int W, int window, const fbref_params *p, uint32_t alpha, int i,
                               float *out);
int fbref_blend_window_balanced(const uint8_t *guides, const uint8_t *styles, int N, int H,
                                int W, int window, const fbref_params *p, uint32_t alpha,
                                float *out);

/* Number of OpenMP threads the oracle uses, and a setter (n <= 0 is ignored). */
int fbref_num_threads(void);
void fbref_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
