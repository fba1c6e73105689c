/*
 * fb.h -- C ABI of libfb.so, a B300 (sm_103a) implementation of the hot path of
 * FastBlend (Duan et al., "FastBlend: a Powerful Model-Free Toolkit Making Video
 * Stylization Easier", arXiv 2311.09265): patch-match NNF search between guide frames
 * (Sec. 3.2, Alg. 1, Eq. 1), NNF-driven remapping of style frames (Sec. 3.3, Alg. 2),
 * sliding-window blending (Sec. 3.4, Eq. 2) and two-keyframe interpolation
 * (Sec. 3.5.2, the linear keyframe combination).
 *
 * Equations are numbered in order of appearance in the paper: Eq. 1 patch loss,
 * Eq. 2 window blend, ..., Eq. 9 the linear two-keyframe combination.
 *
 * Conventions shared by every entry point
 *   Images     H x W x 3 uint8, row-major, channel-fastest (HWC), contiguous.
 *              Frame stacks are N such images back to back.
 *   NNF        H x W x 2 int32: entry x = (row, col) of the SOURCE patch centre matched
 *              to TARGET pixel x (the paper's F(i, j) = (x, y), Sec. 3.2).
 *   Errors     H x W uint32, Eq. 1 evaluated at the returned NNF.
 *   Outputs    float32 in [0, 1] (value / 255), same HWC layout as the inputs.
 *   Patch      k = 2p+1 pixels per side, odd, 3 <= k <= 9; reads outside an image
 *              take the nearest edge pixel (clamp-to-edge).
 *   Sizes      k <= H, W <= 32767.  Frame counts 1 <= N <= 65535.
 *   Memory     Unless an entry point says otherwise, every data pointer is a DEVICE
 *              pointer on the context's device, owned by the caller, and must stay
 *              valid until the work enqueued on `stream` has finished.
 *   Streams    `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *              stream).  Calls enqueue asynchronously and return at once, except
 *              where an entry point says it is synchronous.
 *   Errors     Every call returns an fb_status.  Arguments are validated before any
 *              work is enqueued; on FB_ERR_ARG nothing was launched.  On any error
 *              fb_last_error() holds a message.  A context owns its scratch memory
 *              and is NOT thread-safe; distinct contexts may be used concurrently.
 *   Determinism  Results are a pure function of the inputs and fb_params: integer
 *              patch distances, counter-based random numbers, one IEEE float
 *              division per output value.
 */
#ifndef FB_H
#define FB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FB_API_VERSION 1

typedef enum fb_status {
    FB_OK = 0,
    FB_ERR_ARG = 1,          /* invalid argument; nothing was enqueued          */
    FB_ERR_CUDA = 2,         /* a CUDA runtime call or kernel launch failed      */
    FB_ERR_OOM = 3,          /* device or pinned-host scratch allocation failed  */
    FB_ERR_TIMEOUT = 4,      /* a bounded device-side wait expired               */
    FB_ERR_UNSUPPORTED = 5   /* valid request this library does not implement    */
} fb_status;

typedef struct fb_ctx fb_ctx;

/* Parameters of Alg. 1 (Sec. 3.2). */
typedef struct fb_params {
    int32_t patch;     /* k = 2p+1 (odd, 3..9)                                         */
    int32_t iters;     /* n: iterations per pyramid level, 0..65534                    */
    int32_t levels;    /* pyramid levels, 1..16; level l has ceil(H/2^l) x ceil(W/2^l)  */
    int32_t r0;        /* first random-search radius; 0 => max(H', W') at each level   */
    uint64_t seed;     /* key of the Philox-4x32-10 stream                             */
    uint32_t pair_tag; /* fb_nnf only: stream id of this pair; fb_pair_tag(j, i) makes  */
                       /* fb_nnf reproduce the NNF that the blend/interpolation calls   */
                       /* compute for source frame j -> target frame i                  */
    uint32_t flags;    /* FB_FLAG_* bits below; 0 = the paper's method                  */
    uint32_t alpha;    /* FB_FLAG_BALANCED / fb_nnf_balanced: integer weight of the      */
                       /* guide term of the improved loss, 0..255; ignored otherwise    */
} fb_params;

/* fb_params.flags.  FB_FLAG_LEARNED_INIT (fb_blend_window, fb_interpolate): start Alg. 1
 * from the learned initialiser attached with fb_ctx_set_initnet instead of the random
 * field (an addition to the paper, see fb_initnet below; levels must be 1).
 * FB_FLAG_REPORT_ENERGY (same calls): accumulate the sum of the final Eq. 1 errors of all
 * NNFs of the call, read with fb_ctx_energy. */
#define FB_FLAG_LEARNED_INIT 0x1u
#define FB_FLAG_REPORT_ENERGY 0x2u
/* FB_FLAG_BALANCED (fb_blend_window only): compute the NNFs with the improved loss of
 * Sec. 3.4 instead of Eq. 1, as fb_nnf_balanced does for each pair (j -> i) with source
 * style S_j; levels must be 1, p->alpha <= 255, not with FB_FLAG_LEARNED_INIT.  The
 * energy that FB_FLAG_REPORT_ENERGY sums is then the improved loss. */
#define FB_FLAG_BALANCED 0x4u
/* FB_FLAG_FAST (fb_blend_window only): the fast mode of Sec. 3.4 -- the window sum of
 * Eq. 2 from a remapping table (Alg. 3), its prefix sums (Alg. 4) and the interval query
 * (Alg. 5) on the clip and on the reversed clip, joined by the split identity; O(N log N)
 * NNFs instead of O(N M).  Each NNF is Alg. 1 with the pair tag of its (source, target)
 * frames.  Results differ from the direct sum (remaps of remapped frames); sums are exact
 * integers and each output value one double division rounded to float.  Not with
 * FB_FLAG_BALANCED or FB_FLAG_LEARNED_INIT; all NNFs of the call are held at once
 * (FB_ERR_UNSUPPORTED beyond the pair budget). */
#define FB_FLAG_FAST 0x8u
/* FB_FLAG_ACCURATE (fb_blend_window only): the quality improvement of Sec. 3.4 -- the
 * NNFs of each output frame i are computed together; at the beginning of every
 * iteration the mean remapped frame Tbar_i = (k^2 S_i + sum_j (S_j -> S_i)) / (k^2 c_i),
 * rounded half up to 8 bits, is rebuilt from the current fields, and every pair (j -> i)
 * takes its Jacobi step under alpha ||G_j[F] - G_i||^2 + ||S_j[F] - Tbar_i||^2 (the
 * incumbent re-evaluated first).  levels must be 1, p->alpha <= 255; not with the other
 * mode flags. */
#define FB_FLAG_ACCURATE 0x10u
/* FB_FLAG_TRACKING (fb_interpolate, and fb_blend_window with the plain loss): the tracking
 * of Sec. 3.5.1 -- the NNFs from one source frame (a keyframe; in a blend, a window's
 * source) to consecutive target frames form a chain, and each pair's updating sequence
 * gains, after propagation and before the random search, the matches of the pairs to the
 * previous and next target frame at the same pixel (previous iteration's snapshot).  No
 * pair maps a frame to itself, so a chain ends next to its source.  levels must be 1; all
 * NNFs of the call are held at once (FB_ERR_UNSUPPORTED beyond the pair budget); not with
 * FB_FLAG_LEARNED_INIT, FB_FLAG_BALANCED, FB_FLAG_FAST or FB_FLAG_ACCURATE. */
#define FB_FLAG_TRACKING 0x20u
/* FB_FLAG_ALIGN (fb_interpolate only): the alignment loss of Sec. 3.5.2 (Eq. 10).  For a
 * frame i between keys l < i < r the NNFs F_l (key l -> i) and F_r (key r -> i) are
 * coupled: a candidate u of F_l costs
 *   alpha * Eq.1(G_l at u, G_i at x) + Eq.1(S_l at u, S_r at F_r(x)),
 * the second term the pairwise patch error between the two keyframe styles, with F_r(x)
 * the partner's match of the previous iteration (Jacobi); symmetrically for F_r.  Frames
 * outside the key range have one key and take the plain loss.  alpha (fb_params.alpha)
 * in [0, 255]; levels must be 1; combines with FB_FLAG_TRACKING only (not with
 * FB_FLAG_REPORT_ENERGY: the stored errors mix the two losses). */
#define FB_FLAG_ALIGN 0x40u

/* Create a context on CUDA device `device` (made current for the call).  The context
 * allocates scratch lazily and keeps it for reuse until fb_ctx_destroy. */
int fb_ctx_create(fb_ctx **out, int device);

/* Free the context and its scratch.  Synchronises the device first.  NULL is a no-op. */
int fb_ctx_destroy(fb_ctx *ctx);

/* Wait for `stream`, then report any error a kernel of this context recorded on the
 * device (FB_ERR_TIMEOUT for an expired bounded wait) and clear it. */
int fb_ctx_sync(fb_ctx *ctx, void *stream);

/* Message for the last failing call on this context ("" if none).  Valid until the
 * next call on the context.  ctx may be NULL (then: last argument error seen by a
 * call made with ctx == NULL). */
const char *fb_last_error(const fb_ctx *ctx);

/* Static name of a status code. */
const char *fb_status_string(int status);

/* Number of kernels this context has launched since creation (diagnostics). */
uint64_t fb_ctx_launches(const fb_ctx *ctx);

/* Device scratch currently held by the context, in bytes. */
size_t fb_ctx_scratch_bytes(const fb_ctx *ctx);

/* Kernel families, for fb_ctx_profile_read. */
typedef enum fb_kernel_kind {
    FB_K_PREP = 0,      /* guide frame -> row patches                            */
    FB_K_DOWNSAMPLE,    /* pyramid step                                          */
    FB_K_STYLE,         /* style frame -> 4-byte pixels                          */
    FB_K_INIT,          /* initial NNF and its Eq. 1 errors                      */
    FB_K_ITER,          /* one Jacobi iteration of Alg. 1 (propagation + search) */
    FB_K_UNPACK,        /* packed NNF -> int32 (row, col)                        */
    FB_K_PACK,          /* int32 (row, col) -> packed NNF                        */
    FB_K_COMBINE,       /* Alg. 2 remap fused with Eq. 2 / keyframe weights      */
    FB_K_INITNET,       /* learned initialiser: network forward + initial fields  */
    FB_K_SHAT,          /* improved loss: remapped source style S^ of every pair  */
    FB_K_ENERGY,        /* improved loss: incumbent's loss against the new S^      */
    FB_K_TABLE,         /* fast mode: blending-table entries                      */
    FB_K_COUNT
} fb_kernel_kind;

/* Diagnostics: enable = 1 clears and starts recording a CUDA event pair around every
 * kernel this context launches (on the caller's stream); enable = 0 stops.  Costs
 * two event records per launch while on. */
int fb_ctx_profile(fb_ctx *ctx, int enable);

/* Waits for the recorded events and writes, per fb_kernel_kind, the summed device
 * time in milliseconds (ms[FB_K_COUNT]) and the number of launches
 * (launches[FB_K_COUNT]) recorded since profiling was last enabled. */
int fb_ctx_profile_read(fb_ctx *ctx, double *ms, uint64_t *launches);

/* Diagnostics: measures the device's throughput of dp4a (four byte products summed
 * into a 32-bit accumulator, the instruction that evaluates Eq. 1) with a
 * register-only kernel on every SM.  Writes dp4a instructions per second and the
 * kernel's duration.  Synchronous.  Not part of the method. */
int fb_probe_dp4a(fb_ctx *ctx, double *dp4a_per_s, double *ms);

/* Diagnostics: measures the device's throughput of the instruction sequence the
 * patch-match kernels evaluate Eq. 1 with, on register operands (no memory traffic) on
 * every SM: for patch = 5 the five 15-byte patch rows as two 32-byte slots and one 16-byte
 * half, three dp4a per 4-byte word (<s, t>, |s|^2, |t|^2); for patch = 7 seven 24-byte
 * rows, three dp4a per word likewise; per slot or row the accumulate and the
 * early-exit compare.  Writes Eq. 1 byte pairs per second (3k^2 per candidate) and the
 * kernel's duration.  This is the ALU roofline of the chosen sequence, below the dp4a-only
 * bound of fb_probe_dp4a (k = 5: 60 dp4a for 75 byte pairs instead of 19).  FB_ERR_ARG for
 * other patch sizes.  Synchronous.  Not part of the method. */
int fb_probe_ssd_mix(fb_ctx *ctx, int patch, double *byte_pairs_per_s, double *ms);

/* Diagnostics: measures the device's rate of scattered 32-byte loads, the traffic of the
 * patch-match kernels (every candidate patch row is a 256-bit load of a 32-byte row-patch
 * slot at a data-dependent address): 5 resident 256-thread blocks per SM (40 warps, the
 * k = 5 iteration kernel's occupancy), each thread issuing independent 256-bit loads of
 * pseudo-randomly chosen slots of a `bytes`-sized buffer in the context's scratch.  A
 * buffer that fits L1 measures the L1 data pipe (one 32-byte sector per wavefront); a
 * larger one adds the L2.  Writes 32-byte sectors per second and the kernel's duration.
 * bytes: a power of two in [1 KiB, 1 GiB] (FB_ERR_ARG otherwise).  Synchronous.  Not part
 * of the method. */
int fb_probe_gather(fb_ctx *ctx, size_t bytes, double *sectors_per_s, double *ms);

/* Diagnostics of debug builds: libfb_debug.so (compiled with FB_COUNT_EVALS) counts,
 * in a device-global counter, every candidate the per-call NNF kernels consider -- one
 * per pixel and level for the initial match, then per pixel and iteration one per
 * propagation neighbour inside the image and one per random-search radius, duplicates
 * of the running best included (Alg. 1).  Writes the count accumulated since the last
 * reset and resets it if `reset` is non-zero; synchronous; device of the current
 * context.  The product libfb.so returns FB_ERR_UNSUPPORTED. */
int fb_debug_candidates_considered(uint64_t *count, int reset);

/* Checked builds: libfb_checked.so (compiled with FB_CHECKED) tests, on the device, the
 * index and data invariants the NNF kernels rely on, at the sites below.  A failed check
 * never traps: it records the first failure, counts it, and skips the access or the
 * candidate it guards (a remap match is clamped as in every build), so the kernel runs to
 * its end.  The sites:
 *   FB_CHECK_CANDIDATE  a candidate match outside the image       (a = row, b = column)
 *   FB_CHECK_SNAPSHOT   a stored match -- snapshot, coarser level, chain neighbour or
 *                       partner -- outside its image              (a = row, b = column)
 *   FB_CHECK_ENERGY     a stored error that is not the loss of its stored match (the
 *                       Jacobi snapshot invariant E = L(F); a race or a stale buffer
 *                       breaks it)                                (a = stored, b = loss)
 *   FB_CHECK_SLOT       a paired row-patch slot row past the frame (a = slot row,
 *                                                                  b = slot rows)
 *   FB_CHECK_TABLE      a chain-neighbour or partner pair outside the launch
 *                                                                 (a = pair, b = index)
 *   FB_CHECK_REMAP      a match the remap (Alg. 2) reads outside the image
 *                                                                 (a = row, b = column) */
#define FB_CHECK_CANDIDATE 1u
#define FB_CHECK_SNAPSHOT 2u
#define FB_CHECK_ENERGY 3u
#define FB_CHECK_SLOT 4u
#define FB_CHECK_TABLE 5u
#define FB_CHECK_REMAP 6u

/* State of the device-side checks of a checked build on the current device, summed over
 * the per-call and the batched kernels:
 *   first      0, or the first failed check as (site << 56) | (a << 28) | b, with a and b
 *              the low 28 bits of the site's two values (nullable)
 *   failed     failed checks (nullable)
 *   evaluated  pixel visits that ran the checks: one per pixel per NNF kernel launch and
 *              one per remapped pixel per pair (nullable)
 * reset != 0 zeroes all three after reading.  Synchronous; synchronise the streams of the
 * checked calls first.  The product libfb.so returns FB_ERR_UNSUPPORTED. */
int fb_check_status(uint64_t *first, uint64_t *failed, uint64_t *evaluated, int reset);

/* Philox stream id of the ordered pair (source frame j -> target frame i), as used
 * by fb_blend_window and fb_interpolate: (j << 16) | i. */
uint32_t fb_pair_tag(int j, int i);

/* NNF(S, T) by Alg. 1 (Sec. 3.2) with the Eq. 1 loss, for one source guide
 * `src_guide` and one target guide `tgt_guide`, both H x W x 3.
 *   init_nnf  NULL => Philox random initialisation at the coarsest level; else an
 *             H x W x 2 int32 initial field (requires p->levels == 1; entries are
 *             clamped into the image).
 *   nnf_out   H x W x 2 int32 (written).     err_out  H x W uint32 or NULL.
 * Schedule: every iteration updates all pixels from a snapshot of the previous
 * iteration (Sec. 3.2, parallel update); per pixel the candidates are the four
 * propagation candidates F(x+d) - d, d = (-1,0), (1,0), (0,-1), (0,1), then the random
 * search candidates best + U[-r, r]^2 for r = r0, r0/2, ..., 1; a candidate wins only
 * with a strictly smaller error.  Async on `stream`. */
int fb_nnf(fb_ctx *ctx, const uint8_t *src_guide, const uint8_t *tgt_guide, int H, int W,
           const fb_params *p, const int32_t *init_nnf, int32_t *nnf_out, uint32_t *err_out,
           void *stream);

/* One Jacobi iteration of Alg. 1 (Sec. 3.2 parallel update) from a caller's snapshot:
 * the step fb_nnf takes as its iteration `it` (0-based) at the finest level, on the same
 * candidates, random stream (p->seed, p->pair_tag, it) and strict acceptance.
 *   nnf_in   H x W x 2 int32 snapshot field (device); entries are clamped into the image.
 *   err_in   H x W uint32 (device): the incumbents' errors, taken as given.  Only with
 *            err_in = Eq. 1 of the (clamped) nnf_in is the step Alg. 1's; with that, the
 *            output after iteration it - 1 of fb_nnf (levels = 1) stepped with `it` is
 *            bit-identical to fb_nnf's output after iteration it.  Checked builds
 *            (libfb_checked.so) verify the identity per pixel (FB_CHECK_ENERGY).
 *   nnf_out, err_out  H x W x 2 int32 and H x W uint32 (device, written; may be nnf_in
 *            and err_in: the snapshot is copied before the step).
 *   p        patch, r0, seed and pair_tag are used; levels must be 1 and flags 0 (plain
 *            loss), FB_ERR_ARG otherwise; iters is ignored.  it in [0, 65534].
 * Async on `stream`. */
int fb_nnf_step(fb_ctx *ctx, const uint8_t *src_guide, const uint8_t *tgt_guide, int H, int W,
                const fb_params *p, int it, const int32_t *nnf_in, const uint32_t *err_in,
                int32_t *nnf_out, uint32_t *err_out, void *stream);

/* Alg. 1 under the improved loss of Sec. 3.4 ("balanced mode") for one pair:
 *   L(x) = alpha ||G_src[F(x)] - G_tgt[x]||^2 + ||S_src[F(x)] - S^[x]||^2
 * over k x k RGB patches (clamp-to-edge), S^ = the Alg. 2 remap of src_style through the
 * current field rounded half up to 8 bits, refreshed at the beginning of every
 * iteration; the incumbent's loss is re-evaluated against the refreshed S^ before the
 * iteration's candidates (same schedule, order, random stream and strict acceptance as
 * fb_nnf) are compared with it.  With iters = 0, err_out is the loss of the initial
 * field against the S^ it implies.
 *   src_style  H x W x 3 uint8, the style frame that goes with src_guide (device).
 *   p          levels must be 1; p->alpha in [0, 255]; p->flags ignored.
 *   shat_out   H x W x 3 uint8 or NULL: the S^ of the last iteration.
 * Other arguments and errors as fb_nnf.  Async on `stream`. */
int fb_nnf_balanced(fb_ctx *ctx, const uint8_t *src_guide, const uint8_t *tgt_guide,
                    const uint8_t *src_style, int H, int W, const fb_params *p,
                    const int32_t *init_nnf, int32_t *nnf_out, uint32_t *err_out,
                    uint8_t *shat_out, void *stream);

/* Sec. 3.5.2 alignment (Eq. 10) and Sec. 3.5.1 tracking at the level of the fields: the
 * NNFs from the two keyframes at the ends of a clip segment to every frame between them,
 * as fb_interpolate computes them for a pair of consecutive keys.
 *   guides      (n + 2) x H x W x 3 uint8 (device): key l, the n frames between, key r.
 *   key_styles  2 x H x W x 3 uint8 (device): S_l, S_r.
 *   n           frames between the keys, in [1, 32767].
 *   p           levels must be 1; p->flags: FB_FLAG_ALIGN (coupled loss, p->alpha in
 *               [0, 255]) and / or FB_FLAG_TRACKING; with neither, the 2n independent
 *               Alg. 1 fields.  Pair (0 -> q) and (n + 1 -> q), q = 1..n, draw the
 *               random streams of fb_pair_tag(0, q) and fb_pair_tag(n + 1, q).
 *   init        2n x H x W x 2 int32 initial fields (device, clamped into the image) or
 *               NULL for the random initialisation.
 *   nnf_out     2n x H x W x 2 int32 (device): the fields of key l to frames 1..n, then
 *               those of key r.
 *   err_out     2n x H x W uint32 (device) or NULL: the loss each final match was last
 *               compared under (the coupled loss of Eq. 10 with FB_FLAG_ALIGN, else Eq. 1).
 *               With FB_FLAG_ALIGN it needs iters >= 1 (FB_ERR_ARG otherwise).
 * Errors as fb_nnf; the 2n fields are held at once (no pair budget).  Async on `stream`. */
int fb_nnf_segment(fb_ctx *ctx, const uint8_t *guides, const uint8_t *key_styles, int n, int H,
                   int W, const fb_params *p, const int32_t *init, int32_t *nnf_out,
                   uint32_t *err_out, void *stream);

/* Alg. 2 (Sec. 3.3), memory-efficient remap of `src_style` (H x W x 3) through `nnf`
 * (H x W x 2 int32, entries clamped into the image):
 *   out(x) = sum over the k x k neighbours q of x of S(F(q^) - (q^ - x)) / (255 k^2),
 * with q^ = q clamped into the image and the source index clamped into the image.
 * out: H x W x 3 float32.  No patch tensor is formed: O(HW) memory.  Async. */
int fb_remap(fb_ctx *ctx, const uint8_t *src_style, const int32_t *nnf, int H, int W,
             int patch, float *out, void *stream);

/* Eq. 2 (Sec. 3.4): sliding-window blend of N style frames guided by N guide frames.
 * For each frame i the window [i-M, i+M], M = (window-1)/2, is truncated to the clip;
 *   out_i = (S_i + sum_{j in window, j != i} (S_j -> S_i)) / (frames in window),
 * where (S_j -> S_i) is the Alg. 2 remap of S_j through NNF(G_j, G_i) computed by
 * Alg. 1 with pair tag fb_pair_tag(j, i).  window must be odd and >= 1.
 *   guides, styles: N x H x W x 3 uint8;  out: N x H x W x 3 float32.
 * Pointers are either all device pointers (async) or all host pointers; with host
 * pointers the call stages the data through the context and returns when `out` is
 * filled (pinned host memory makes the copies faster; pageable memory works). */
int fb_blend_window(fb_ctx *ctx, const uint8_t *guides, const uint8_t *styles, int N, int H,
                    int W, int window, const fb_params *p, float *out, void *stream);

/* Sec. 3.5.2: render every frame of an N-frame guide video from stylised keyframes.
 *   key_idx     HOST array of n_keys strictly increasing frame indices in [0, N).
 *   key_styles  n_keys x H x W x 3 uint8, keyframe m's style at key_idx[m].
 * For l < i < r consecutive keys:
 *   out_i = ((r - i)(S_l -> G_i) + (i - l)(S_r -> G_i)) / (r - l);
 * keyframes are output unchanged (S/255); frames before the first / after the last
 * key use that key alone.  n_keys == 1 renders the whole video from one frame.
 * Memory rules as fb_blend_window (device => async, host => synchronous). */
int fb_interpolate(fb_ctx *ctx, const uint8_t *guides, int N, int H, int W,
                   const int32_t *key_idx, const uint8_t *key_styles, int n_keys,
                   const fb_params *p, float *out, void *stream);

/* Output-frame ranges of one clip, for splitting a clip across GPUs (one process per GPU,
 * each blending its own range; no data exchange between them).  Every output frame of
 * Eq. 2 depends only on the frames of its window [i - M, i + M] (Sec. 3.4), so a range of
 * output frames [a, b) needs only the input frames [a - M, b + M) (clipped to the clip):
 * the range plus an M-frame halo on either side.  Each NNF keeps the random stream of its
 * clip frames, fb_pair_tag(j, i), so the range's output frames are bit-identical to the
 * same frames of fb_blend_window over the whole clip.
 *   n_total     frames in the whole clip (the windows are truncated at its ends).
 *   frame_base  clip index of guides[0] / styles[0]; the call holds n_in frames,
 *               clip frames [frame_base, frame_base + n_in).
 *   out_first, n_out  the output frames [out_first, out_first + n_out) (clip indices);
 *               out holds n_out frames, n_out x H x W x 3 float32.
 * FB_ERR_ARG when an output frame's window reaches outside the held input frames.
 * Modes: plain, FB_FLAG_BALANCED, FB_FLAG_ACCURATE (its mean frame couples only the NNFs
 * of one output frame), FB_FLAG_LEARNED_INIT, FB_FLAG_REPORT_ENERGY.  FB_FLAG_FAST and
 * FB_FLAG_TRACKING couple output frames across the clip: FB_ERR_UNSUPPORTED.  Memory
 * rules and everything else as fb_blend_window. */
int fb_blend_window_range(fb_ctx *ctx, const uint8_t *guides, const uint8_t *styles, int n_in,
                          int H, int W, int window, const fb_params *p, int n_total,
                          int frame_base, int out_first, int n_out, float *out, void *stream);

/* The output frames [out_first, out_first + n_out) of fb_interpolate over the whole
 * N-frame clip (Sec. 3.5.2: every frame depends only on its keys), bit-identical to those
 * frames of the whole-clip call.  guides holds all N frames (the keys are the sources);
 * out holds n_out frames.  FB_FLAG_ALIGN is supported (its two coupled NNFs belong to
 * the same output frame); FB_FLAG_TRACKING is not (FB_ERR_UNSUPPORTED).  Other arguments
 * as fb_interpolate. */
int fb_interpolate_range(fb_ctx *ctx, const uint8_t *guides, int N, int H, int W,
                         const int32_t *key_idx, const uint8_t *key_styles, int n_keys,
                         const fb_params *p, int out_first, int n_out, float *out, void *stream);

/* Host-only split of an N-frame clip into n_shards contiguous ranges of output frames of
 * about equal work (blend, window > 0: an output frame's work is its NNFs plus its
 * combine; interpolation, window = 0: one unit per frame), for shard `shard` in
 * [0, n_shards): the output range [*out_first, *out_first + *n_out) (never empty) and
 * the input frames [*frame_base, *frame_base + *n_in) that fb_blend_window_range needs
 * for it (the range plus the (window - 1) / 2 halo, clipped; interpolation: the whole
 * clip).  The shards cover every output frame exactly once.  No CUDA calls; FB_ERR_ARG
 * for N outside [1, 65535], an even or negative window, n_shards outside [1, N] or shard
 * outside [0, n_shards). */
int fb_shard_plan(int N, int window, int n_shards, int shard, int *frame_base, int *n_in,
                  int *out_first, int *n_out);

/* One clip of a batched submission (fb_blend_batch).  All pointers are device
 * pointers of the context's device, owned by the caller. */
typedef struct fb_clip_desc {
    const uint8_t *guides;  /* N x H x W x 3 guide frames                        */
    const uint8_t *styles;  /* N x H x W x 3 style frames                        */
    float *out;             /* N x H x W x 3 output, float32 in [0, 1]           */
    int32_t N, H, W;        /* 1 <= N <= 65535; patch <= H, W <= 32767            */
    int32_t window;         /* odd, >= 1 (Eq. 2, truncated at the clip ends)     */
    int32_t patch;          /* odd, 3..9                                         */
    int32_t reserved;       /* must be 0                                         */
} fb_clip_desc;

#define FB_BATCH_NO_GRAPH 0x1u            /* launch directly, do not capture/replay */
#define FB_BATCH_VARIANT(v) (((uint32_t)(v) + 1u) << 8)  /* force tile variant v (0..3) */
#define FB_BATCH_CLAIM(c) ((uint32_t)(c) << 16)  /* force c tiles per iteration claim (1..64) */
#define FB_BATCH_PERSISTENT (1u << 24)  /* force the persistent kernels for every patch size */
#define FB_BATCH_PER_CLIP (2u << 24)    /* force per-clip launches for every patch size       */

/* Eq. 2 window blends of n_clips clips of uneven size, window and patch in one
 * submission.  This batched, persistent form is not in the paper; the paper only
 * notes that images are processed in batches (Sec. 3.2) and that a task manager
 * schedules the NNF tasks (Sec. 3.4.1).  Each clip's output is bit-identical to
 * fb_blend_window on that clip with the same fb_params (p->patch is ignored: every
 * clip carries its own patch; p->levels must be 1).
 *   clips  HOST array of n_clips descriptors (copied; need not outlive the call).
 * Mechanics: all NNFs of all clips are cut into 32-column tiles and processed by
 * persistent kernels (grid = SMs x resident blocks) that walk a flattened work list,
 * one launch per Jacobi iteration and patch size, in chunks whose NNF buffers fit the
 * pair budget.  The first submission of a given manifest (pointers, shapes, params)
 * tunes the tile shape / occupancy per patch size on a few iterations of the size's
 * first chunk (all variants give identical results), then captures the whole
 * submission into a CUDA graph that later submissions with the same manifest replay
 * (FB_BATCH_NO_GRAPH: direct launches).  The tuner chooses, per patch size, the tile
 * shape / occupancy variant and the number of consecutive tiles one claim of the
 * iteration kernel covers (1, 2, 4 or 8), timing every combination on a prefix of the
 * size's first chunk, and then the launch mode: those persistent kernels, or per-clip
 * launches of the kernels fb_blend_window uses (one clip segment after another, spread
 * over three branches of the graph so that one clip's launch tails overlap the next clip's
 * work), whichever ran the same prefix faster.  FB_BATCH_VARIANT / FB_BATCH_CLAIM force
 * the persistent kernels with that variant / claim; FB_BATCH_PERSISTENT /
 * FB_BATCH_PER_CLIP force the mode.  The context keeps the tables, scratch and graph of the two most recent
 * manifests.  Async on `stream`; do not call it while `stream` is being captured. */
int fb_blend_batch(fb_ctx *ctx, const fb_clip_desc *clips, int n_clips, const fb_params *p,
                   uint32_t flags, void *stream);

/* One NNF of a blend or interpolation call, as the call enumerates it (host-only). */
typedef struct fb_pair_info {
    int32_t src;        /* source frame j (blend) or keyframe l / r (interpolation) */
    int32_t tgt;        /* target frame i: the output frame the NNF is remapped into */
    uint32_t tag;       /* fb_pair_tag(src, tgt): its random stream */
    uint32_t weight;    /* integer weight of its remapped style in frame tgt's numerator
                           (blend: 1; interpolation: Eq. 9's r - i or i - l, or 1) */
    int32_t prev, next; /* FB_FLAG_TRACKING: the pairs (src -> tgt - 1), (src -> tgt + 1),
                           or -1 */
    int32_t partner;    /* FB_FLAG_ALIGN: the other key's pair to tgt, or -1 */
    int32_t out_frame;  /* = tgt */
} fb_pair_info;

/* Host-only enumeration of the NNFs of a call (no CUDA calls), in the order the call
 * computes them: grouped by output frame in increasing order; within a frame, sources in
 * increasing order (blend) or the left key before the right key (interpolation).
 *   window > 0: fb_blend_window's pairs (j -> i), 0 < |i - j| <= (window - 1) / 2 inside
 *               the clip (key_idx NULL, n_keys 0, window odd).
 *   window = 0: fb_interpolate's pairs for the sorted keys key_idx[0..n_keys).
 *   flags: FB_FLAG_TRACKING and / or (interpolation) FB_FLAG_ALIGN fill prev / next /
 *          partner as the tracking and alignment kernels use them.
 * *n_pairs receives the count; out (capacity cap) may be NULL to query it.  FB_ERR_ARG
 * for invalid arguments or cap below the count. */
int fb_pair_plan(int N, int window, const int32_t *key_idx, int n_keys, uint32_t flags,
                 fb_pair_info *out, size_t cap, size_t *n_pairs);

/* The NNFs of fb_blend_window_range / fb_interpolate_range for the output frames
 * [out_first, out_first + n_out) of an N-frame clip, in their order, with clip frame
 * indices (src, tgt and out_frame) as fb_pair_plan gives them: exactly the entries of
 * fb_pair_plan over the whole clip whose out_frame lies in the range, except that
 * `partner` indexes this list (prev / next are -1: tracking has no range form).  flags: 0 or
 * (interpolation) FB_FLAG_ALIGN.  Host only; errors as fb_pair_plan, and FB_ERR_ARG for a
 * range outside the clip. */
int fb_pair_plan_range(int N, int window, const int32_t *key_idx, int n_keys, uint32_t flags,
                       int out_first, int n_out, fb_pair_info *out, size_t cap, size_t *n_pairs);

/* Host-only planning of the fast mode (FB_FLAG_FAST) for N frames and `window`: the
 * number of distinct NNFs it computes, of blending-table entries it builds and of query
 * pieces it remaps (the direct sum of Eq. 2 computes sum_i (window_i - 1) NNFs).  No CUDA
 * calls; FB_ERR_ARG for N outside [1, 65535] or an even / non-positive window. */
int fb_fast_plan(int N, int window, uint64_t *n_nnfs, uint64_t *n_entries, uint64_t *n_pieces);

/* Host-only planning of a batch (no CUDA calls): number of NNFs, persistent-kernel work
 * items per iteration (32x8 tiles) and chunks under a pair budget of budget_bytes of
 * NNF scratch (0 = the library's default). */
int fb_batch_plan(const fb_clip_desc *clips, int n_clips, const fb_params *p, size_t budget_bytes,
                  uint64_t *n_pairs, uint64_t *n_items, int *n_chunks);

/* Bytes of NNF scratch (four H x W words per NNF) one chunk of pairs may use in this
 * context's blend, interpolation and batch calls (0 = the default, 8 GiB; minimum
 * 1 MiB).  Larger inputs run in more chunks; results do not depend on it. */
int fb_ctx_set_pair_budget(fb_ctx *ctx, size_t bytes);

/* Sum and number of the final Eq. 1 errors accumulated by the last call made with
 * FB_FLAG_REPORT_ENERGY (waits for the device). */
int fb_ctx_energy(fb_ctx *ctx, double *sum, uint64_t *count);

/* Tile variant the autotuner chose for patch size k in this context, or -1. */
int fb_ctx_batch_variant(const fb_ctx *ctx, int patch);

/* Tiles per iteration claim the autotuner chose for patch size k in this context, or -1. */
int fb_ctx_batch_claim(const fb_ctx *ctx, int patch);

/* Launch mode the autotuner chose for patch size k in this context: 0 persistent kernels,
 * 1 per-clip launches, -1 not tuned. */
int fb_ctx_batch_mode(const fb_ctx *ctx, int patch);

/* ---------------------------------------------------------------------------------
 * Learned NNF initialiser.  Not in the paper (its method is model-free and needs no
 * training, Sec. 3.1): a small BF16 convolutional pyramid that maps a pair of guide
 * frames (source, target) at 1/4 or 1/8 of their resolution to an offset field, trained
 * on NNFs that Alg. 1 itself computes, so that Alg. 1 can start near its answer and run
 * fewer iterations.  Convolutions run on the tcgen05 tensor cores (BF16 operands, FP32
 * accumulation); forward, backward and the Adam update are this library's kernels.
 * Architecture: 12 3x3 conv layers (encoder 8->32->32, ->64/2->64, ->96/2->96,
 * ->128/2->128; decoder with nearest upsampling and skip concatenation 224->96,
 * 160->64, 96->32; head 32->8 of which channels 0,1 are the (row, col) offset / 16 in
 * full-resolution pixels), ReLU except on the head; 779,592 parameters.  The network
 * runs at Hq x Wq = H/D x W/D for a downscale D in {4, 8} (D x D box means of the
 * guides); H and W must be multiples of 8 D.  All pointers are device pointers unless
 * stated.  A net belongs to the device current at creation; not thread-safe.
 * --------------------------------------------------------------------------------- */
typedef struct fb_initnet fb_initnet;

/* Allocate a net for up to max_pairs pairs of H x W frames at downscale D (4 or 8);
 * parameters start at zero: set them with fb_initnet_set_params.  FB_ERR_ARG if H or W
 * is not a multiple of 8 D. */
int fb_initnet_create(fb_ctx *ctx, fb_initnet **out, int max_pairs, int H, int W, int downscale);
int fb_initnet_destroy(fb_initnet *net);
const char *fb_initnet_last_error(const fb_initnet *net);

/* Number of FP32 parameters, laid out per layer as weights [Cout][3][3][Cin] then biases
 * [Cout]; get/set copy them between the device and a HOST array of that length (set
 * also resets the Adam state). */
size_t fb_initnet_param_count(const fb_initnet *net);
int fb_initnet_get_params(fb_initnet *net, float *host_out);
int fb_initnet_set_params(fb_initnet *net, const float *host_in);
/* Gradient of the last train step, same layout, to a HOST array. */
int fb_initnet_get_grads(fb_initnet *net, float *host_out);
/* Adam state, for checkpoint / resume: the first and second moment estimates (HOST arrays
 * of fb_initnet_param_count floats, parameter layout) and the number of updates taken.
 * Set after fb_initnet_set_params, which resets them.  FB_ERR_ARG for NULL arrays. */
int fb_initnet_get_optimizer(fb_initnet *net, float *m_out, float *v_out, uint64_t *step_out);
int fb_initnet_set_optimizer(fb_initnet *net, const float *m_in, const float *v_in, uint64_t step);

/* Forward pass for n pairs: src, tgt are n x H x W x 3 uint8 stacks (pair p = source
 * frame src[p] -> target frame tgt[p]).  head_out (nullable): n x Hq x Wq x 8 float,
 * channels 0,1 = predicted (row, col) offset / 16.  Async on `stream`. */
int fb_initnet_forward(fb_initnet *net, const uint8_t *src, const uint8_t *tgt, int n,
                       float *head_out, void *stream);

/* Initial NNF of the n pairs of the last forward pass: F0(x) = clamp(x + rint(16 *
 * head(x / D))), written as n x H x W x 2 int32.  Async. */
int fb_initnet_init_nnf(fb_initnet *net, int n, int32_t *nnf_out, void *stream);

/* One training step on n pairs: forward, smooth-L1 loss (1 pixel transition) between
 * 16 * head[..., 0:2] and `target` (n x Hq x Wq x 2 float, full-resolution pixels)
 * weighted by `weight` (n x Hq x Wq float, or NULL = 1) and divided by weight_sum,
 * backward, and an Adam update with step size lr (lr = 0: gradients only).  The loss
 * is written to the device float *loss_out (nullable).  Async. */
int fb_initnet_train_step(fb_initnet *net, const uint8_t *src, const uint8_t *tgt, int n,
                          const float *target, const float *weight, float weight_sum, float lr,
                          float *loss_out, void *stream);

/* Attach (or with NULL detach) the learned initialiser used by FB_FLAG_LEARNED_INIT. */
int fb_ctx_set_initnet(fb_ctx *ctx, fb_initnet *net);

/* Training targets from fields computed by Alg. 1 (nnf: n x H x W x 2 int32): per D x D
 * block the mean offset F(x) - x (target, n x H/D x W/D x 2 float) and weight 1 where
 * every offset of the block lies within D/2 pixels of that mean, else 0 (weight,
 * nullable).  D = downscale, 4 or 8.  Async. */
int fb_initnet_targets(const int32_t *nnf, int n, int H, int W, int downscale, float *target,
                       float *weight, void *stream);

/* FB_ERR_TIMEOUT if a tensor-core kernel of this net hit its bounded wait since the last
 * call (the flag is then cleared), else FB_OK.  Synchronous.  Outputs of the pass that
 * timed out are undefined; the net stays usable. */
int fb_initnet_status(fb_initnet *net);

/* Diagnostics (failure detection): the number of polls a tensor-core kernel's progress
 * wait (operands landed, a pipeline stage free, the accumulator complete) makes on the
 * current device before the CTA gives up, drains the MMAs it committed and the copies it
 * issued (those waits keep the full limit), skips its epilogue, releases its tensor memory
 * and raises the net's timeout flag (fb_initnet_status).  polls = 0 makes every progress
 * wait give up at once, so a forward or training pass reports FB_ERR_TIMEOUT without any
 * fault; polls < 0 restores the default (2^26, far beyond any real wait).  Waits for the
 * device before and after; call it with no other work of this library in flight.  Not
 * part of the method. */
int fb_debug_set_wait_limit(int64_t polls);

/* Single 3x3 convolution layer (zero padding 1) on the tensor cores, for tests:
 *   x   n x H x W x Cin bf16 (uint16 storage), w Cout x 3 x 3 x Cin bf16, bias Cout f32,
 *   y   n x Ho x Wo x Cout, Ho = ceil(H / stride): bf16 (y_bf16) or f32 (y_f32, no ReLU
 *       applied to the f32 output when relu = 0).
 * Backward: dz = gradient at the pre-activation output (bf16), wt = the weights
 * transposed to Cin x 3 x 3 x Cout (bf16); dx (nullable) n x H x W x Cin f32 written;
 * dw (nullable) Cout x 3 x 3 x Cin f32 ADDED to.  Cin, Cout multiples of 8, Cout <= 128.
 * status: device int set to 1 if a bounded wait expired.  Async. */
int fb_conv3x3_forward(const uint16_t *x, int n, int H, int W, int Cin, const uint16_t *w,
                       const float *bias, int Cout, int stride, int relu, uint16_t *y_bf16,
                       float *y_f32, int *status, void *stream);
int fb_conv3x3_backward(const uint16_t *x, int n, int H, int W, int Cin, const uint16_t *wt,
                        int Cout, int stride, const uint16_t *dz, float *dx, float *dw,
                        int *status, void *stream);

/* Operand staging of the initialiser's convolutions (process-wide; for tests and
 * measurement).  Layers whose output rows tile 128-pixel blocks stage both operands with
 * tiled TMA loads (the activation box displaced per tap and traversed with the layer's
 * stride, zero-filled outside the image, swizzled rows); other layers gather them with
 * cp.async.  mode 0 (default): the TMA-fed forward and stride-1 input gradients whose
 * tiles are whole rows of one image with a width divisible by 8 and Cin % 32 == 0 load one
 * halo box of R + 2 rows per tap column and channel block and take the three row taps as
 * views into it (the same products in another order: equal to fp32 rounding); the TMA-fed
 * weight gradients run.  mode 2: every TMA-fed convolution loads one box per tap, which
 * accumulates the same products in the same order as the gathers (identical outputs).
 * mode 1: gathers only.  mode -1 leaves the setting; *tma_launches (nullable) receives the
 * number of TMA-staged launches so far.  FB_ERR_ARG for other modes. */
int fb_conv_gemm_path(int mode, uint64_t *tma_launches);

/* Bytes of the fixed device scratch array used by fb_blend_window_noalloc. */
#define FB_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)

/* fb_blend_window without a context or any device allocation, for callers that cannot
 * allocate device memory.  The paper has no counterpart to this entry point.  Some
 * callers are not allowed to call cudaMalloc or any allocator where they
 * blend (a host callback or stream-ordered pipeline that must not synchronise the
 * device, a plug-in whose host application owns all device memory, a process held to
 * a device-memory budget fixed at start-up), and every other entry point here needs a
 * context that allocates.  This one takes no context and allocates nothing: all its
 * scratch lives in one file-scope device array of FB_NOALLOC_SCRATCH_BYTES (64 MiB),
 * which every GPU that loads libfb.so holds until the process exits.
 *   Arguments and result are those of fb_blend_window, on the CURRENT device; guides,
 *   styles and out must be device memory of that device (host pointers -> FB_ERR_ARG).
 *   A blend whose scratch (row patches and styles of N frames at every
 *   pyramid level, four H x W words per NNF, the pair tables) exceeds the array is
 *   rejected with FB_ERR_ARG and a message giving both sizes; so is one with more than
 *   65535 NNFs.  Errors are reported through fb_last_error(NULL).
 *   Set-up: every call looks up the array's device address on the current device
 *   (cudaGetSymbolAddress; a host-side lookup, so the address is never stale, even after
 *   a device reset); the first call on a device also loads the library's device code
 *   there, so make that first call before any stream capture.
 *   Sharing: every call on a device uses the same array and leaves its contents
 *   behind; nothing in it needs to start at zero (every word is written before it is
 *   read).  Calls whose work overlaps on the GPU (different streams, or host threads
 *   without ordering) race on the array and corrupt each other's results: order them.
 *   Results are bit-identical to fb_blend_window.  Async on `stream`. */
int fb_blend_window_noalloc(const uint8_t *guides, const uint8_t *styles, int N, int H, int W,
                            int window, const fb_params *p, float *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FB_H */
