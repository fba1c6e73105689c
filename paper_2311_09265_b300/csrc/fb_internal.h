// fb_internal.h -- host-side declarations shared by the kernels and the C-ABI layer
// of libfb.so.  Not part of the public interface (that is include/fb.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "fb.h"

namespace fb {

// NNF entries on the device are packed (row << 16) | col; H, W <= 32767.
// Guide frames are pre-laid out as "row patches": the row patch of (r, c) is the k
// pixels (r, clamp(c-p .. c+p)) as 3k bytes in rowpatch_words(k) 32-bit words (zero
// padded), so one patch row of Eq. 1 is one aligned 16- or 32-byte load.
//   k = 5 ("paired"): one 32-byte slot per column c and row pair q = 0 .. (H+3)/2,
//     holding the row patches of rows clamp(2q-2) and clamp(2q-1): the rows -2 .. H+1
//     that a clamped 5x5 patch can touch are all present, and one load brings two rows.
//   other k: one slot per pixel holding the row patch of (r, c).
__host__ __device__ constexpr int rowpatch_words(int k) { return ((3 * k + 3) / 4 + 3) / 4 * 4; }
__host__ __device__ constexpr bool rowpatch_paired(int k) { return k == 5; }
__host__ __device__ constexpr int rowpatch_pair_rows(int H) { return (H + 5) / 2; }
// 32-bit words of one guide frame's row patches.
__host__ __device__ inline size_t rowpatch_frame_words(int k, int H, int W) {
    return rowpatch_paired(k) ? static_cast<size_t>(rowpatch_pair_rows(H)) * W * 8
                              : static_cast<size_t>(H) * W * rowpatch_words(k);
}

// One ordered pair (source guide frame -> target guide frame) and how its remap
// enters the output.
struct PairDesc {
    int32_t src;       // guide slot of the source frame (G_j)
    int32_t tgt;       // guide slot of the target frame (G_i)
    uint32_t tag;      // Philox stream id of the pair
    int32_t style;     // style slot remapped through this pair's NNF
    uint32_t weight;   // integer weight of the remapped style in the output numerator
    int32_t pad[3];    // tracking and alignment kernels only: pad[0] / pad[1] = chain
                       // neighbours (pair indices for targets tgt - 1 / tgt + 1, or -1);
                       // pad[2] = the alignment partner (the other key's pair to tgt, or -1)
};

// One output frame: out = (self_w * S_self * k^2 / k^2 ... ) see combine kernel.
struct JobDesc {
    int32_t out_frame;   // index of the output frame
    int32_t self_style;  // style slot added with weight self_w * k^2, or -1
    uint32_t self_w;     // weight of the un-remapped self style (before the k^2 factor)
    int32_t first_pair;  // first pair (global index) of this output frame
    int32_t n_pairs;     // number of consecutive pairs
    uint32_t den;        // integer denominator (255 k^2 * total weight)
    int32_t pad[2];
};

struct LevelGeom {
    int H, W;
    const uint32_t* rp;      // n_guides frames of rowpatch_frame_words(k, H, W) words
};

// Adds n kernel launches made on behalf of ctx to its launch counter (fb_api.cu).
void count_launches(fb_ctx* ctx, int n);

// ---- launchers (fb_kernels.cu); each returns the cudaError_t of the launch ------
cudaError_t launch_prep_guides(int k, const uint8_t* frames, int n_frames, int H, int W,
                               uint32_t* rp, cudaStream_t st);
cudaError_t launch_downsample(const uint8_t* in, int n_frames, int H, int W, uint8_t* out,
                              cudaStream_t st);
cudaError_t launch_style_rgbx(const uint8_t* in, size_t n_px, uint32_t* out, cudaStream_t st);

// mode 0: Philox random init; 1: upsample from the coarse field; 2: user int32 field.
cudaError_t launch_nnf_init(int k, const PairDesc* pairs, int pair0, int n_pairs,
                            const LevelGeom& g, int mode, const uint32_t* coarse_F, int Hc,
                            int Wc, const int32_t* user_init, uint64_t seed, int level,
                            uint32_t* F, uint32_t* E, cudaStream_t st);
cudaError_t launch_nnf_iter(int k, const PairDesc* pairs, int pair0, int n_pairs,
                            const LevelGeom& g, int r0, uint64_t seed, int level, int it,
                            const uint32_t* Fp, const uint32_t* Ep, uint32_t* Fn, uint32_t* En,
                            cudaStream_t st);
cudaError_t launch_nnf_unpack(const uint32_t* F, const uint32_t* E, size_t npx, int32_t* nnf_out,
                              uint32_t* err_out, cudaStream_t st);
cudaError_t launch_nnf_pack(const int32_t* nnf, int H, int W, uint32_t* F, cudaStream_t st);
// Tracking (Sec. 3.5.1), level 0: one Jacobi iteration of the launch's pairs in which a
// pair's pad[0] / pad[1] (pair indices of the same launch, -1 for none) name its chain
// neighbours, whose matches at the same pixel are tried after propagation.
cudaError_t launch_nnf_iter_track(int k, const PairDesc* pairs, int pair0, int n_pairs, const LevelGeom& g,
                                  int r0, uint64_t seed, int it, const uint32_t* Fp, const uint32_t* Ep,
                                  uint32_t* Fn, uint32_t* En, cudaStream_t st);
// Alignment of Sec. 3.5.2 (Eq. 10): pairs with pad[2] >= 0 (the partner pair's index)
// take the coupled loss, the others the plain one; tracking adds the chain neighbours.
cudaError_t launch_nnf_iter_align(int k, const PairDesc* pairs, int pair0, int n_pairs, const LevelGeom& g,
                                  const uint32_t* srp, uint32_t alpha, bool tracking, int r0, uint64_t seed,
                                  int it, const uint32_t* Fp, const uint32_t* Ep, uint32_t* Fn, uint32_t* En,
                                  cudaStream_t st);

// Fast mode of Sec. 3.4 (Algs. 3-5).  A blending-table entry: the exact sum
// k^2 S_frame + the Alg. 2 votes of its sources, each source one NNF pair (index into the
// pair table; the pair's style is the source frame), stored as 16 bytes per pixel.
struct FastEntry {
    int32_t frame, first_src, n_src, pad;
};
// An output frame: the sum of its pieces (entry, NNF pair to the frame or -1 for the
// identity), minus k^4 S_frame, over 255 k^4 count (the frames in its window).
struct FastJob {
    int32_t frame, first_piece, n_pieces, count;
};
cudaError_t launch_fast_table(int k, const FastEntry* entries, int n_entries, const int32_t* src_pairs,
                              const PairDesc* pairs, const uint32_t* F, const uint32_t* styles, int H,
                              int W, uint4* out, cudaStream_t st);
cudaError_t launch_fast_combine(int k, const FastJob* jobs, int n_jobs, const int2* pieces,
                                const uint32_t* F, const uint4* entries, const uint32_t* styles, int H,
                                int W, float* out, cudaStream_t st);

// Improved loss of Sec. 3.4: S^ images of a chunk's pairs (n_pairs x H x W x 3 bytes,
// from the fields F and the RGBX styles), the loss of the current fields against their
// S^ row patches (shat_rp: n_pairs frames; srp: the source styles' row patches), and the
// Jacobi step under that loss (which evaluates the incumbent's loss itself).  Level 0.
cudaError_t launch_shat(int k, const PairDesc* pairs, int pair0, int n_pairs, int H, int W,
                       const uint32_t* F, const uint32_t* styles, uint8_t* shat, cudaStream_t st);
// The style target of a pair is row-patch slot pl (its own S^) or, with slot_by_target,
// slot pd.tgt - target0 (the mean remapped frame Tbar of its output frame, accurate mode).
cudaError_t launch_energy_balanced(int k, const PairDesc* pairs, int pair0, int n_pairs,
                                   const LevelGeom& g, const uint32_t* srp, const uint32_t* shat_rp,
                                   int slot_by_target, int target0, uint32_t alpha, const uint32_t* F,
                                   uint32_t* E, cudaStream_t st);
cudaError_t launch_nnf_iter_balanced(int k, const PairDesc* pairs, int pair0, int n_pairs,
                                     const LevelGeom& g, const uint32_t* srp, const uint32_t* shat_rp,
                                     int slot_by_target, int target0, uint32_t alpha, int r0,
                                     uint64_t seed, int it, const uint32_t* Fp, uint32_t* Fn,
                                     uint32_t* En, cudaStream_t st);
// Accurate mode: Tbar (8-bit, n_jobs x H x W x 3) of output jobs [job0, job0 + n_jobs)
// from the chunk's fields (pair-local planes from pair0).
cudaError_t launch_tbar(int k, const JobDesc* jobs, int job0, int n_jobs, const PairDesc* pairs, int pair0,
                        const uint32_t* F, const uint32_t* styles, int H, int W, uint8_t* out,
                        cudaStream_t st);
cudaError_t launch_combine(int k, const JobDesc* jobs, int job0, int n_jobs,
                           const PairDesc* pairs, int pair0, const uint32_t* F,
                           const uint32_t* styles, int H, int W, float* out, cudaStream_t st);

cudaError_t launch_energy_sum(const uint32_t* E, size_t n, double* acc, cudaStream_t st);

// ---- learned initialiser (fb_net.cu), used by the blend / interpolation pipeline ----
// Forward pass of `net` on pairs [first, first + n) of a pair table over the guide
// stack `guides` (H x W frames), then the initial fields F0 of those pairs written as
// n x H x W x 2 int32 to nnf_out.  Returns an fb_status.
int initnet_init_pairs(::fb_initnet* net, const uint8_t* guides, const PairDesc* pairs, int first,
                       int n, int32_t* nnf_out, cudaStream_t st);
int initnet_max_pairs(const ::fb_initnet* net);
void initnet_dims(const ::fb_initnet* net, int* H, int* W);

// ---- batched persistent path (fb_batch.cu) --------------------------------------
// One clip of a batch submission (device table).
// Both descriptors are read by the batch kernels as 16-byte vectors (fb_batch.cu): keep
// them 16-byte aligned with the field offsets asserted below.
struct alignas(16) BatchClip {
    int32_t H, W, N, r0;     // r0: first random-search radius for this clip
    const uint32_t* rp;      // row patches of the clip's N guide frames
    const uint32_t* styles;  // RGBX styles of the clip's N frames
    float* out;              // the caller's N x H x W x 3 output
};
// One NNF of a chunk: pair (src -> tgt) of clip `clip`, its F/E plane at fe_off.
struct alignas(16) BatchPair {
    int32_t clip, src, tgt, style;
    uint32_t tag, weight;
    uint64_t fe_off;
};
static_assert(sizeof(BatchClip) == 48 && offsetof(BatchClip, rp) == 16, "BatchClip layout");
static_assert(sizeof(BatchPair) == 32 && offsetof(BatchPair, tag) == 16 &&
                  offsetof(BatchPair, fe_off) == 24, "BatchPair layout");
// One output frame of a chunk; its pairs are [first_pair, first_pair + n_pairs).
struct alignas(16) BatchJob {
    int32_t clip, frame, first_pair, n_pairs;
    uint32_t den;
    int32_t pad[3];
};
static_assert(sizeof(BatchJob) == 32, "BatchJob layout");

// Tile shapes / occupancies the autotuner chooses among (same results for all).
constexpr int kBatchVariants = 4;
// Consecutive tiles of one pair (or output frame) that one claim of a persistent batch
// kernel covers: the claim's descriptor loads and block barrier are paid once per claim
// instead of once per tile.  The iteration kernel's claim size is chosen by the batch
// autotuner among kIterClaimChoices (kIterTilesPerClaim when it is forced or not tuned);
// the remap reads F and styles around each pixel, so its units stay one tile (neighbouring
// tiles then run side by side and share L1/L2 lines).  Work unit u of a launch is
// (unit_pair[u], first tile unit_tile[u]) and covers tiles
// [first, min(first + per_claim, tiles of the pair)).
#ifndef FB_COMBINE_TILES_PER_CLAIM
#define FB_COMBINE_TILES_PER_CLAIM 1
#endif
constexpr int kIterTilesPerClaim = 4;
constexpr int kIterClaimChoices[] = {1, 2, 4, 8};
constexpr int kIterClaimCount = 4;
constexpr int kInitTilesPerClaim = 16;
constexpr int kCombineTilesPerClaim = FB_COMBINE_TILES_PER_CLAIM;
const char* batch_variant_name(int v);
// Work units: item_pair[u] = pair of unit u, item_tile[u] = its first tile within the
// pair (claims of kIterTilesPerClaim / kInitTilesPerClaim tiles).  `counter` must be
// zero when the launch starts (one int per launch).
cudaError_t launch_batch_init(int k, int variant, const BatchPair* pairs, const BatchClip* clips,
                              const int32_t* item_pair, const int32_t* item_tile, int n_items,
                              int* counter, uint64_t seed, uint32_t* F, uint32_t* E, int grid,
                              cudaStream_t st);
cudaError_t launch_batch_iter(int k, int variant, const BatchPair* pairs, const BatchClip* clips,
                              const int32_t* item_pair, const int32_t* item_tile, int n_items,
                              int per_claim, int* counter, uint64_t seed, int it, const uint32_t* Fp,
                              const uint32_t* Ep, uint32_t* Fn, uint32_t* En, int grid,
                              cudaStream_t st);
cudaError_t launch_batch_combine(int k, const BatchJob* jobs, const BatchPair* pairs,
                                 const BatchClip* clips, const int32_t* item_job,
                                 const int32_t* item_tile, int n_items, int* counter,
                                 const uint32_t* F, int grid, cudaStream_t st);
// Rows per tile of a variant (tiles are 32 columns wide).
int batch_variant_tile_h(int variant);
// Resident blocks per SM of the variant's iteration kernel for patch k (occupancy API).
int batch_iter_blocks_per_sm(int k, int variant);

// dp4a throughput probe (fb_calib.cu): blocks x 256 threads x iters x chains dp4a.
constexpr int kDp4aProbeChains = 32;
// Resident 256-thread blocks per SM of the gather probe: 40 warps, the k = 5 iteration
// kernel's occupancy.
constexpr int kIterProbeBlocksPerSm = 5;
cudaError_t launch_dp4a_probe(int blocks, int iters, uint32_t* sink, cudaStream_t st);
// Eq. 1 instruction-sequence probe (fb_calib.cu): blocks x 256 threads x iters candidates of
// the patch-k kernels' per-candidate dp4a sequence (k = 5 or 7), 3k^2 byte pairs each.
cudaError_t launch_ssd_mix_probe(int k, int blocks, int iters, uint32_t* sink, cudaStream_t st);
// Scattered 256-bit loads of a buffer of `slots` (a power of two) 32-byte slots.
cudaError_t launch_gather_probe(const uint32_t* buf, uint32_t slots, int blocks, int iters, uint32_t* sink,
                                cudaStream_t st);

#ifdef FB_CHECKED
// Checked builds: the device-side check words (fb_check.cuh) of the per-call kernels
// (fb_kernels.cu) and of the batched kernels (fb_batch.cu): first failure, failures,
// visits; zeroed after reading if reset.
cudaError_t check_read_kernels(unsigned long long out[3], bool reset);
cudaError_t check_read_batch(unsigned long long out[3], bool reset);
#endif

}  // namespace fb
