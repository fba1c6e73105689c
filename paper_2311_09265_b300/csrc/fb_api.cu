// fb_api.cu -- the C ABI of libfb.so (declared in include/fb.h): argument checks,
// the per-call plan (pairs, output jobs, scratch layout), the scratch arena and the
// launch sequence of the FastBlend hot path.
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <array>
#include <cstring>
#include <functional>
#include <string>
#include <map>
#include <vector>

#include "fb.h"
#include "fb_internal.h"

struct fb_ctx {
    int device = 0;
    char* arena = nullptr;          // device scratch, grown on demand
    size_t arena_cap = 0;
    char* pinned = nullptr;         // pinned host staging for the pair/job tables
    size_t pinned_cap = 0;
    cudaEvent_t upload_done = nullptr;
    bool upload_pending = false;
    // Host-buffer calls: a copy stream that moves the styles in and the blended frames out
    // while the main stream computes, and the events that order the two.
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> xfer_ev;
    uint64_t launches = 0;
    int* dev_status = nullptr;      // device-side error word written by bounded waits
    std::string err;
    // Optional per-launch CUDA-event timing (fb_ctx_profile).
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    // Batched submissions: tuned tile variant per patch size, and the cached manifests.
    int tuned_variant[10] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
    int tuned_claim[10] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1};  // tiles per iteration claim
    int tuned_mode[10] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1};   // persistent or per-clip
    size_t pair_budget = 0;  // bytes of NNF scratch per chunk; 0 = kPairBudgetBytes
    fb_initnet* init_net = nullptr;  // learned initialiser for FB_FLAG_LEARNED_INIT
    double* energy = nullptr;        // device: sum of final errors (FB_FLAG_REPORT_ENERGY)
    uint64_t energy_count = 0;
    struct BatchEntry;
    std::vector<BatchEntry*> batch_cache;  // most recent last
};

// One cached batch manifest: its key, device tables and scratch, and its graph.
struct fb_ctx::BatchEntry {
    std::vector<uint8_t> key;
    char* dev = nullptr;
    size_t bytes = 0;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches_per_run = 0;
    std::vector<std::function<cudaError_t(cudaStream_t)>> steps;  // the submission's launches
    std::vector<int> step_kind;
    // Per-clip launch mode: the streams the clip segments of a chunk are spread over
    // (graph branches) and the events that fork them from and join them to the caller's.
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev;
};

namespace {

using fb::JobDesc;
using fb::LevelGeom;
using fb::PairDesc;
using fb::FastEntry;
using fb::FastJob;

thread_local std::string g_null_ctx_err;

// Bytes of F/E ping-pong scratch one chunk of pairs may use.
constexpr size_t kPairBudgetBytes = size_t(8) << 30;
constexpr int kMaxChunkPairs = 65535;  // grid.y limit

int fail(fb_ctx* ctx, int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_null_ctx_err = buf;
    return status;
}

#define FB_CUDA(ctx, expr)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? FB_ERR_OOM : FB_ERR_CUDA,    \
                        "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

cudaEvent_t next_event(fb_ctx* ctx) {
    if (ctx->ev_used == ctx->ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ctx->ev_pool.push_back(e);
    }
    return ctx->ev_pool[ctx->ev_used++];
}

// Launch through `expr`; with profiling on, bracket it with an event pair on `st`.
#define FB_LAUNCH(ctx, st, kind, expr)                                        \
    do {                                                                      \
        cudaEvent_t ea_ = nullptr, eb_ = nullptr;                             \
        if ((ctx)->profiling) {                                               \
            ea_ = next_event(ctx);                                            \
            eb_ = next_event(ctx);                                            \
            if (ea_ && eb_) FB_CUDA(ctx, cudaEventRecord(ea_, st));           \
        }                                                                     \
        FB_CUDA(ctx, (expr));                                                 \
        ++(ctx)->launches;                                                    \
        if (ea_ && eb_) {                                                     \
            FB_CUDA(ctx, cudaEventRecord(eb_, st));                           \
            (ctx)->recs.push_back(fb_ctx::Rec{(kind), ea_, eb_});             \
        }                                                                     \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Bump allocator over the arena.  With base == nullptr it only measures.
struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(char* b) : base(b) {}
    template <class T>
    T* take(size_t n) {
        off = align_up(off, 256);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

int ensure_arena(fb_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->arena_cap) return FB_OK;
    // Work already enqueued may still use the old block.
    FB_CUDA(ctx, cudaDeviceSynchronize());
    if (ctx->arena) {
        cudaFree(ctx->arena);
        ctx->arena = nullptr;
        ctx->arena_cap = 0;
    }
    const size_t want = align_up(bytes + bytes / 8, size_t(1) << 20);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&ctx->arena), want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->arena = nullptr;
        return fail(ctx, FB_ERR_OOM, "device scratch of %zu bytes: %s", want, cudaGetErrorString(e));
    }
    ctx->arena_cap = want;
    return FB_OK;
}

int ensure_pinned(fb_ctx* ctx, size_t bytes) {
    if (ctx->upload_pending) {
        FB_CUDA(ctx, cudaEventSynchronize(ctx->upload_done));
        ctx->upload_pending = false;
    }
    if (bytes <= ctx->pinned_cap) return FB_OK;
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    ctx->pinned = nullptr;
    ctx->pinned_cap = 0;
    const size_t want = align_up(bytes, size_t(1) << 16);
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&ctx->pinned), want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, FB_ERR_OOM, "pinned staging of %zu bytes: %s", want, cudaGetErrorString(e));
    }
    ctx->pinned_cap = want;
    return FB_OK;
}

enum class Mem { Device, Host, Invalid };

Mem classify(const fb_ctx* ctx, const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return Mem::Host;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return a.device == ctx->device ? Mem::Device : Mem::Invalid;
    return Mem::Host;
}

int check_params(fb_ctx* ctx, const fb_params* p, int H, int W) {
    if (!p) return fail(ctx, FB_ERR_ARG, "params is NULL");
    if (p->patch < 3 || p->patch > 9 || (p->patch & 1) == 0)
        return fail(ctx, FB_ERR_ARG, "patch must be odd in [3, 9], got %d", p->patch);
    if (p->iters < 0 || p->iters > 65534)
        return fail(ctx, FB_ERR_ARG, "iters must be in [0, 65534], got %d", p->iters);
    if (p->levels < 1 || p->levels > 16)
        return fail(ctx, FB_ERR_ARG, "levels must be in [1, 16], got %d", p->levels);
    if (p->r0 < 0 || p->r0 > (1 << 20))
        return fail(ctx, FB_ERR_ARG, "r0 must be in [0, 2^20], got %d", p->r0);
    if (p->flags & ~(FB_FLAG_LEARNED_INIT | FB_FLAG_REPORT_ENERGY | FB_FLAG_BALANCED | FB_FLAG_FAST |
                     FB_FLAG_ACCURATE | FB_FLAG_TRACKING | FB_FLAG_ALIGN))
        return fail(ctx, FB_ERR_ARG, "unknown flags 0x%x", p->flags);
    if (p->flags & FB_FLAG_ALIGN) {
        if (p->levels != 1) return fail(ctx, FB_ERR_ARG, "FB_FLAG_ALIGN requires levels == 1");
        if (p->alpha > 255) return fail(ctx, FB_ERR_ARG, "alpha must be in [0, 255], got %u", p->alpha);
        if (p->flags & (FB_FLAG_LEARNED_INIT | FB_FLAG_REPORT_ENERGY | FB_FLAG_BALANCED | FB_FLAG_FAST |
                        FB_FLAG_ACCURATE))
            return fail(ctx, FB_ERR_ARG, "FB_FLAG_ALIGN combines with FB_FLAG_TRACKING only");
    }
    if (p->flags & FB_FLAG_TRACKING) {
        if (p->levels != 1) return fail(ctx, FB_ERR_ARG, "FB_FLAG_TRACKING requires levels == 1");
        if (p->flags & FB_FLAG_LEARNED_INIT)
            return fail(ctx, FB_ERR_ARG, "FB_FLAG_TRACKING does not combine with FB_FLAG_LEARNED_INIT");
        if (p->flags & (FB_FLAG_BALANCED | FB_FLAG_FAST | FB_FLAG_ACCURATE))
            return fail(ctx, FB_ERR_ARG, "FB_FLAG_TRACKING applies to the plain loss and the direct sum");
    }
    if (p->flags & FB_FLAG_ACCURATE) {
        if (p->flags & (FB_FLAG_BALANCED | FB_FLAG_FAST | FB_FLAG_LEARNED_INIT))
            return fail(ctx, FB_ERR_ARG, "FB_FLAG_ACCURATE does not combine with the other mode flags");
        if (p->levels != 1) return fail(ctx, FB_ERR_ARG, "FB_FLAG_ACCURATE requires levels == 1");
        if (p->alpha > 255) return fail(ctx, FB_ERR_ARG, "alpha must be in [0, 255], got %u", p->alpha);
    }
    if ((p->flags & FB_FLAG_FAST) && (p->flags & (FB_FLAG_BALANCED | FB_FLAG_LEARNED_INIT)))
        return fail(ctx, FB_ERR_ARG, "FB_FLAG_FAST does not combine with FB_FLAG_BALANCED or FB_FLAG_LEARNED_INIT");
    if (p->flags & FB_FLAG_BALANCED) {
        if (p->levels != 1) return fail(ctx, FB_ERR_ARG, "FB_FLAG_BALANCED requires levels == 1");
        if (p->alpha > 255) return fail(ctx, FB_ERR_ARG, "alpha must be in [0, 255], got %u", p->alpha);
        if (p->flags & FB_FLAG_LEARNED_INIT)
            return fail(ctx, FB_ERR_ARG, "FB_FLAG_BALANCED does not combine with FB_FLAG_LEARNED_INIT");
    }
    if (H < p->patch || W < p->patch || H > 32767 || W > 32767)
        return fail(ctx, FB_ERR_ARG, "image %dx%d outside [patch, 32767]", H, W);
    return FB_OK;
}

struct Levels {
    int n;
    int h[16], w[16];
};

Levels level_dims(int H, int W, int levels) {
    Levels L;
    L.n = levels;
    L.h[0] = H;
    L.w[0] = W;
    for (int l = 1; l < levels; ++l) {
        L.h[l] = (L.h[l - 1] + 1) / 2;
        L.w[l] = (L.w[l - 1] + 1) / 2;
    }
    return L;
}

// Device buffers of one call.
struct Buffers {
    uint8_t* raw[16] = {};       // downsampled guides, levels >= 1
    uint32_t* rec[16] = {};   // row patches per level
    uint32_t* styles = nullptr;
    uint32_t* srec = nullptr;      // improved loss: style row patches (level 0)
    uint8_t* shat_img = nullptr;   // improved loss: S^ of a chunk's pairs, H x W x 3 each
    uint32_t* shat_rec = nullptr;  // ... and their row patches
    uint32_t *FA = nullptr, *FB = nullptr, *EA = nullptr, *EB = nullptr;
    int32_t* init = nullptr;     // learned initial fields of a chunk (int32 pairs)
    PairDesc* pairs = nullptr;
    JobDesc* jobs = nullptr;
    uint8_t* in_guides = nullptr;  // host-staging copies
    uint8_t* in_styles = nullptr;
    float* in_out = nullptr;
};

void carve(Carver& cv, Buffers& b, const Levels& L, int k, int n_guides, int n_styles,
           size_t chunk_pairs, size_t n_pairs, size_t n_jobs, bool staging, size_t guide_bytes,
           size_t style_bytes, size_t out_floats, bool learned = false,
           bool balanced = false, bool style_rows = false) {
    for (int l = 0; l < L.n; ++l) {
        const size_t npx = static_cast<size_t>(L.h[l]) * L.w[l];
        if (l > 0) b.raw[l] = cv.take<uint8_t>(static_cast<size_t>(n_guides) * npx * 3);
        b.rec[l] = cv.take<uint32_t>(static_cast<size_t>(n_guides) * fb::rowpatch_frame_words(k, L.h[l], L.w[l]));
    }
    const size_t npx0 = static_cast<size_t>(L.h[0]) * L.w[0];
    b.styles = cv.take<uint32_t>(static_cast<size_t>(n_styles) * npx0);
    b.FA = cv.take<uint32_t>(chunk_pairs * npx0);
    b.FB = cv.take<uint32_t>(chunk_pairs * npx0);
    b.EA = cv.take<uint32_t>(chunk_pairs * npx0);
    b.EB = cv.take<uint32_t>(chunk_pairs * npx0);
    if (learned) b.init = cv.take<int32_t>(chunk_pairs * npx0 * 2);
    if (balanced || style_rows) {
        const size_t fw = fb::rowpatch_frame_words(k, L.h[0], L.w[0]);
        b.srec = cv.take<uint32_t>(static_cast<size_t>(n_styles) * fw);
        if (balanced) {
            b.shat_img = cv.take<uint8_t>(chunk_pairs * npx0 * 3);
            b.shat_rec = cv.take<uint32_t>(chunk_pairs * fw);
        }
    }
    b.pairs = cv.take<PairDesc>(n_pairs > 0 ? n_pairs : 1);
    b.jobs = cv.take<JobDesc>(n_jobs > 0 ? n_jobs : 1);
    if (staging) {
        b.in_guides = cv.take<uint8_t>(guide_bytes);
        b.in_styles = cv.take<uint8_t>(style_bytes);
        b.in_out = cv.take<float>(out_floats);
    }
}

int upload_tables(fb_ctx* ctx, const std::vector<PairDesc>& pairs, const std::vector<JobDesc>& jobs,
                  Buffers& b, cudaStream_t st) {
    const size_t pb = pairs.size() * sizeof(PairDesc), jb = jobs.size() * sizeof(JobDesc);
    if (pb + jb == 0) return FB_OK;
    int rc = ensure_pinned(ctx, pb + jb + 256);
    if (rc) return rc;
    if (pb) std::memcpy(ctx->pinned, pairs.data(), pb);
    if (jb) std::memcpy(ctx->pinned + align_up(pb, 256), jobs.data(), jb);
    if (pb) FB_CUDA(ctx, cudaMemcpyAsync(b.pairs, ctx->pinned, pb, cudaMemcpyHostToDevice, st));
    if (jb)
        FB_CUDA(ctx, cudaMemcpyAsync(b.jobs, ctx->pinned + align_up(pb, 256), jb,
                                     cudaMemcpyHostToDevice, st));
    FB_CUDA(ctx, cudaEventRecord(ctx->upload_done, st));
    ctx->upload_pending = true;
    return FB_OK;
}

// Guide frames (n of them, contiguous at `frames`) -> row patches at every
// pyramid level, into guide slots [slot0, slot0 + n).
int prep_guides(fb_ctx* ctx, const Buffers& b, const Levels& L, int k, const uint8_t* frames,
                int n, int slot0, cudaStream_t st) {
    const uint8_t* cur = frames;
    for (int l = 0; l < L.n; ++l) {
        const size_t npx = static_cast<size_t>(L.h[l]) * L.w[l];
        if (l > 0) {
            uint8_t* dst = b.raw[l] + static_cast<size_t>(slot0) * npx * 3;
            FB_LAUNCH(ctx, st, FB_K_DOWNSAMPLE, fb::launch_downsample(cur, n, L.h[l - 1], L.w[l - 1], dst, st));
            cur = dst;
        }
        FB_LAUNCH(ctx, st, FB_K_PREP, fb::launch_prep_guides(k, cur, n, L.h[l], L.w[l],
                                              b.rec[l] + static_cast<size_t>(slot0) *
                                                             fb::rowpatch_frame_words(k, L.h[l], L.w[l]), st));
    }
    return FB_OK;
}

// Alg. 1 for pairs [pair0, pair0 + n) of the uploaded table.  The final level-0
// field and errors are returned in *F_out / *E_out (one of the ping-pong buffers).
int run_nnf(fb_ctx* ctx, const Buffers& b, const Levels& L, const fb_params* p, int pair0, int n,
            const int32_t* user_init, cudaStream_t st, uint32_t** F_out, uint32_t** E_out) {
    const int k = p->patch;
    uint32_t *Fc = b.FA, *Ec = b.EA, *Fo = b.FB, *Eo = b.EB;
    for (int l = L.n - 1; l >= 0; --l) {
        LevelGeom g{L.h[l], L.w[l], b.rec[l]};
        if (l == L.n - 1) {
            FB_LAUNCH(ctx, st, FB_K_INIT, fb::launch_nnf_init(k, b.pairs, pair0, n, g, user_init ? 2 : 0, nullptr,
                                               0, 0, user_init, p->seed, l, Fc, Ec, st));
        } else {
            FB_LAUNCH(ctx, st, FB_K_INIT, fb::launch_nnf_init(k, b.pairs, pair0, n, g, 1, Fc, L.h[l + 1],
                                               L.w[l + 1], nullptr, p->seed, l, Fo, Eo, st));
            std::swap(Fc, Fo);
            std::swap(Ec, Eo);
        }
        const int r0 = p->r0 > 0 ? p->r0 : (L.h[l] > L.w[l] ? L.h[l] : L.w[l]);
        const bool tracking = (p->flags & FB_FLAG_TRACKING) != 0;  // levels == 1
        const bool align = (p->flags & FB_FLAG_ALIGN) != 0;        // levels == 1
        for (int it = 0; it < p->iters; ++it) {
            if (align)
                FB_LAUNCH(ctx, st, FB_K_ITER, fb::launch_nnf_iter_align(k, b.pairs, pair0, n, g, b.srec, p->alpha,
                                                                       tracking, r0, p->seed, it, Fc, Ec, Fo, Eo,
                                                                       st));
            else if (tracking)
                FB_LAUNCH(ctx, st, FB_K_ITER, fb::launch_nnf_iter_track(k, b.pairs, pair0, n, g, r0, p->seed, it, Fc,
                                                                       Ec, Fo, Eo, st));
            else
                FB_LAUNCH(ctx, st, FB_K_ITER, fb::launch_nnf_iter(k, b.pairs, pair0, n, g, r0, p->seed, l, it, Fc, Ec,
                                                   Fo, Eo, st));
            std::swap(Fc, Fo);
            std::swap(Ec, Eo);
        }
    }
    *F_out = Fc;
    *E_out = Ec;
    return FB_OK;
}

// Alg. 1 under the improved loss of Sec. 3.4 (level 0 only) for pairs [pair0, pair0 + n):
// at the beginning of every iteration S^ is rebuilt from the fields (remap of the source
// style, rounded, laid out as row patches); the Jacobi step then re-evaluates each
// incumbent against it before comparing candidates.  With no iterations the loss of the
// initial field is left in E.
int run_nnf_balanced(fb_ctx* ctx, const Buffers& b, int H, int W, const fb_params* p, int pair0,
                     int n, const int32_t* user_init, cudaStream_t st, uint32_t** F_out,
                     uint32_t** E_out) {
    const int k = p->patch;
    const LevelGeom g{H, W, b.rec[0]};
    uint32_t *Fc = b.FA, *Ec = b.EA, *Fo = b.FB, *Eo = b.EB;
    FB_LAUNCH(ctx, st, FB_K_INIT, fb::launch_nnf_init(k, b.pairs, pair0, n, g, user_init ? 2 : 0, nullptr, 0, 0,
                                                      user_init, p->seed, 0, Fc, Ec, st));
    const int r0 = p->r0 > 0 ? p->r0 : (H > W ? H : W);
    const int rounds = p->iters > 0 ? p->iters : 1;
    for (int it = 0; it < rounds; ++it) {
        FB_LAUNCH(ctx, st, FB_K_SHAT, fb::launch_shat(k, b.pairs, pair0, n, H, W, Fc, b.styles, b.shat_img, st));
        FB_LAUNCH(ctx, st, FB_K_PREP, fb::launch_prep_guides(k, b.shat_img, n, H, W, b.shat_rec, st));
        if (p->iters == 0) {
            FB_LAUNCH(ctx, st, FB_K_ENERGY, fb::launch_energy_balanced(k, b.pairs, pair0, n, g, b.srec, b.shat_rec,
                                                                       0, 0, p->alpha, Fc, Ec, st));
            break;
        }
        // the iteration kernel re-evaluates the incumbent against the new S^ itself
        FB_LAUNCH(ctx, st, FB_K_ITER, fb::launch_nnf_iter_balanced(k, b.pairs, pair0, n, g, b.srec, b.shat_rec,
                                                                   0, 0, p->alpha, r0, p->seed, it, Fc, Fo, Eo, st));
        std::swap(Fc, Fo);
        std::swap(Ec, Eo);
    }
    *F_out = Fc;
    *E_out = Ec;
    return FB_OK;
}

// Accurate mode of Sec. 3.4 for the pairs of output jobs [job0, job0 + n_jobs) (pairs
// [pair0, pair0 + n_pairs), level 0): at the beginning of every iteration the mean
// remapped frame Tbar of every output frame is rebuilt from the current fields (rounded,
// laid out as row patches in the S^ buffers, one slot per job), then every pair takes a
// Jacobi step under alpha * Eq.1(guides) + Eq.1(source style, Tbar of its output frame).
int run_nnf_accurate(fb_ctx* ctx, const Buffers& b, int H, int W, const fb_params* p, int job0,
                     int n_jobs, int target0, int pair0, int n, cudaStream_t st, uint32_t** F_out,
                     uint32_t** E_out) {
    const int k = p->patch;
    const LevelGeom g{H, W, b.rec[0]};
    uint32_t *Fc = b.FA, *Ec = b.EA, *Fo = b.FB, *Eo = b.EB;
    FB_LAUNCH(ctx, st, FB_K_INIT, fb::launch_nnf_init(k, b.pairs, pair0, n, g, 0, nullptr, 0, 0, nullptr, p->seed,
                                                      0, Fc, Ec, st));
    const int r0 = p->r0 > 0 ? p->r0 : (H > W ? H : W);
    for (int it = 0; it < p->iters; ++it) {
        FB_LAUNCH(ctx, st, FB_K_SHAT, fb::launch_tbar(k, b.jobs, job0, n_jobs, b.pairs, pair0, Fc, b.styles, H, W,
                                                      b.shat_img, st));
        FB_LAUNCH(ctx, st, FB_K_PREP, fb::launch_prep_guides(k, b.shat_img, n_jobs, H, W, b.shat_rec, st));
        FB_LAUNCH(ctx, st, FB_K_ITER, fb::launch_nnf_iter_balanced(k, b.pairs, pair0, n, g, b.srec, b.shat_rec,
                                                                   1, target0, p->alpha, r0, p->seed, it, Fc, Fo,
                                                                   Eo, st));
        std::swap(Fc, Fo);
        std::swap(Ec, Eo);
    }
    *F_out = Fc;
    *E_out = Ec;
    return FB_OK;
}

// Sec. 3.5.1: a pair's chain neighbours are the pairs from the same source frame to the
// frames before and after its target.  No pair maps a frame to itself (a keyframe, or the
// source of a blend window), so chains end next to their source.  The indices are those of
// the call's pair table, which the tracking kernel sees in one launch.
void set_chain_neighbours(std::vector<PairDesc>& pairs) {
    std::map<std::pair<int, int>, int> index;
    for (size_t q = 0; q < pairs.size(); ++q) index[{pairs[q].src, pairs[q].tgt}] = static_cast<int>(q);
    for (PairDesc& pd : pairs) {
        auto a = index.find({pd.src, pd.tgt - 1}), b = index.find({pd.src, pd.tgt + 1});
        pd.pad[0] = a == index.end() ? -1 : a->second;
        pd.pad[1] = b == index.end() ? -1 : b->second;
    }
}

// Eq. 2 (a1, blending): one job per output frame i; its pairs are (j -> i) for j in the
// window [i - M, i + M] truncated to the clip [0, N), j != i, in increasing j, each weight 1.
// Output frames [i0, i1) of the clip (default: all); job q writes output slot q = i - i0.
// Guide and style slots are clip frames minus `base` (the clip frame held in slot 0), while
// every pair keeps the Philox stream of its clip frames, fb_pair_tag(j, i): a call over a
// range of output frames with the input frames their windows need (Sec. 3.4's sliding
// window makes that range plus M frames on either side) computes the very NNFs, and so the
// very output frames, that the whole-clip call does.
void blend_pairs(int N, int k, int window, uint32_t flags, std::vector<PairDesc>& pairs,
                 std::vector<JobDesc>& jobs, int i0 = 0, int i1 = -1, int base = 0) {
    const int M = (window - 1) / 2;
    if (i1 < 0) i1 = N;
    pairs.clear();
    jobs.assign(i1 - i0, JobDesc{});
    for (int i = i0; i < i1; ++i) {
        const int lo = i - M < 0 ? 0 : i - M, hi = i + M > N - 1 ? N - 1 : i + M;
        jobs[i - i0] = JobDesc{i - i0, i - base, 1u, static_cast<int32_t>(pairs.size()), hi - lo,
                               static_cast<uint32_t>(255 * k * k * (hi - lo + 1)), {0, 0}};
        for (int j = lo; j <= hi; ++j)
            if (j != i) pairs.push_back(PairDesc{j - base, i - base, fb_pair_tag(j, i), j - base, 1u, {-1, -1, -1}});
    }
    if (flags & FB_FLAG_TRACKING) set_chain_neighbours(pairs);
}

// Sec. 3.5.2 (a1, interpolation; Eq. 9): keys are copied; a frame between keys l < i < r
// takes the pairs (l -> i) with weight r - i and (r -> i) with weight i - l over r - l
// (Eq. 10 partners of each other under FB_FLAG_ALIGN); a frame outside the key range
// takes its nearest key alone, weight 1.  Key styles are indexed by key number.  Output
// frames [i0, i1) of the clip (default: all), job q writing output slot q = i - i0; guide
// slots are clip frames (the call holds every guide frame).
void interp_pairs(int N, int k, const int32_t* key_idx, int n_keys, uint32_t flags,
                  std::vector<PairDesc>& pairs, std::vector<JobDesc>& jobs, int i0 = 0, int i1 = -1) {
    const uint32_t kk255 = static_cast<uint32_t>(255 * k * k);
    if (i1 < 0) i1 = N;
    pairs.clear();
    jobs.assign(i1 - i0, JobDesc{});
    int m_left = -1;  // last key index < i
    int next = 0;     // first key with frame >= i
    for (int i = 0; i < i1; ++i) {
        while (next < n_keys && key_idx[next] < i) m_left = next++;
        if (i < i0) continue;
        const bool is_key = next < n_keys && key_idx[next] == i;
        const int m_right = is_key ? (next + 1 < n_keys ? next + 1 : -1) : (next < n_keys ? next : -1);
        JobDesc j{i - i0, -1, 0u, static_cast<int32_t>(pairs.size()), 0, kk255, {0, 0}};
        if (is_key) {
            j.self_style = next;
            j.self_w = 1u;
        } else if (m_left >= 0 && m_right >= 0) {
            const int l = key_idx[m_left], r = key_idx[m_right];
            const int q = static_cast<int>(pairs.size());
            const int32_t pl = (flags & FB_FLAG_ALIGN) ? q + 1 : -1, pr = (flags & FB_FLAG_ALIGN) ? q : -1;
            pairs.push_back(PairDesc{l, i, fb_pair_tag(l, i), m_left, static_cast<uint32_t>(r - i), {-1, -1, pl}});
            pairs.push_back(PairDesc{r, i, fb_pair_tag(r, i), m_right, static_cast<uint32_t>(i - l), {-1, -1, pr}});
            j.n_pairs = 2;
            j.den = kk255 * static_cast<uint32_t>(r - l);
        } else {
            const int m = m_left >= 0 ? m_left : m_right;
            const int l = key_idx[m];
            pairs.push_back(PairDesc{l, i, fb_pair_tag(l, i), m, 1u, {-1, -1, -1}});
            j.n_pairs = 1;
        }
        jobs[i - i0] = j;
    }
    if (flags & FB_FLAG_TRACKING) set_chain_neighbours(pairs);
}

// The copy stream and at least n ordering events (created on first use).
int ensure_xfer(fb_ctx* ctx, size_t n) {
    if (!ctx->copy_stream)
        FB_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    while (ctx->xfer_ev.size() < n) {
        cudaEvent_t e = nullptr;
        FB_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->xfer_ev.push_back(e);
    }
    return FB_OK;
}

// Group consecutive output jobs into chunks whose pairs fit the F/E budget.
struct Chunk {
    int job0, n_jobs, pair0, n_pairs;
};

size_t pair_budget(const fb_ctx* ctx) {
    return ctx && ctx->pair_budget ? ctx->pair_budget : kPairBudgetBytes;
}

int make_chunks(fb_ctx* ctx, const std::vector<JobDesc>& jobs, size_t npx0,
                std::vector<Chunk>& chunks, size_t& max_pairs, size_t extra_per_pair = 0,
                size_t cap_pairs = 0) {
    const size_t per_pair = npx0 * 4 * sizeof(uint32_t) + extra_per_pair;
    size_t cap = pair_budget(ctx) / per_pair;
    if (cap > static_cast<size_t>(kMaxChunkPairs)) cap = kMaxChunkPairs;
    if (cap_pairs > 0 && cap_pairs < cap) cap = cap_pairs;
    if (cap < 1) cap = 1;
    max_pairs = 0;
    Chunk cur{0, 0, jobs.empty() ? 0 : jobs[0].first_pair, 0};
    for (size_t j = 0; j < jobs.size(); ++j) {
        const size_t np = static_cast<size_t>(jobs[j].n_pairs);
        if (np > cap)
            return fail(ctx, FB_ERR_OOM, "output frame needs %zu NNFs; the pair budget holds %zu",
                        np, cap);
        if (cur.n_pairs + np > cap && cur.n_jobs > 0) {
            chunks.push_back(cur);
            cur = Chunk{static_cast<int>(j), 0, jobs[j].first_pair, 0};
        }
        cur.n_jobs += 1;
        cur.n_pairs += static_cast<int>(np);
    }
    if (cur.n_jobs > 0) chunks.push_back(cur);
    for (const Chunk& c : chunks)
        if (static_cast<size_t>(c.n_pairs) > max_pairs) max_pairs = c.n_pairs;
    return FB_OK;
}

// Shared driver of fb_blend_window and fb_interpolate (and their range forms): N guide
// frames, a style stack, a pair table and one job per output frame (out holds
// jobs.size() frames).
int run_pipeline(fb_ctx* ctx, const uint8_t* guides, int N, int H, int W, const uint8_t* styles,
                 int n_styles, const std::vector<PairDesc>& pairs, const std::vector<JobDesc>& jobs,
                 const fb_params* p, float* out, cudaStream_t st) {
    const int k = p->patch;
    const Levels L = level_dims(H, W, p->levels);
    const size_t npx0 = static_cast<size_t>(H) * W;

    const Mem mg = classify(ctx, guides), ms = classify(ctx, styles), mo = classify(ctx, out);
    if (mg == Mem::Invalid || ms == Mem::Invalid || mo == Mem::Invalid)
        return fail(ctx, FB_ERR_ARG, "a device pointer belongs to another device");
    if (!(mg == ms && ms == mo))
        return fail(ctx, FB_ERR_ARG, "guides, styles and out must all be device or all host memory");
    const bool staging = mg == Mem::Host;

    const bool accurate = (p->flags & FB_FLAG_ACCURATE) != 0;
    const bool balanced = (p->flags & FB_FLAG_BALANCED) != 0 || accurate;
    // the improved loss keeps each pair's S^ image and row patches next to its F/E (the
    // accurate mode uses the same buffers for the Tbar of each output frame)
    const size_t extra = balanced ? npx0 * 3 + fb::rowpatch_frame_words(k, H, W) * sizeof(uint32_t) : 0;
    std::vector<Chunk> chunks;
    size_t max_pairs = 0;
    int rc = make_chunks(ctx, jobs, npx0, chunks, max_pairs, extra);
    if (rc) return rc;
    // Host buffers: at least kStagingChunks chunks (each still millions of pixels per
    // launch), so that a chunk's frames leave on the copy stream while the next chunk's
    // NNFs are computed.  Tracking chains run through whole clips: one chunk.
    constexpr size_t kStagingChunks = 4, kStagingChunkPixels = size_t(1) << 21;
    if (staging && !(p->flags & FB_FLAG_TRACKING) && chunks.size() < kStagingChunks &&
        pairs.size() * npx0 >= kStagingChunks * kStagingChunkPixels) {
        size_t cap = (pairs.size() + kStagingChunks - 1) / kStagingChunks, most = 1;
        for (const JobDesc& j : jobs) most = std::max(most, static_cast<size_t>(j.n_pairs));
        chunks.clear();
        rc = make_chunks(ctx, jobs, npx0, chunks, max_pairs, extra, std::max(cap, most));
        if (rc) return rc;
    }
    if ((p->flags & FB_FLAG_TRACKING) && chunks.size() > 1)
        return fail(ctx, FB_ERR_UNSUPPORTED, "tracking keeps all %zu NNFs of the call at once; the pair budget does not",
                    pairs.size());

    const size_t guide_bytes = static_cast<size_t>(N) * npx0 * 3;
    const size_t style_bytes = static_cast<size_t>(n_styles) * npx0 * 3;
    const size_t out_floats = jobs.size() * npx0 * 3;  // one output frame per job
    const bool learned = (p->flags & FB_FLAG_LEARNED_INIT) != 0;
    if (learned) {
        if (!ctx->init_net) return fail(ctx, FB_ERR_ARG, "FB_FLAG_LEARNED_INIT without fb_ctx_set_initnet");
        int nh = 0, nw = 0;
        fb::initnet_dims(ctx->init_net, &nh, &nw);
        if (nh != H || nw != W || p->levels != 1)
            return fail(ctx, FB_ERR_ARG, "the learned initialiser was built for %dx%d frames and levels == 1",
                        nh, nw);
    }
    Buffers b;
    Carver measure(nullptr);
    const bool align = (p->flags & FB_FLAG_ALIGN) != 0;
    carve(measure, b, L, k, N, n_styles, max_pairs, pairs.size(), jobs.size(), staging, guide_bytes,
          style_bytes, out_floats, learned, balanced, align);
    rc = ensure_arena(ctx, measure.off);
    if (rc) return rc;
    Carver cv(ctx->arena);
    carve(cv, b, L, k, N, n_styles, max_pairs, pairs.size(), jobs.size(), staging, guide_bytes,
          style_bytes, out_floats, learned, balanced, align);

    rc = upload_tables(ctx, pairs, jobs, b, st);
    if (rc) return rc;
    const uint8_t* g_dev = guides;
    const uint8_t* s_dev = styles;
    float* o_dev = out;
    // Host buffers: the guides come in on the main stream (the search needs them first);
    // the styles on the copy stream, after the main stream's earlier work on the arena,
    // while the guides are prepared and (plain search) the NNFs computed; the blended
    // frames go out on the copy stream in groups, each as soon as its combine is done.
    constexpr int kOutGroups = 4;
    const bool styles_late = staging && !balanced && !align;  // only the combine reads them
    bool frames_in_order = true;  // output frame of job j is j: a group's frames are contiguous
    for (size_t j = 0; j < jobs.size(); ++j) frames_in_order = frames_in_order && jobs[j].out_frame == static_cast<int>(j);
    size_t ev = 0;  // next ordering event
    if (ctx->copy_stream) {  // a failed earlier call may have left copies of the arena in flight
        rc = ensure_xfer(ctx, 1);
        if (rc) return rc;
        FB_CUDA(ctx, cudaEventRecord(ctx->xfer_ev[0], ctx->copy_stream));
        FB_CUDA(ctx, cudaStreamWaitEvent(st, ctx->xfer_ev[0], 0));
    }
    if (staging) {
        rc = ensure_xfer(ctx, 2 + kOutGroups * chunks.size() + 1);
        if (rc) return rc;
        FB_CUDA(ctx, cudaMemcpyAsync(b.in_guides, guides, guide_bytes, cudaMemcpyHostToDevice, st));
        FB_CUDA(ctx, cudaEventRecord(ctx->xfer_ev[ev], st));
        FB_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->xfer_ev[ev++], 0));
        FB_CUDA(ctx, cudaMemcpyAsync(b.in_styles, styles, style_bytes, cudaMemcpyHostToDevice, ctx->copy_stream));
        FB_CUDA(ctx, cudaEventRecord(ctx->xfer_ev[ev], ctx->copy_stream));
        g_dev = b.in_guides;
        s_dev = b.in_styles;
        o_dev = b.in_out;
    }
    const size_t styles_in = ev++;
    auto convert_styles = [&]() -> int {
        if (staging) FB_CUDA(ctx, cudaStreamWaitEvent(st, ctx->xfer_ev[styles_in], 0));
        FB_LAUNCH(ctx, st, FB_K_STYLE,
                  fb::launch_style_rgbx(s_dev, static_cast<size_t>(n_styles) * npx0, b.styles, st));
        return FB_OK;
    };

    rc = prep_guides(ctx, b, L, k, g_dev, N, 0, st);
    if (rc) return rc;
    if (!styles_late) {
        rc = convert_styles();
        if (rc) return rc;
    }
    bool styles_ready = !styles_late;
    if (balanced || align)
        FB_LAUNCH(ctx, st, FB_K_PREP, fb::launch_prep_guides(k, s_dev, n_styles, H, W, b.srec, st));

    if (p->flags & FB_FLAG_REPORT_ENERGY) {
        FB_CUDA(ctx, cudaMemsetAsync(ctx->energy, 0, sizeof(double), st));
        ctx->energy_count = 0;
    }
    for (const Chunk& c : chunks) {
        uint32_t *F = nullptr, *E = nullptr;
        if (c.n_pairs > 0) {
            const int32_t* init = nullptr;
            if (p->flags & FB_FLAG_LEARNED_INIT) {
                // Initial fields of the chunk's pairs from the learned initialiser, in
                // batches of at most its capacity, into the learned-init buffer.
                const int cap = fb::initnet_max_pairs(ctx->init_net);
                for (int q = 0; q < c.n_pairs; q += cap) {
                    const int cnt = c.n_pairs - q < cap ? c.n_pairs - q : cap;
                    cudaEvent_t ea = nullptr, eb = nullptr;
                    if (ctx->profiling) {
                        ea = next_event(ctx);
                        eb = next_event(ctx);
                        if (ea && eb) FB_CUDA(ctx, cudaEventRecord(ea, st));
                    }
                    int r2 = fb::initnet_init_pairs(ctx->init_net, g_dev, b.pairs, c.pair0 + q, cnt,
                                                    b.init + static_cast<size_t>(q) * npx0 * 2, st);
                    if (r2) return fail(ctx, r2, "learned initialiser failed");
                    ctx->launches += 17;  // input, 3 concatenations, 12 convolutions, offsets
                    if (ea && eb) {
                        FB_CUDA(ctx, cudaEventRecord(eb, st));
                        ctx->recs.push_back(fb_ctx::Rec{FB_K_INITNET, ea, eb});
                    }
                }
                init = b.init;
            }
            rc = accurate ? run_nnf_accurate(ctx, b, H, W, p, c.job0, c.n_jobs, jobs[c.job0].self_style, c.pair0,
                                             c.n_pairs, st, &F, &E)
                 : balanced ? run_nnf_balanced(ctx, b, H, W, p, c.pair0, c.n_pairs, init, st, &F, &E)
                            : run_nnf(ctx, b, L, p, c.pair0, c.n_pairs, init, st, &F, &E);
            if (rc) return rc;
            if (p->flags & FB_FLAG_REPORT_ENERGY) {
                FB_LAUNCH(ctx, st, FB_K_ITER, fb::launch_energy_sum(E, static_cast<size_t>(c.n_pairs) * npx0,
                                                                   ctx->energy, st));
                ctx->energy_count += static_cast<uint64_t>(c.n_pairs) * npx0;
            }
        }
        if (!styles_ready) {
            rc = convert_styles();
            if (rc) return rc;
            styles_ready = true;
        }
        if (!staging || !frames_in_order) {
            FB_LAUNCH(ctx, st, FB_K_COMBINE, fb::launch_combine(k, b.jobs, c.job0, c.n_jobs, b.pairs, c.pair0, F,
                                                               b.styles, H, W, o_dev, st));
            continue;
        }
        // Output frames = job indices; each group's frames leave while the next combines.
        const int per = (c.n_jobs + kOutGroups - 1) / kOutGroups;
        for (int j0 = c.job0; j0 < c.job0 + c.n_jobs; j0 += per) {
            const int nj = std::min(per, c.job0 + c.n_jobs - j0);
            FB_LAUNCH(ctx, st, FB_K_COMBINE, fb::launch_combine(k, b.jobs, j0, nj, b.pairs, c.pair0, F, b.styles, H,
                                                               W, o_dev, st));
            FB_CUDA(ctx, cudaEventRecord(ctx->xfer_ev[ev], st));
            FB_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->xfer_ev[ev++], 0));
            const size_t f0 = static_cast<size_t>(jobs[j0].out_frame) * npx0 * 3;
            FB_CUDA(ctx, cudaMemcpyAsync(out + f0, o_dev + f0, static_cast<size_t>(nj) * npx0 * 3 * sizeof(float),
                                         cudaMemcpyDeviceToHost, ctx->copy_stream));
        }
    }

    if (staging) {
        if (!styles_ready) FB_CUDA(ctx, cudaStreamWaitEvent(st, ctx->xfer_ev[styles_in], 0));
        if (!frames_in_order)
            FB_CUDA(ctx, cudaMemcpyAsync(out, o_dev, out_floats * sizeof(float), cudaMemcpyDeviceToHost, st));
        FB_CUDA(ctx, cudaEventRecord(ctx->xfer_ev[ev], ctx->copy_stream));
        FB_CUDA(ctx, cudaStreamWaitEvent(st, ctx->xfer_ev[ev++], 0));
        FB_CUDA(ctx, cudaStreamSynchronize(st));
    }
    return FB_OK;
}

// ---------------------------------------------------------------------------------
// Fast mode of Sec. 3.4
// ---------------------------------------------------------------------------------
struct FastPlan {
    std::vector<PairDesc> pairs;   // distinct NNFs (source frame -> target frame)
    std::vector<FastEntry> entries;
    std::vector<int32_t> src_pairs;
    std::vector<FastJob> jobs;
    std::vector<int2> pieces;
};

// Blending-table entries and queries of every output frame.  Positions t of the table
// run over the clip (rev = 0) or the reversed clip (rev = 1, frame N - 1 - t).  Entry
// (rev, j, L) sums the 2^L positions [j - 2^L + 1, j] remapped to position j; the query
// for [l, r] walks t = r, r - 2^L, ... with the largest L whose low L bits of t are set
// and whose entry stays in [l, r] (Alg. 5), each piece remapped to position r.
void plan_fast(int N, int window, FastPlan& plan) {
    const int M = (window - 1) / 2;
    std::map<std::pair<int, int>, int> pair_of;
    std::map<std::array<int, 3>, int> entry_of;
    auto frame = [N](int rev, int t) { return rev ? N - 1 - t : t; };
    auto get_pair = [&](int src, int tgt) {
        auto it = pair_of.find({src, tgt});
        if (it != pair_of.end()) return it->second;
        const int id = static_cast<int>(plan.pairs.size());
        plan.pairs.push_back(PairDesc{src, tgt, fb_pair_tag(src, tgt), src, 1u, {0, 0, 0}});
        pair_of[{src, tgt}] = id;
        return id;
    };
    auto get_entry = [&](int rev, int j, int L) {
        const std::array<int, 3> key{rev, j, L};
        auto it = entry_of.find(key);
        if (it != entry_of.end()) return it->second;
        FastEntry e{frame(rev, j), static_cast<int32_t>(plan.src_pairs.size()), 0, 0};
        for (int a = j - (1 << L) + 1; a < j; ++a) plan.src_pairs.push_back(get_pair(frame(rev, a), frame(rev, j)));
        e.n_src = static_cast<int32_t>(plan.src_pairs.size()) - e.first_src;
        const int id = static_cast<int>(plan.entries.size());
        plan.entries.push_back(e);
        entry_of[key] = id;
        return id;
    };
    for (int i = 0; i < N; ++i) {
        const int lo = i - M < 0 ? 0 : i - M, hi = i + M > N - 1 ? N - 1 : i + M;
        FastJob job{i, static_cast<int32_t>(plan.pieces.size()), 0, hi - lo + 1};
        const int spans[2][3] = {{0, lo, i}, {1, N - 1 - hi, N - 1 - i}};
        for (const auto& sp : spans) {
            const int rev = sp[0], l = sp[1], r = sp[2];
            for (int t = r; t >= l;) {
                int L = 0;
                while (((t >> L) & 1) && t - (1 << (L + 1)) + 1 >= l) ++L;
                const int e = get_entry(rev, t, L);
                const int pr = t == r ? -1 : get_pair(frame(rev, t), frame(rev, r));
                plan.pieces.push_back(make_int2(e, pr));
                t -= 1 << L;
            }
        }
        job.n_pieces = static_cast<int32_t>(plan.pieces.size()) - job.first_piece;
        plan.jobs.push_back(job);
    }
}

int run_fast_pipeline(fb_ctx* ctx, const uint8_t* guides, const uint8_t* styles, int N, int H, int W,
                      const FastPlan& plan, const fb_params* p, float* out, cudaStream_t st) {
    const int k = p->patch;
    const Levels L = level_dims(H, W, p->levels);
    const size_t npx0 = static_cast<size_t>(H) * W;
    const Mem mg = classify(ctx, guides), ms = classify(ctx, styles), mo = classify(ctx, out);
    if (mg == Mem::Invalid || ms == Mem::Invalid || mo == Mem::Invalid)
        return fail(ctx, FB_ERR_ARG, "a device pointer belongs to another device");
    if (!(mg == ms && ms == mo))
        return fail(ctx, FB_ERR_ARG, "guides, styles and out must all be device or all host memory");
    const bool staging = mg == Mem::Host;
    const size_t n_pairs = plan.pairs.size(), n_entries = plan.entries.size();
    if (n_pairs > static_cast<size_t>(kMaxChunkPairs) || n_pairs * npx0 * 16 > pair_budget(ctx) ||
        n_entries > static_cast<size_t>(kMaxChunkPairs))
        return fail(ctx, FB_ERR_UNSUPPORTED, "fast mode holds all %zu NNFs of the call at once; the pair budget does not",
                    n_pairs);
    const size_t fbytes = static_cast<size_t>(N) * npx0 * 3;

    Buffers b;
    FastEntry* d_entries = nullptr;
    int32_t* d_src = nullptr;
    FastJob* d_jobs = nullptr;
    int2* d_pieces = nullptr;
    uint4* d_table = nullptr;
    auto layout = [&](Carver& c) {
        carve(c, b, L, k, N, N, n_pairs, n_pairs > 0 ? n_pairs : 1, 0, staging, fbytes, fbytes, fbytes);
        d_table = c.take<uint4>(n_entries * npx0);
        d_entries = c.take<FastEntry>(n_entries);
        d_src = c.take<int32_t>(plan.src_pairs.size() > 0 ? plan.src_pairs.size() : 1);
        d_jobs = c.take<FastJob>(plan.jobs.size());
        d_pieces = c.take<int2>(plan.pieces.size());
    };
    Carver measure(nullptr);
    layout(measure);
    int rc = ensure_arena(ctx, measure.off);
    if (rc) return rc;
    Carver cv(ctx->arena);
    layout(cv);
    rc = upload_tables(ctx, plan.pairs, {}, b, st);
    if (rc) return rc;
    FB_CUDA(ctx, cudaMemcpyAsync(d_entries, plan.entries.data(), n_entries * sizeof(FastEntry),
                                 cudaMemcpyHostToDevice, st));
    if (!plan.src_pairs.empty())
        FB_CUDA(ctx, cudaMemcpyAsync(d_src, plan.src_pairs.data(), plan.src_pairs.size() * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, st));
    FB_CUDA(ctx, cudaMemcpyAsync(d_jobs, plan.jobs.data(), plan.jobs.size() * sizeof(FastJob),
                                 cudaMemcpyHostToDevice, st));
    FB_CUDA(ctx, cudaMemcpyAsync(d_pieces, plan.pieces.data(), plan.pieces.size() * sizeof(int2),
                                 cudaMemcpyHostToDevice, st));
    const uint8_t* g_dev = guides;
    const uint8_t* s_dev = styles;
    float* o_dev = out;
    // Host buffers as in run_pipeline: styles in on the copy stream while the NNFs are
    // computed (only the tables read them), frames out in groups as their queries finish.
    constexpr int kOutGroups = 4;
    bool frames_in_order = true;
    for (size_t j = 0; j < plan.jobs.size(); ++j)
        frames_in_order = frames_in_order && plan.jobs[j].frame == static_cast<int>(j);
    if (ctx->copy_stream) {  // a failed earlier call may have left copies of the arena in flight
        rc = ensure_xfer(ctx, 1);
        if (rc) return rc;
        FB_CUDA(ctx, cudaEventRecord(ctx->xfer_ev[0], ctx->copy_stream));
        FB_CUDA(ctx, cudaStreamWaitEvent(st, ctx->xfer_ev[0], 0));
    }
    size_t ev = 0;
    if (staging) {
        rc = ensure_xfer(ctx, 2 + kOutGroups + 1);
        if (rc) return rc;
        FB_CUDA(ctx, cudaMemcpyAsync(b.in_guides, guides, fbytes, cudaMemcpyHostToDevice, st));
        FB_CUDA(ctx, cudaEventRecord(ctx->xfer_ev[ev], st));
        FB_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->xfer_ev[ev++], 0));
        FB_CUDA(ctx, cudaMemcpyAsync(b.in_styles, styles, fbytes, cudaMemcpyHostToDevice, ctx->copy_stream));
        FB_CUDA(ctx, cudaEventRecord(ctx->xfer_ev[ev++], ctx->copy_stream));
        g_dev = b.in_guides;
        s_dev = b.in_styles;
        o_dev = b.in_out;
    }
    rc = prep_guides(ctx, b, L, k, g_dev, N, 0, st);
    if (rc) return rc;
    if (p->flags & FB_FLAG_REPORT_ENERGY) {
        FB_CUDA(ctx, cudaMemsetAsync(ctx->energy, 0, sizeof(double), st));
        ctx->energy_count = 0;
    }
    uint32_t *F = b.FA, *E = b.EA;
    if (n_pairs > 0) {
        rc = run_nnf(ctx, b, L, p, 0, static_cast<int>(n_pairs), nullptr, st, &F, &E);
        if (rc) return rc;
        if (p->flags & FB_FLAG_REPORT_ENERGY) {
            FB_LAUNCH(ctx, st, FB_K_ITER, fb::launch_energy_sum(E, n_pairs * npx0, ctx->energy, st));
            ctx->energy_count += static_cast<uint64_t>(n_pairs) * npx0;
        }
    }
    if (staging) FB_CUDA(ctx, cudaStreamWaitEvent(st, ctx->xfer_ev[1], 0));  // the styles are in
    FB_LAUNCH(ctx, st, FB_K_STYLE, fb::launch_style_rgbx(s_dev, static_cast<size_t>(N) * npx0, b.styles, st));
    FB_LAUNCH(ctx, st, FB_K_TABLE, fb::launch_fast_table(k, d_entries, static_cast<int>(n_entries), d_src, b.pairs,
                                                         F, b.styles, H, W, d_table, st));
    const int n_jobs = static_cast<int>(plan.jobs.size());
    if (!staging || !frames_in_order) {
        FB_LAUNCH(ctx, st, FB_K_COMBINE, fb::launch_fast_combine(k, d_jobs, n_jobs, d_pieces, F, d_table, b.styles,
                                                                 H, W, o_dev, st));
        if (staging) FB_CUDA(ctx, cudaMemcpyAsync(out, o_dev, fbytes * sizeof(float), cudaMemcpyDeviceToHost, st));
    } else {
        const int per = (n_jobs + kOutGroups - 1) / kOutGroups;
        for (int j0 = 0; j0 < n_jobs; j0 += per) {
            const int nj = std::min(per, n_jobs - j0);
            FB_LAUNCH(ctx, st, FB_K_COMBINE, fb::launch_fast_combine(k, d_jobs + j0, nj, d_pieces, F, d_table,
                                                                     b.styles, H, W, o_dev, st));
            FB_CUDA(ctx, cudaEventRecord(ctx->xfer_ev[ev], st));
            FB_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->xfer_ev[ev++], 0));
            const size_t f0 = static_cast<size_t>(j0) * npx0 * 3;
            FB_CUDA(ctx, cudaMemcpyAsync(out + f0, o_dev + f0, static_cast<size_t>(nj) * npx0 * 3 * sizeof(float),
                                         cudaMemcpyDeviceToHost, ctx->copy_stream));
        }
    }
    if (staging) {
        FB_CUDA(ctx, cudaEventRecord(ctx->xfer_ev[ev], ctx->copy_stream));
        FB_CUDA(ctx, cudaStreamWaitEvent(st, ctx->xfer_ev[ev++], 0));
        FB_CUDA(ctx, cudaStreamSynchronize(st));
    }
    return FB_OK;
}

}  // namespace

namespace fb {
// Error message of a call that has no context (read back by fb_last_error(NULL)).
void set_null_ctx_error(const char* msg) { g_null_ctx_err = msg; }
}  // namespace fb


// ---------------------------------------------------------------------------------
// Batched submissions (fb_blend_batch)
// ---------------------------------------------------------------------------------
namespace {

using fb::BatchClip;
using fb::BatchJob;
using fb::BatchPair;

struct HostChunk {
    int k = 0;
    std::vector<BatchPair> pairs;
    std::vector<BatchJob> jobs;
    size_t fe_elems = 0;  // sum of H*W over the chunk's pairs
};

int check_clips(fb_ctx* ctx, const fb_clip_desc* clips, int n, const fb_params* p, bool pointers) {
    if (!clips || n < 1) return fail(ctx, FB_ERR_ARG, "clips must be a non-empty host array");
    if (!p) return fail(ctx, FB_ERR_ARG, "params is NULL");
    if (p->levels != 1) return fail(ctx, FB_ERR_UNSUPPORTED, "batched submissions use levels == 1");
    if (p->flags & (FB_FLAG_BALANCED | FB_FLAG_FAST | FB_FLAG_ACCURATE | FB_FLAG_TRACKING | FB_FLAG_ALIGN))
        return fail(ctx, FB_ERR_UNSUPPORTED, "batched submissions use the plain loss and the direct sum");
    for (int c = 0; c < n; ++c) {
        const fb_clip_desc& d = clips[c];
        fb_params q = *p;
        q.patch = d.patch;
        int rc = check_params(ctx, &q, d.H, d.W);
        if (rc) return rc;
        if (d.N < 1 || d.N > 65535) return fail(ctx, FB_ERR_ARG, "clip %d: N = %d outside [1, 65535]", c, d.N);
        if (d.window < 1 || (d.window & 1) == 0)
            return fail(ctx, FB_ERR_ARG, "clip %d: window must be odd and >= 1", c);
        if (d.reserved != 0) return fail(ctx, FB_ERR_ARG, "clip %d: reserved must be 0", c);
        if (pointers) {
            if (!d.guides || !d.styles || !d.out)
                return fail(ctx, FB_ERR_ARG, "clip %d: NULL pointer", c);
            if (classify(ctx, d.guides) != Mem::Device || classify(ctx, d.styles) != Mem::Device ||
                classify(ctx, d.out) != Mem::Device)
                return fail(ctx, FB_ERR_ARG, "clip %d: pointers must be device memory of the context's device", c);
        }
    }
    return FB_OK;
}

// Clips in patch-size order; per patch size, output frames in clip order grouped into
// chunks whose F/E ping-pong (4 words per pixel and pair) fits budget_bytes.
int plan_chunks(fb_ctx* ctx, const fb_clip_desc* clips, int n, size_t budget_bytes,
                std::vector<HostChunk>& chunks) {
    const size_t budget_elems = budget_bytes / (4 * sizeof(uint32_t));
    for (int k = 3; k <= 9; k += 2) {
        HostChunk cur;
        cur.k = k;
        for (int c = 0; c < n; ++c) {
            const fb_clip_desc& d = clips[c];
            if (d.patch != k) continue;
            const size_t npx = static_cast<size_t>(d.H) * d.W;
            const int M = (d.window - 1) / 2;
            for (int i = 0; i < d.N; ++i) {
                const int lo = i - M < 0 ? 0 : i - M, hi = i + M > d.N - 1 ? d.N - 1 : i + M;
                const size_t need = static_cast<size_t>(hi - lo) * npx;
                if (need > budget_elems)
                    return fail(ctx, FB_ERR_OOM, "clip %d frame %d needs %zu NNF words; the budget holds %zu",
                                c, i, need, budget_elems);
                if (cur.fe_elems + need > budget_elems || cur.pairs.size() + (hi - lo) > 0x7FFFFFFF) {
                    chunks.push_back(std::move(cur));
                    cur = HostChunk();
                    cur.k = k;
                }
                BatchJob j{};
                j.clip = c;
                j.frame = i;
                j.first_pair = static_cast<int32_t>(cur.pairs.size());
                j.n_pairs = hi - lo;
                j.den = static_cast<uint32_t>(255 * k * k * (hi - lo + 1));
                cur.jobs.push_back(j);
                for (int jj = lo; jj <= hi; ++jj) {
                    if (jj == i) continue;
                    BatchPair bp{};
                    bp.clip = c;
                    bp.src = jj;
                    bp.tgt = i;
                    bp.style = jj;
                    bp.tag = fb_pair_tag(jj, i);
                    bp.weight = 1u;
                    bp.fe_off = cur.fe_elems;
                    cur.pairs.push_back(bp);
                    cur.fe_elems += npx;
                }
            }
        }
        if (!cur.jobs.empty()) chunks.push_back(std::move(cur));
    }
    return FB_OK;
}

size_t tiles_of(int H, int W, int th) {
    return static_cast<size_t>((W + 31) / 32) * static_cast<size_t>((H + th - 1) / th);
}

// Work units of the persistent kernels: runs of `per_claim` consecutive tiles (tile
// height th) of one pair, pair-major.
void item_maps(const HostChunk& ch, const fb_clip_desc* clips, int th, int per_claim,
               std::vector<int32_t>& ip, std::vector<int32_t>& it) {
    ip.clear();
    it.clear();
    for (size_t p = 0; p < ch.pairs.size(); ++p) {
        const fb_clip_desc& d = clips[ch.pairs[p].clip];
        const size_t nt = tiles_of(d.H, d.W, th);
        for (size_t t = 0; t < nt; t += static_cast<size_t>(per_claim)) {
            ip.push_back(static_cast<int32_t>(p));
            it.push_back(static_cast<int32_t>(t));
        }
    }
}

// Work units of the combine kernel: runs of kCombineTilesPerClaim 32x8 tiles of one
// output frame.
void job_maps(const HostChunk& ch, const fb_clip_desc* clips, std::vector<int32_t>& ij,
              std::vector<int32_t>& it) {
    ij.clear();
    it.clear();
    for (size_t j = 0; j < ch.jobs.size(); ++j) {
        const fb_clip_desc& d = clips[ch.jobs[j].clip];
        const size_t nt = tiles_of(d.H, d.W, 8);
        for (size_t t = 0; t < nt; t += static_cast<size_t>(fb::kCombineTilesPerClaim)) {
            ij.push_back(static_cast<int32_t>(j));
            it.push_back(static_cast<int32_t>(t));
        }
    }
}

std::vector<uint8_t> manifest_key(const fb_clip_desc* clips, int n, const fb_params* p,
                                  uint32_t flags) {
    std::vector<uint8_t> key(sizeof(fb_clip_desc) * n + sizeof(fb_params) + sizeof(flags));
    std::memcpy(key.data(), clips, sizeof(fb_clip_desc) * n);
    fb_params q = *p;
    q.patch = 0;
    q.pair_tag = 0;
    std::memcpy(key.data() + sizeof(fb_clip_desc) * n, &q, sizeof(q));
    std::memcpy(key.data() + sizeof(fb_clip_desc) * n + sizeof(q), &flags, sizeof(flags));
    return key;
}

void drop_entry(fb_ctx::BatchEntry* be) {
    if (be->exec) cudaGraphExecDestroy(be->exec);
    if (be->dev) cudaFree(be->dev);
    for (cudaStream_t x : be->side) cudaStreamDestroy(x);
    for (cudaEvent_t x : be->ev) cudaEventDestroy(x);
    delete be;
}

// Launch modes of a patch size in a batch: the persistent kernels over the flattened work
// list, or per-clip launches of the kernels fb_blend_window uses, one clip segment (the
// consecutive output frames of one clip in a chunk) after another on a few graph branches.
constexpr int kModePersistent = 0, kModePerClip = 1;
constexpr int kPerClipBranches = 3;

// FB_BATCH_MODE(m): launch mode forced to m - 1 (0: tuned).
int forced_mode(uint32_t flags) {
    const uint32_t m = (flags >> 24) & 0x3u;
    return m == 0 ? -1 : static_cast<int>(m) - 1;
}

// A chunk's clip segments: [job0, job0 + nj) of one clip with pairs [pair0, pair0 + np),
// each within the per-call kernels' grid limit (65535 pairs, 65535 jobs).
struct ClipSeg {
    int clip, job0, nj, pair0, np;
};
std::vector<ClipSeg> clip_segments(const HostChunk& ch) {
    std::vector<ClipSeg> out;
    for (size_t j = 0; j < ch.jobs.size(); ++j) {
        const BatchJob& bj = ch.jobs[j];
        if (out.empty() || out.back().clip != bj.clip || out.back().np + bj.n_pairs > kMaxChunkPairs ||
            out.back().nj + 1 > kMaxChunkPairs)
            out.push_back(ClipSeg{bj.clip, static_cast<int>(j), 0, bj.first_pair, 0});
        out.back().nj += 1;
        out.back().np += bj.n_pairs;
    }
    return out;
}

int forced_variant(uint32_t flags) {
    const uint32_t v = (flags >> 8) & 0xFFu;
    return v == 0 ? -1 : static_cast<int>(v) - 1;
}

// FB_BATCH_CLAIM(c): tiles per claim of the iteration kernel forced to c (0: tuned).
int forced_claim(uint32_t flags) {
    const uint32_t c = (flags >> 16) & 0xFFu;
    return c == 0 ? -1 : static_cast<int>(c);
}

// The first pairs of a chunk, enough for about `waves` rounds of tiles over the GPU: the
// autotuner times its candidates on this prefix so that tuning costs a few milliseconds
// whatever the chunk's size.
HostChunk tuning_prefix(const HostChunk& ch, const fb_clip_desc* clips, size_t tiles_wanted) {
    HostChunk t;
    t.k = ch.k;
    size_t tiles = 0;
    for (const BatchPair& bp : ch.pairs) {
        if (tiles >= tiles_wanted) break;
        t.pairs.push_back(bp);
        tiles += tiles_of(clips[bp.clip].H, clips[bp.clip].W, 8);
    }
    return t;
}

// Builds a cache entry: device tables and scratch, tuning, the list of launches and,
// unless FB_BATCH_NO_GRAPH, the instantiated graph of the whole submission.
int build_entry(fb_ctx* ctx, const fb_clip_desc* clips, int n, const fb_params* p, uint32_t flags,
                cudaStream_t st, fb_ctx::BatchEntry* be) {
    std::vector<HostChunk> chunks;
    int rc = plan_chunks(ctx, clips, n, pair_budget(ctx), chunks);
    if (rc) return rc;
    int sms = 0;
    FB_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));

    // ---- device layout ----
    Carver cv(nullptr);
    struct ClipBufs { uint32_t* rp; uint32_t* sty; };
    size_t n_counters = 2;  // tuning launches
    for (const HostChunk& ch : chunks) n_counters += 2 + static_cast<size_t>(p->iters);
    auto layout = [&](Carver& c, BatchClip** d_clips, std::vector<ClipBufs>& cb,
                      uint32_t** fe, std::vector<std::array<void*, 10>>& tabs, int** counters) {
        *counters = c.take<int>(n_counters);
        *d_clips = c.take<BatchClip>(n);
        cb.assign(n, ClipBufs{});
        for (int i = 0; i < n; ++i) {
            const size_t npx = static_cast<size_t>(clips[i].H) * clips[i].W;
            cb[i].rp = c.take<uint32_t>(static_cast<size_t>(clips[i].N) *
                                        fb::rowpatch_frame_words(clips[i].patch, clips[i].H, clips[i].W));
            cb[i].sty = c.take<uint32_t>(static_cast<size_t>(clips[i].N) * npx);
        }
        size_t max_fe = 1;
        for (const HostChunk& ch : chunks) max_fe = std::max(max_fe, ch.fe_elems);
        for (int q = 0; q < 4; ++q) fe[q] = c.take<uint32_t>(max_fe);
        tabs.assign(chunks.size(), {});
        for (size_t ci = 0; ci < chunks.size(); ++ci) {
            const HostChunk& ch = chunks[ci];
            size_t max_items = 0;  // the 32x4 variant has the most tiles
            for (const BatchPair& bp : ch.pairs) max_items += tiles_of(clips[bp.clip].H, clips[bp.clip].W, 4);
            size_t job_items = 0;
            for (const BatchJob& j : ch.jobs) job_items += tiles_of(clips[j.clip].H, clips[j.clip].W, 8);
            tabs[ci][0] = c.take<BatchPair>(std::max<size_t>(ch.pairs.size(), 1));
            tabs[ci][1] = c.take<int32_t>(std::max<size_t>(max_items, 1));
            tabs[ci][2] = c.take<int32_t>(std::max<size_t>(max_items, 1));
            tabs[ci][3] = c.take<BatchJob>(std::max<size_t>(ch.jobs.size(), 1));
            tabs[ci][4] = c.take<int32_t>(std::max<size_t>(job_items, 1));
            tabs[ci][5] = c.take<int32_t>(std::max<size_t>(job_items, 1));
            tabs[ci][6] = c.take<int32_t>(std::max<size_t>(max_items, 1));  // init units
            tabs[ci][7] = c.take<int32_t>(std::max<size_t>(max_items, 1));
            // the per-call kernels' pair and job tables of the chunk (per-clip mode)
            tabs[ci][8] = c.take<PairDesc>(std::max<size_t>(ch.pairs.size(), 1));
            tabs[ci][9] = c.take<JobDesc>(std::max<size_t>(ch.jobs.size(), 1));
        }
    };
    BatchClip* d_clips = nullptr;
    std::vector<ClipBufs> cb;
    uint32_t* fe[4] = {};
    std::vector<std::array<void*, 10>> tabs;
    int* counters = nullptr;
    layout(cv, &d_clips, cb, fe, tabs, &counters);
    be->bytes = align_up(cv.off, 1 << 20);
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&be->dev), be->bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        be->dev = nullptr;
        return fail(ctx, FB_ERR_OOM, "batch scratch of %zu bytes: %s", be->bytes, cudaGetErrorString(e));
    }
    Carver real(be->dev);
    layout(real, &d_clips, cb, fe, tabs, &counters);

    // ---- static tables ----
    std::vector<BatchClip> hclips(n);
    for (int i = 0; i < n; ++i) {
        const int r0 = p->r0 > 0 ? p->r0 : std::max(clips[i].H, clips[i].W);
        hclips[i] = BatchClip{clips[i].H, clips[i].W, clips[i].N, r0, cb[i].rp, cb[i].sty, clips[i].out};
    }
    FB_CUDA(ctx, cudaMemcpy(d_clips, hclips.data(), sizeof(BatchClip) * n, cudaMemcpyHostToDevice));
    std::vector<int32_t> m0, m1;
    std::vector<int> job_units(chunks.size(), 0);
    for (size_t ci = 0; ci < chunks.size(); ++ci) {
        const HostChunk& ch = chunks[ci];
        if (!ch.pairs.empty())
            FB_CUDA(ctx, cudaMemcpy(tabs[ci][0], ch.pairs.data(), sizeof(BatchPair) * ch.pairs.size(),
                                    cudaMemcpyHostToDevice));
        FB_CUDA(ctx, cudaMemcpy(tabs[ci][3], ch.jobs.data(), sizeof(BatchJob) * ch.jobs.size(),
                                cudaMemcpyHostToDevice));
        job_maps(ch, clips, m0, m1);
        job_units[ci] = static_cast<int>(m0.size());
        FB_CUDA(ctx, cudaMemcpy(tabs[ci][4], m0.data(), sizeof(int32_t) * m0.size(), cudaMemcpyHostToDevice));
        FB_CUDA(ctx, cudaMemcpy(tabs[ci][5], m1.data(), sizeof(int32_t) * m1.size(), cudaMemcpyHostToDevice));
        // The same NNFs in the per-call kernels' tables: what blend_pairs builds for the clip
        // (frame slots of the clip, the clip-frame streams), pair indices of the chunk.
        std::vector<PairDesc> pd(ch.pairs.size());
        for (size_t q = 0; q < ch.pairs.size(); ++q) {
            const BatchPair& bp = ch.pairs[q];
            pd[q] = PairDesc{bp.src, bp.tgt, bp.tag, bp.style, bp.weight, {-1, -1, -1}};
        }
        std::vector<JobDesc> jd(ch.jobs.size());
        for (size_t q = 0; q < ch.jobs.size(); ++q) {
            const BatchJob& bj = ch.jobs[q];
            jd[q] = JobDesc{bj.frame, bj.frame, 1u, bj.first_pair, bj.n_pairs, bj.den, {0, 0}};
        }
        if (!pd.empty())
            FB_CUDA(ctx, cudaMemcpy(tabs[ci][8], pd.data(), sizeof(PairDesc) * pd.size(), cudaMemcpyHostToDevice));
        FB_CUDA(ctx, cudaMemcpy(tabs[ci][9], jd.data(), sizeof(JobDesc) * jd.size(), cudaMemcpyHostToDevice));
    }

    // ---- the launches of one submission ----
    // First the work counters of the persistent launches are zeroed (kind -1: not a kernel).
    be->steps.push_back([counters, n_counters](cudaStream_t s) {
        return cudaMemsetAsync(counters, 0, n_counters * sizeof(int), s);
    });
    be->step_kind.push_back(-1);
    for (int i = 0; i < n; ++i) {
        const fb_clip_desc d = clips[i];
        const ClipBufs b = cb[i];
        be->steps.push_back([d, b](cudaStream_t s) {
            return fb::launch_prep_guides(d.patch, d.guides, d.N, d.H, d.W, b.rp, s);
        });
        be->step_kind.push_back(FB_K_PREP);
        be->steps.push_back([d, b](cudaStream_t s) {
            return fb::launch_style_rgbx(d.styles, static_cast<size_t>(d.N) * d.H * d.W, b.sty, s);
        });
        be->step_kind.push_back(FB_K_STYLE);
    }
    // Tile variant and iteration claim size per patch size: forced, tuned earlier in this
    // context, or tuned now.  Every (variant, claim) candidate -- the ones not forced -- runs
    // iterations 1-2 (after an untimed iteration 0) over a prefix of the size's first chunk
    // (about 32 rounds of 32x8 tiles over the GPU); the fastest is kept.  All candidates give
    // the same results.
    int variant_of[10], claim_of[10], mode_of[10];
    for (int k = 0; k < 10; ++k) {
        variant_of[k] = forced_variant(flags) >= 0 ? forced_variant(flags) : ctx->tuned_variant[k];
        claim_of[k] = forced_claim(flags) >= 0 ? forced_claim(flags) : ctx->tuned_claim[k];
        mode_of[k] = forced_mode(flags) >= 0 ? forced_mode(flags) : ctx->tuned_mode[k];
        if (forced_variant(flags) >= 0 || forced_claim(flags) >= 0)
            mode_of[k] = forced_mode(flags) >= 0 ? forced_mode(flags) : kModePersistent;
        if (forced_variant(flags) < 0 && forced_claim(flags) >= 0 && ctx->tuned_variant[k] >= 0 &&
            ctx->tuned_claim[k] != forced_claim(flags))
            variant_of[k] = -1;   // the variant was tuned for another claim size: tune again
        if (forced_claim(flags) < 0 && forced_variant(flags) >= 0 && ctx->tuned_claim[k] >= 0 &&
            ctx->tuned_variant[k] != forced_variant(flags))
            claim_of[k] = -1;
    }
    bool prepped = false;
    for (size_t ci = 0; ci < chunks.size(); ++ci) {
        const HostChunk& full_ch = chunks[ci];
        if ((variant_of[full_ch.k] >= 0 && claim_of[full_ch.k] >= 0 && mode_of[full_ch.k] >= 0) ||
            full_ch.pairs.empty())
            continue;
        const HostChunk ch = tuning_prefix(full_ch, clips, static_cast<size_t>(sms) * 8 * 32);
        if (!prepped) {
            for (size_t q = 0; q < 1 + 2 * static_cast<size_t>(n); ++q) FB_CUDA(ctx, be->steps[q](st));
            prepped = true;
        }
        const BatchPair* d_pairs = static_cast<const BatchPair*>(tabs[ci][0]);
        int32_t* d_ip = static_cast<int32_t*>(tabs[ci][1]);
        int32_t* d_it = static_cast<int32_t*>(tabs[ci][2]);
        int32_t* d_ip0 = static_cast<int32_t*>(tabs[ci][6]);
        int32_t* d_it0 = static_cast<int32_t*>(tabs[ci][7]);
        std::vector<int32_t> u0, u1;
        float best = 0.f;
        int best_v = -1, best_c = -1;
        cudaEvent_t a = nullptr, b = nullptr;
        FB_CUDA(ctx, cudaEventCreate(&a));
        FB_CUDA(ctx, cudaEventCreate(&b));
        std::vector<int> claim_list(fb::kIterClaimChoices, fb::kIterClaimChoices + fb::kIterClaimCount);
        if (claim_of[ch.k] >= 0) claim_list.assign(1, claim_of[ch.k]);
        for (int cand = 0; cand < fb::kBatchVariants * static_cast<int>(claim_list.size()); ++cand) {
            const int v = cand / static_cast<int>(claim_list.size());
            const int claim = claim_list[cand % claim_list.size()];
            if (variant_of[ch.k] >= 0 && v != variant_of[ch.k]) continue;
            item_maps(ch, clips, fb::batch_variant_tile_h(v), claim, m0, m1);
            item_maps(ch, clips, fb::batch_variant_tile_h(v), fb::kInitTilesPerClaim, u0, u1);
            FB_CUDA(ctx, cudaMemcpyAsync(d_ip, m0.data(), sizeof(int32_t) * m0.size(), cudaMemcpyHostToDevice, st));
            FB_CUDA(ctx, cudaMemcpyAsync(d_it, m1.data(), sizeof(int32_t) * m1.size(), cudaMemcpyHostToDevice, st));
            FB_CUDA(ctx, cudaMemcpyAsync(d_ip0, u0.data(), sizeof(int32_t) * u0.size(), cudaMemcpyHostToDevice, st));
            FB_CUDA(ctx, cudaMemcpyAsync(d_it0, u1.data(), sizeof(int32_t) * u1.size(), cudaMemcpyHostToDevice, st));
            const int grid = sms * fb::batch_iter_blocks_per_sm(ch.k, v);
            FB_CUDA(ctx, cudaMemsetAsync(counters, 0, 2 * sizeof(int), st));
            FB_CUDA(ctx, fb::launch_batch_init(ch.k, v, d_pairs, d_clips, d_ip0, d_it0, static_cast<int>(u0.size()),
                                               counters, p->seed, fe[0], fe[1], grid, st));
            // One untimed iteration, then two timed ones (ping-pong F/E; results discarded).
            for (int it = 0; it < 3; ++it) {
                if (it == 1) FB_CUDA(ctx, cudaEventRecord(a, st));
                const int s0 = (it & 1) ? 2 : 0, s1 = (it & 1) ? 0 : 2;
                FB_CUDA(ctx, cudaMemsetAsync(counters + 1, 0, sizeof(int), st));
                FB_CUDA(ctx, fb::launch_batch_iter(ch.k, v, d_pairs, d_clips, d_ip, d_it, static_cast<int>(m0.size()),
                                                   claim, counters + 1, p->seed, it, fe[s0], fe[s0 + 1], fe[s1],
                                                   fe[s1 + 1], grid, st));
            }
            FB_CUDA(ctx, cudaEventRecord(b, st));
            FB_CUDA(ctx, cudaEventSynchronize(b));
            float ms = 0.f;
            FB_CUDA(ctx, cudaEventElapsedTime(&ms, a, b));
            ctx->launches += 4;
            if (best_v < 0 || ms < best) {
                best = ms;
                best_v = v;
                best_c = claim;
            }
        }
        // The per-clip mode on the same prefix: the per-call kernels over each run of one
        // clip's pairs, the same untimed iteration and two timed ones.
        float per_clip_ms = -1.f;
        if (mode_of[ch.k] < 0) {
            const PairDesc* d_pd = static_cast<const PairDesc*>(tabs[ci][8]);
            std::vector<std::array<int, 3>> runs;  // clip, first pair, pairs
            for (size_t q = 0; q < ch.pairs.size(); ++q) {
                if (runs.empty() || runs.back()[0] != ch.pairs[q].clip)
                    runs.push_back({ch.pairs[q].clip, static_cast<int>(q), 0});
                runs.back()[2] += 1;
            }
            for (int it = -1; it < 3; ++it) {
                if (it == 1) FB_CUDA(ctx, cudaEventRecord(a, st));
                for (const auto& rn : runs) {
                    const fb_clip_desc& d = clips[rn[0]];
                    const LevelGeom g{d.H, d.W, cb[rn[0]].rp};
                    const size_t off = ch.pairs[rn[1]].fe_off;
                    const int r0 = p->r0 > 0 ? p->r0 : std::max(d.H, d.W);
                    if (it < 0) {
                        FB_CUDA(ctx, fb::launch_nnf_init(ch.k, d_pd, rn[1], rn[2], g, 0, nullptr, 0, 0, nullptr,
                                                         p->seed, 0, fe[0] + off, fe[1] + off, st));
                    } else {
                        const int s0 = (it & 1) ? 2 : 0, s1 = (it & 1) ? 0 : 2;
                        FB_CUDA(ctx, fb::launch_nnf_iter(ch.k, d_pd, rn[1], rn[2], g, r0, p->seed, 0, it,
                                                         fe[s0] + off, fe[s0 + 1] + off, fe[s1] + off,
                                                         fe[s1 + 1] + off, st));
                    }
                }
            }
            FB_CUDA(ctx, cudaEventRecord(b, st));
            FB_CUDA(ctx, cudaEventSynchronize(b));
            FB_CUDA(ctx, cudaEventElapsedTime(&per_clip_ms, a, b));
            ctx->launches += 4 * runs.size();
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        variant_of[ch.k] = best_v;
        claim_of[ch.k] = best_c;
        if (mode_of[ch.k] < 0) mode_of[ch.k] = per_clip_ms >= 0.f && per_clip_ms < best ? kModePerClip : kModePersistent;
        if (forced_variant(flags) < 0 && forced_claim(flags) < 0 && forced_mode(flags) < 0) {
            ctx->tuned_variant[ch.k] = best_v;   // a free choice: remember it
            ctx->tuned_claim[ch.k] = best_c;
            ctx->tuned_mode[ch.k] = mode_of[ch.k];
        }
    }
    int* next_counter = counters + 2;
    // Per-clip chunks spread their clip segments over side streams (graph branches) when the
    // submission is captured; launched directly, they run on the caller's stream.
    const bool branches = !(flags & FB_BATCH_NO_GRAPH);
    bool any_per_clip = false;
    for (const HostChunk& ch : chunks) any_per_clip = any_per_clip || mode_of[ch.k] == kModePerClip;
    if (branches && any_per_clip) {
        for (int q = 0; q < kPerClipBranches; ++q) {
            cudaStream_t x = nullptr;
            FB_CUDA(ctx, cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
            be->side.push_back(x);
        }
    }
    for (size_t ci = 0; ci < chunks.size(); ++ci) {
        const HostChunk& ch = chunks[ci];
        if (mode_of[ch.k] == kModePerClip) {
            // The kernels and tables fb_blend_window uses, segment by segment (bit-identical
            // results: the same pairs, streams and schedule).
            const int k = ch.k;
            const uint64_t seed = p->seed;
            const int iters = p->iters;
            const PairDesc* d_pd = static_cast<const PairDesc*>(tabs[ci][8]);
            const JobDesc* d_jd = static_cast<const JobDesc*>(tabs[ci][9]);
            cudaEvent_t fork = nullptr;
            std::vector<cudaEvent_t> joins;
            if (branches) {
                FB_CUDA(ctx, cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
                be->ev.push_back(fork);
                for (size_t b = 0; b < be->side.size(); ++b) {
                    cudaEvent_t e2 = nullptr;
                    FB_CUDA(ctx, cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
                    be->ev.push_back(e2);
                    joins.push_back(e2);
                }
                const std::vector<cudaStream_t> side = be->side;
                be->steps.push_back([fork, side](cudaStream_t s) {
                    cudaError_t e2 = cudaEventRecord(fork, s);
                    for (cudaStream_t x : side)
                        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(x, fork, 0);
                    return e2;
                });
                be->step_kind.push_back(-1);
            }
            const std::vector<ClipSeg> segs = clip_segments(ch);
            for (size_t q = 0; q < segs.size(); ++q) {
                const ClipSeg sg = segs[q];
                if (sg.np <= 0 && sg.nj <= 0) continue;
                const fb_clip_desc d = clips[sg.clip];
                const LevelGeom g{d.H, d.W, cb[sg.clip].rp};
                const uint32_t* sty = cb[sg.clip].sty;
                const int r0 = p->r0 > 0 ? p->r0 : std::max(d.H, d.W);
                const size_t off = sg.np > 0 ? ch.pairs[sg.pair0].fe_off : 0;
                cudaStream_t side = branches ? be->side[q % be->side.size()] : nullptr;
                auto on = [side](cudaStream_t s) { return side ? side : s; };
                uint32_t *Fc = fe[0] + off, *Ec = fe[1] + off, *Fo = fe[2] + off, *Eo = fe[3] + off;
                if (sg.np > 0) {
                    be->steps.push_back([=](cudaStream_t s) {
                        return fb::launch_nnf_init(k, d_pd, sg.pair0, sg.np, g, 0, nullptr, 0, 0, nullptr, seed, 0, Fc,
                                                   Ec, on(s));
                    });
                    be->step_kind.push_back(FB_K_INIT);
                    for (int it = 0; it < iters; ++it) {
                        uint32_t *a = Fc, *ea = Ec, *b = Fo, *eb = Eo;
                        be->steps.push_back([=](cudaStream_t s) {
                            return fb::launch_nnf_iter(k, d_pd, sg.pair0, sg.np, g, r0, seed, 0, it, a, ea, b, eb, on(s));
                        });
                        be->step_kind.push_back(FB_K_ITER);
                        std::swap(Fc, Fo);
                        std::swap(Ec, Eo);
                    }
                }
                const uint32_t* Ffin = Fc;
                float* out = d.out;
                be->steps.push_back([=](cudaStream_t s) {
                    return fb::launch_combine(k, d_jd, sg.job0, sg.nj, d_pd, sg.pair0, Ffin, sty, d.H, d.W, out, on(s));
                });
                be->step_kind.push_back(FB_K_COMBINE);
            }
            if (branches) {
                const std::vector<cudaStream_t> side = be->side;
                be->steps.push_back([joins, side](cudaStream_t s) {
                    cudaError_t e2 = cudaSuccess;
                    for (size_t b = 0; b < side.size() && e2 == cudaSuccess; ++b) {
                        e2 = cudaEventRecord(joins[b], side[b]);
                        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, joins[b], 0);
                    }
                    return e2;
                });
                be->step_kind.push_back(-1);
            }
            continue;
        }
        const int v = variant_of[ch.k] >= 0 ? variant_of[ch.k] : 0;
        const int claim = claim_of[ch.k] >= 0 ? claim_of[ch.k] : fb::kIterTilesPerClaim;
        std::vector<int32_t> u0, u1;
        item_maps(ch, clips, fb::batch_variant_tile_h(v), claim, m0, m1);
        item_maps(ch, clips, fb::batch_variant_tile_h(v), fb::kInitTilesPerClaim, u0, u1);
        if (!m0.empty()) {
            FB_CUDA(ctx, cudaMemcpyAsync(tabs[ci][1], m0.data(), sizeof(int32_t) * m0.size(), cudaMemcpyHostToDevice, st));
            FB_CUDA(ctx, cudaMemcpyAsync(tabs[ci][2], m1.data(), sizeof(int32_t) * m1.size(), cudaMemcpyHostToDevice, st));
            FB_CUDA(ctx, cudaMemcpyAsync(tabs[ci][6], u0.data(), sizeof(int32_t) * u0.size(), cudaMemcpyHostToDevice, st));
            FB_CUDA(ctx, cudaMemcpyAsync(tabs[ci][7], u1.data(), sizeof(int32_t) * u1.size(), cudaMemcpyHostToDevice, st));
        }
        FB_CUDA(ctx, cudaStreamSynchronize(st));  // host vectors are reused
        const int n_items = static_cast<int>(m0.size());
        const int n_init_units = static_cast<int>(u0.size());
        const int k = ch.k;
        const uint64_t seed = p->seed;
        const int iters = p->iters;
        const int grid = sms * fb::batch_iter_blocks_per_sm(k, v);
        const int cgrid = sms * 8;
        const BatchPair* d_pairs = static_cast<const BatchPair*>(tabs[ci][0]);
        const int32_t* d_ip = static_cast<const int32_t*>(tabs[ci][1]);
        const int32_t* d_it = static_cast<const int32_t*>(tabs[ci][2]);
        const int32_t* d_ip0 = static_cast<const int32_t*>(tabs[ci][6]);
        const int32_t* d_it0 = static_cast<const int32_t*>(tabs[ci][7]);
        const BatchJob* d_jobs = static_cast<const BatchJob*>(tabs[ci][3]);
        const int32_t* d_ij = static_cast<const int32_t*>(tabs[ci][4]);
        const int32_t* d_ijt = static_cast<const int32_t*>(tabs[ci][5]);
        uint32_t *Fc = fe[0], *Ec = fe[1], *Fo = fe[2], *Eo = fe[3];
        if (n_items > 0) {
            int* cnt = next_counter++;
            be->steps.push_back([=](cudaStream_t s) {
                return fb::launch_batch_init(k, v, d_pairs, d_clips, d_ip0, d_it0, n_init_units, cnt, seed, Fc, Ec, grid, s);
            });
            be->step_kind.push_back(FB_K_INIT);
            for (int it = 0; it < iters; ++it) {
                uint32_t *a = Fc, *ea = Ec, *b = Fo, *eb = Eo;
                int* cnt_it = next_counter++;
                be->steps.push_back([=](cudaStream_t s) {
                    return fb::launch_batch_iter(k, v, d_pairs, d_clips, d_ip, d_it, n_items, claim, cnt_it, seed, it, a,
                                                 ea, b, eb, grid, s);
                });
                be->step_kind.push_back(FB_K_ITER);
                std::swap(Fc, Fo);
                std::swap(Ec, Eo);
            }
        }
        const uint32_t* Ffinal = Fc;
        const int jn = job_units[ci];
        int* cnt_c = next_counter++;
        be->steps.push_back([=](cudaStream_t s) {
            return fb::launch_batch_combine(k, d_jobs, d_pairs, d_clips, d_ij, d_ijt, jn, cnt_c, Ffinal, cgrid, s);
        });
        be->step_kind.push_back(FB_K_COMBINE);
    }
    be->launches_per_run = 0;
    for (int kind : be->step_kind) be->launches_per_run += kind >= 0 ? 1 : 0;

    if (!(flags & FB_BATCH_NO_GRAPH)) {
        // Capture on a private stream (the legacy default stream cannot be captured);
        // nothing runs during capture.  The graph is launched on the caller's stream.
        cudaStream_t cap = nullptr;
        FB_CUDA(ctx, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t be_ = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (be_ != cudaSuccess) {
            cudaStreamDestroy(cap);
            return fail(ctx, FB_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(be_));
        }
        cudaError_t le = cudaSuccess;
        for (auto& f : be->steps)
            if (le == cudaSuccess) le = f(cap);
        cudaError_t ce = cudaStreamEndCapture(cap, &g);
        cudaStreamDestroy(cap);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return fail(ctx, FB_ERR_CUDA, "graph capture of the batch failed: %s",
                        cudaGetErrorString(le != cudaSuccess ? le : ce));
        }
        e = cudaGraphInstantiate(&be->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            be->exec = nullptr;
            return fail(ctx, FB_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
        }
    }
    return FB_OK;
}

}  // namespace

extern "C" int fb_batch_plan(const fb_clip_desc* clips, int n_clips, const fb_params* p,
                             size_t budget_bytes, uint64_t* n_pairs, uint64_t* n_items,
                             int* n_chunks) {
    int rc = check_clips(nullptr, clips, n_clips, p, false);
    if (rc) return rc;
    std::vector<HostChunk> chunks;
    rc = plan_chunks(nullptr, clips, n_clips, budget_bytes ? budget_bytes : kPairBudgetBytes, chunks);
    if (rc) return rc;
    uint64_t np = 0, ni = 0;
    for (const HostChunk& ch : chunks) {
        np += ch.pairs.size();
        for (const BatchPair& bp : ch.pairs) ni += tiles_of(clips[bp.clip].H, clips[bp.clip].W, 8);
    }
    if (n_pairs) *n_pairs = np;
    if (n_items) *n_items = ni;
    if (n_chunks) *n_chunks = static_cast<int>(chunks.size());
    return FB_OK;
}

namespace fb {
void count_launches(fb_ctx* ctx, int n) {
    if (ctx) ctx->launches += static_cast<uint64_t>(n);
}
}  // namespace fb

extern "C" int fb_pair_plan(int N, int window, const int32_t* key_idx, int n_keys, uint32_t flags,
                            fb_pair_info* out, size_t cap, size_t* n_pairs) {
    if (N < 1 || N > 65535) return FB_ERR_ARG;
    if (flags & ~(FB_FLAG_TRACKING | FB_FLAG_ALIGN)) return FB_ERR_ARG;
    std::vector<PairDesc> pairs;
    std::vector<JobDesc> jobs;
    if (window > 0) {
        if ((window & 1) == 0 || key_idx || n_keys || (flags & FB_FLAG_ALIGN)) return FB_ERR_ARG;
        blend_pairs(N, 3, window, flags, pairs, jobs);
    } else {
        if (window < 0 || !key_idx || n_keys < 1 || n_keys > N) return FB_ERR_ARG;
        for (int m = 0; m < n_keys; ++m)
            if (key_idx[m] < 0 || key_idx[m] >= N || (m > 0 && key_idx[m] <= key_idx[m - 1])) return FB_ERR_ARG;
        interp_pairs(N, 3, key_idx, n_keys, flags, pairs, jobs);
    }
    if (n_pairs) *n_pairs = pairs.size();
    if (!out) return FB_OK;
    if (cap < pairs.size()) return FB_ERR_ARG;
    for (const JobDesc& j : jobs)
        for (int q = 0; q < j.n_pairs; ++q) {
            const PairDesc& pd = pairs[j.first_pair + q];
            out[j.first_pair + q] = fb_pair_info{pd.src, pd.tgt, pd.tag, pd.weight, pd.pad[0], pd.pad[1],
                                                 pd.pad[2], j.out_frame};
        }
    return FB_OK;
}

extern "C" int fb_pair_plan_range(int N, int window, const int32_t* key_idx, int n_keys, uint32_t flags,
                                  int out_first, int n_out, fb_pair_info* out, size_t cap, size_t* n_pairs) {
    if (N < 1 || N > 65535 || n_out < 1 || out_first < 0 || out_first + n_out > N) return FB_ERR_ARG;
    if (flags & ~FB_FLAG_ALIGN) return FB_ERR_ARG;  // tracking has no range form
    std::vector<PairDesc> pairs;
    std::vector<JobDesc> jobs;
    if (window > 0) {
        if ((window & 1) == 0 || key_idx || n_keys || (flags & FB_FLAG_ALIGN)) return FB_ERR_ARG;
        blend_pairs(N, 3, window, flags, pairs, jobs, out_first, out_first + n_out, 0);
    } else {
        if (window < 0 || !key_idx || n_keys < 1 || n_keys > N) return FB_ERR_ARG;
        for (int m = 0; m < n_keys; ++m)
            if (key_idx[m] < 0 || key_idx[m] >= N || (m > 0 && key_idx[m] <= key_idx[m - 1])) return FB_ERR_ARG;
        interp_pairs(N, 3, key_idx, n_keys, flags, pairs, jobs, out_first, out_first + n_out);
    }
    if (n_pairs) *n_pairs = pairs.size();
    if (!out) return FB_OK;
    if (cap < pairs.size()) return FB_ERR_ARG;
    for (const JobDesc& j : jobs)
        for (int q = 0; q < j.n_pairs; ++q) {
            const PairDesc& pd = pairs[j.first_pair + q];
            out[j.first_pair + q] = fb_pair_info{pd.src, pd.tgt, pd.tag, pd.weight, pd.pad[0], pd.pad[1],
                                                 pd.pad[2], out_first + j.out_frame};
        }
    return FB_OK;
}

extern "C" int fb_shard_plan(int N, int window, int n_shards, int shard, int* frame_base, int* n_in,
                             int* out_first, int* n_out) {
    if (N < 1 || N > 65535 || window < 0 || (window > 0 && (window & 1) == 0)) return FB_ERR_ARG;
    if (n_shards < 1 || n_shards > N || shard < 0 || shard >= n_shards) return FB_ERR_ARG;
    // Work per output frame: its NNFs (blend: the truncated window's other frames), or one
    // unit per frame for interpolation.  Shard s takes the output frames whose cumulative
    // work before them lies in [s T / n, (s + 1) T / n) (T the total), so the shards are
    // contiguous, cover the clip once and carry about equal work; each keeps at least one
    // frame (n_shards <= N).
    const int M = window > 0 ? (window - 1) / 2 : 0;
    auto work = [&](int i) -> uint64_t {
        if (window == 0) return 1;
        const int lo = i - M < 0 ? 0 : i - M, hi = i + M > N - 1 ? N - 1 : i + M;
        return static_cast<uint64_t>(hi - lo) + 1;  // + 1: the frame's own combine
    };
    uint64_t total = 0;
    for (int i = 0; i < N; ++i) total += work(i);
    std::vector<int> start(n_shards + 1, N);
    start[0] = 0;
    uint64_t acc = 0;
    int s = 1;
    for (int i = 0; i < N && s < n_shards; ++i) {
        // frame i opens shard s once the work before it reaches s/n of the total
        while (s < n_shards && acc * n_shards >= total * static_cast<uint64_t>(s)) start[s++] = i;
        acc += work(i);
    }
    for (int q = 1; q <= n_shards; ++q) {  // at least one frame per shard
        const int lo = start[q - 1] + 1, hi = N - (n_shards - q);
        if (q < n_shards) start[q] = start[q] < lo ? lo : start[q] > hi ? hi : start[q];
    }
    const int a = start[shard], b = start[shard + 1];
    const int in_lo = window > 0 ? (a - M < 0 ? 0 : a - M) : 0;
    const int in_hi = window > 0 ? (b + M > N ? N : b + M) : N;
    if (frame_base) *frame_base = in_lo;
    if (n_in) *n_in = in_hi - in_lo;
    if (out_first) *out_first = a;
    if (n_out) *n_out = b - a;
    return FB_OK;
}

extern "C" int fb_fast_plan(int N, int window, uint64_t* n_nnfs, uint64_t* n_entries,
                            uint64_t* n_pieces) {
    if (N < 1 || N > 65535 || window < 1 || (window & 1) == 0) return FB_ERR_ARG;
    FastPlan plan;
    plan_fast(N, window, plan);
    if (n_nnfs) *n_nnfs = plan.pairs.size();
    if (n_entries) *n_entries = plan.entries.size();
    if (n_pieces) *n_pieces = plan.pieces.size();
    return FB_OK;
}

// Checked builds: the device-side check words of the per-call and the batched kernels
// (fb_check.cuh), combined; the product build reports FB_ERR_UNSUPPORTED.
extern "C" int fb_check_status(uint64_t* first, uint64_t* failed, uint64_t* evaluated, int reset) {
#ifdef FB_CHECKED
    unsigned long long a[3] = {}, b[3] = {};
    if (fb::check_read_kernels(a, reset != 0) != cudaSuccess || fb::check_read_batch(b, reset != 0) != cudaSuccess) {
        cudaGetLastError();
        return FB_ERR_CUDA;
    }
    if (first) *first = a[0] ? a[0] : b[0];
    if (failed) *failed = a[1] + b[1];
    if (evaluated) *evaluated = a[2] + b[2];
    return FB_OK;
#else
    (void)first;
    (void)failed;
    (void)evaluated;
    (void)reset;
    return FB_ERR_UNSUPPORTED;
#endif
}

extern "C" int fb_ctx_set_initnet(fb_ctx* ctx, fb_initnet* net) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    ctx->init_net = net;
    return FB_OK;
}

extern "C" int fb_ctx_energy(fb_ctx* ctx, double* sum, uint64_t* count) {
    if (!ctx || !sum || !count) return fail(ctx, FB_ERR_ARG, "NULL argument");
    DeviceGuard dg(ctx->device);
    FB_CUDA(ctx, cudaMemcpy(sum, ctx->energy, sizeof(double), cudaMemcpyDeviceToHost));
    *count = ctx->energy_count;
    return FB_OK;
}

extern "C" int fb_ctx_set_pair_budget(fb_ctx* ctx, size_t bytes) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    if (bytes != 0 && bytes < (size_t(1) << 20))
        return fail(ctx, FB_ERR_ARG, "pair budget below 1 MiB");
    ctx->pair_budget = bytes;
    return FB_OK;
}

extern "C" int fb_ctx_batch_mode(const fb_ctx* ctx, int patch) {
    if (!ctx || patch < 0 || patch > 9) return -1;
    return ctx->tuned_mode[patch];
}

extern "C" int fb_ctx_batch_claim(const fb_ctx* ctx, int patch) {
    if (!ctx || patch < 0 || patch > 9) return -1;
    return ctx->tuned_claim[patch];
}

extern "C" int fb_ctx_batch_variant(const fb_ctx* ctx, int patch) {
    if (!ctx || patch < 0 || patch > 9) return -1;
    return ctx->tuned_variant[patch];
}

extern "C" int fb_blend_batch(fb_ctx* ctx, const fb_clip_desc* clips, int n_clips,
                              const fb_params* p, uint32_t flags, void* stream) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    ctx->err.clear();
    if (flags & ~(FB_BATCH_NO_GRAPH | 0xFF00u | 0xFF0000u | 0x3000000u))
        return fail(ctx, FB_ERR_ARG, "unknown flags 0x%x", flags);
    if (forced_mode(flags) > kModePerClip) return fail(ctx, FB_ERR_ARG, "launch mode %d outside [0, 1]", forced_mode(flags));
    if (forced_mode(flags) == kModePerClip && (forced_variant(flags) >= 0 || forced_claim(flags) >= 0))
        return fail(ctx, FB_ERR_ARG, "a tile variant or claim size applies to the persistent mode only");
    if (forced_variant(flags) >= fb::kBatchVariants)
        return fail(ctx, FB_ERR_ARG, "tile variant %d outside [0, %d)", forced_variant(flags), fb::kBatchVariants);
    if (forced_claim(flags) > 64) return fail(ctx, FB_ERR_ARG, "claim of %d tiles outside [1, 64]", forced_claim(flags));
    DeviceGuard dg(ctx->device);
    int rc = check_clips(ctx, clips, n_clips, p, true);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const std::vector<uint8_t> key = manifest_key(clips, n_clips, p, flags);
    fb_ctx::BatchEntry* be = nullptr;
    for (size_t i = 0; i < ctx->batch_cache.size(); ++i) {
        if (ctx->batch_cache[i]->key == key) {
            be = ctx->batch_cache[i];
            ctx->batch_cache.erase(ctx->batch_cache.begin() + i);
            ctx->batch_cache.push_back(be);
            break;
        }
    }
    if (!be) {
        FB_CUDA(ctx, cudaStreamSynchronize(st));
        while (ctx->batch_cache.size() >= 2) {
            drop_entry(ctx->batch_cache.front());
            ctx->batch_cache.erase(ctx->batch_cache.begin());
        }
        be = new fb_ctx::BatchEntry();
        be->key = key;
        rc = build_entry(ctx, clips, n_clips, p, flags, st, be);
        if (rc) {
            drop_entry(be);
            return rc;
        }
        ctx->batch_cache.push_back(be);
    }
    if (be->exec) {
        FB_CUDA(ctx, cudaGraphLaunch(be->exec, st));
        ctx->launches += be->launches_per_run;
    } else {
        for (size_t i = 0; i < be->steps.size(); ++i) {
            const int kind = be->step_kind[i];
            if (kind < 0)
                FB_CUDA(ctx, be->steps[i](st));
            else
                FB_LAUNCH(ctx, st, kind, be->steps[i](st));
        }
    }
    return FB_OK;
}

extern "C" {

int fb_ctx_create(fb_ctx** out, int device) {
    if (!out) return fail(nullptr, FB_ERR_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, FB_ERR_CUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
    }
    if (device < 0 || device >= n)
        return fail(nullptr, FB_ERR_ARG, "device %d out of range (%d devices)", device, n);
    DeviceGuard dg(device);
    if (!dg.ok) return fail(nullptr, FB_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    fb_ctx* ctx = new fb_ctx();
    ctx->device = device;
    if (cudaEventCreateWithFlags(&ctx->upload_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&ctx->dev_status), sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->dev_status, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&ctx->energy), sizeof(double)) != cudaSuccess ||
        cudaMemset(ctx->energy, 0, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->upload_done) cudaEventDestroy(ctx->upload_done);
        if (ctx->dev_status) cudaFree(ctx->dev_status);
        delete ctx;
        return fail(nullptr, FB_ERR_CUDA, "context set-up failed on device %d", device);
    }
    *out = ctx;
    return FB_OK;
}

int fb_ctx_destroy(fb_ctx* ctx) {
    if (!ctx) return FB_OK;
    DeviceGuard dg(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->arena) cudaFree(ctx->arena);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->upload_done) cudaEventDestroy(ctx->upload_done);
    if (ctx->dev_status) cudaFree(ctx->dev_status);
    if (ctx->energy) cudaFree(ctx->energy);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->xfer_ev) cudaEventDestroy(e);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (fb_ctx::BatchEntry* be : ctx->batch_cache) {
        if (be->exec) cudaGraphExecDestroy(be->exec);
        if (be->dev) cudaFree(be->dev);
        delete be;
    }
    delete ctx;
    return FB_OK;
}

int fb_ctx_sync(fb_ctx* ctx, void* stream) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    DeviceGuard dg(ctx->device);
    FB_CUDA(ctx, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int status = 0;
    FB_CUDA(ctx, cudaMemcpy(&status, ctx->dev_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) {
        FB_CUDA(ctx, cudaMemset(ctx->dev_status, 0, sizeof(int)));
        return fail(ctx, FB_ERR_TIMEOUT, "a bounded device wait expired (code %d)", status);
    }
    return FB_OK;
}

const char* fb_last_error(const fb_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_null_ctx_err.c_str();
}

const char* fb_status_string(int status) {
    switch (status) {
        case FB_OK: return "FB_OK";
        case FB_ERR_ARG: return "FB_ERR_ARG";
        case FB_ERR_CUDA: return "FB_ERR_CUDA";
        case FB_ERR_OOM: return "FB_ERR_OOM";
        case FB_ERR_TIMEOUT: return "FB_ERR_TIMEOUT";
        case FB_ERR_UNSUPPORTED: return "FB_ERR_UNSUPPORTED";
        default: return "FB_ERR_UNKNOWN";
    }
}

uint64_t fb_ctx_launches(const fb_ctx* ctx) { return ctx ? ctx->launches : 0; }

int fb_ctx_profile(fb_ctx* ctx, int enable) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    DeviceGuard dg(ctx->device);
    if (enable) {
        // Events of an earlier record may still be pending; wait before reusing them.
        for (const fb_ctx::Rec& r : ctx->recs) FB_CUDA(ctx, cudaEventSynchronize(r.b));
        ctx->recs.clear();
        ctx->ev_used = 0;
    }
    ctx->profiling = enable != 0;
    return FB_OK;
}

int fb_ctx_profile_read(fb_ctx* ctx, double* ms, uint64_t* launches) {
    if (!ctx || !ms || !launches) return fail(ctx, FB_ERR_ARG, "NULL argument");
    DeviceGuard dg(ctx->device);
    for (int k = 0; k < FB_K_COUNT; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    for (const fb_ctx::Rec& r : ctx->recs) {
        FB_CUDA(ctx, cudaEventSynchronize(r.b));
        float t = 0.f;
        FB_CUDA(ctx, cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.kind] += t;
        launches[r.kind] += 1;
    }
    return FB_OK;
}

size_t fb_ctx_scratch_bytes(const fb_ctx* ctx) { return ctx ? ctx->arena_cap : 0; }

int fb_probe_dp4a(fb_ctx* ctx, double* dp4a_per_s, double* ms) {
    if (!ctx || !dp4a_per_s || !ms) return fail(ctx, FB_ERR_ARG, "NULL argument");
    DeviceGuard dg(ctx->device);
    int sms = 0;
    FB_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const int blocks = sms * 8, iters = 1 << 14;
    Carver measure(nullptr);
    measure.take<uint32_t>(blocks);
    int rc = ensure_arena(ctx, measure.off);
    if (rc) return rc;
    cudaEvent_t a = nullptr, b = nullptr;
    FB_CUDA(ctx, cudaEventCreate(&a));
    FB_CUDA(ctx, cudaEventCreate(&b));
    uint32_t* sink = reinterpret_cast<uint32_t*>(ctx->arena);
    FB_CUDA(ctx, fb::launch_dp4a_probe(blocks, iters / 16, sink, nullptr));  // warm-up
    FB_CUDA(ctx, cudaEventRecord(a, nullptr));
    FB_CUDA(ctx, fb::launch_dp4a_probe(blocks, iters, sink, nullptr));
    FB_CUDA(ctx, cudaEventRecord(b, nullptr));
    FB_CUDA(ctx, cudaEventSynchronize(b));
    float t = 0.f;
    FB_CUDA(ctx, cudaEventElapsedTime(&t, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->launches += 2;
    *ms = t;
    *dp4a_per_s = static_cast<double>(blocks) * 256.0 * iters * fb::kDp4aProbeChains / (t * 1e-3);
    return FB_OK;
}

int fb_probe_ssd_mix(fb_ctx* ctx, int patch, double* byte_pairs_per_s, double* ms) {
    if (!ctx || !byte_pairs_per_s || !ms) return fail(ctx, FB_ERR_ARG, "NULL argument");
    if (patch != 5 && patch != 7) return fail(ctx, FB_ERR_ARG, "patch must be 5 or 7, got %d", patch);
    DeviceGuard dg(ctx->device);
    int sms = 0;
    FB_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const int blocks = sms * 8, iters = 1 << 12;
    Carver measure(nullptr);
    measure.take<uint32_t>(blocks);
    int rc = ensure_arena(ctx, measure.off);
    if (rc) return rc;
    cudaEvent_t a = nullptr, b = nullptr;
    FB_CUDA(ctx, cudaEventCreate(&a));
    FB_CUDA(ctx, cudaEventCreate(&b));
    uint32_t* sink = reinterpret_cast<uint32_t*>(ctx->arena);
    FB_CUDA(ctx, fb::launch_ssd_mix_probe(patch, blocks, iters / 16, sink, nullptr));  // warm-up
    FB_CUDA(ctx, cudaEventRecord(a, nullptr));
    FB_CUDA(ctx, fb::launch_ssd_mix_probe(patch, blocks, iters, sink, nullptr));
    FB_CUDA(ctx, cudaEventRecord(b, nullptr));
    FB_CUDA(ctx, cudaEventSynchronize(b));
    float t = 0.f;
    FB_CUDA(ctx, cudaEventElapsedTime(&t, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->launches += 2;
    *ms = t;
    *byte_pairs_per_s = static_cast<double>(blocks) * 256.0 * iters * 3.0 * patch * patch / (t * 1e-3);
    return FB_OK;
}

int fb_probe_gather(fb_ctx* ctx, size_t bytes, double* sectors_per_s, double* ms) {
    if (!ctx || !sectors_per_s || !ms) return fail(ctx, FB_ERR_ARG, "NULL argument");
    if (bytes < 1024 || bytes > (size_t(1) << 30) || (bytes & (bytes - 1)) != 0)
        return fail(ctx, FB_ERR_ARG, "bytes must be a power of two in [1 KiB, 1 GiB], got %zu", bytes);
    DeviceGuard dg(ctx->device);
    int sms = 0;
    FB_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const int blocks = sms * fb::kIterProbeBlocksPerSm, iters = 1 << 11;
    Carver measure(nullptr);
    measure.take<uint32_t>(bytes / 4);
    measure.take<uint32_t>(blocks);
    int rc = ensure_arena(ctx, measure.off);
    if (rc) return rc;
    Carver cv(ctx->arena);
    uint32_t* buf = cv.take<uint32_t>(bytes / 4);
    uint32_t* sink = cv.take<uint32_t>(blocks);
    cudaEvent_t a = nullptr, b = nullptr;
    FB_CUDA(ctx, cudaEventCreate(&a));
    FB_CUDA(ctx, cudaEventCreate(&b));
    FB_CUDA(ctx, cudaMemsetAsync(buf, 0x5A, bytes, nullptr));
    const uint32_t slots = static_cast<uint32_t>(bytes / 32);
    FB_CUDA(ctx, fb::launch_gather_probe(buf, slots, blocks, iters / 16, sink, nullptr));  // warm-up
    FB_CUDA(ctx, cudaEventRecord(a, nullptr));
    FB_CUDA(ctx, fb::launch_gather_probe(buf, slots, blocks, iters, sink, nullptr));
    FB_CUDA(ctx, cudaEventRecord(b, nullptr));
    FB_CUDA(ctx, cudaEventSynchronize(b));
    float t = 0.f;
    FB_CUDA(ctx, cudaEventElapsedTime(&t, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->launches += 2;
    *ms = t;
    *sectors_per_s = static_cast<double>(blocks) * 256.0 * iters * 4.0 / (t * 1e-3);
    return FB_OK;
}

uint32_t fb_pair_tag(int j, int i) {
    return (static_cast<uint32_t>(j) << 16) | static_cast<uint32_t>(i & 0xFFFF);
}

int fb_nnf(fb_ctx* ctx, const uint8_t* src_guide, const uint8_t* tgt_guide, int H, int W,
           const fb_params* p, const int32_t* init_nnf, int32_t* nnf_out, uint32_t* err_out,
           void* stream) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    ctx->err.clear();
    int rc = check_params(ctx, p, H, W);
    if (rc) return rc;
    if (!src_guide || !tgt_guide || !nnf_out)
        return fail(ctx, FB_ERR_ARG, "src_guide, tgt_guide and nnf_out must be non-NULL");
    if (init_nnf && p->levels != 1)
        return fail(ctx, FB_ERR_ARG, "an initial NNF requires levels == 1");
    if (p->flags & FB_FLAG_BALANCED)
        return fail(ctx, FB_ERR_ARG, "the improved loss needs the source style: use fb_nnf_balanced");
    if (p->flags & (FB_FLAG_FAST | FB_FLAG_ACCURATE))
        return fail(ctx, FB_ERR_ARG, "FB_FLAG_FAST and FB_FLAG_ACCURATE apply to fb_blend_window only");
    if (p->flags & (FB_FLAG_TRACKING | FB_FLAG_ALIGN))
        return fail(ctx, FB_ERR_ARG, "FB_FLAG_TRACKING and FB_FLAG_ALIGN apply to whole clips");
    DeviceGuard dg(ctx->device);
    for (const void* q : {static_cast<const void*>(src_guide), static_cast<const void*>(tgt_guide),
                          static_cast<const void*>(nnf_out), static_cast<const void*>(init_nnf),
                          static_cast<const void*>(err_out)})
        if (q && classify(ctx, q) != Mem::Device)
            return fail(ctx, FB_ERR_ARG, "fb_nnf takes device pointers of the context's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Levels L = level_dims(H, W, p->levels);
    const size_t npx0 = static_cast<size_t>(H) * W;

    Buffers b;
    Carver measure(nullptr);
    carve(measure, b, L, p->patch, 2, 0, 1, 1, 0, false, 0, 0, 0);
    rc = ensure_arena(ctx, measure.off);
    if (rc) return rc;
    Carver cv(ctx->arena);
    carve(cv, b, L, p->patch, 2, 0, 1, 1, 0, false, 0, 0, 0);

    std::vector<PairDesc> pairs(1);
    pairs[0] = PairDesc{0, 1, p->pair_tag, 0, 1u, {0, 0, 0}};
    rc = upload_tables(ctx, pairs, {}, b, st);
    if (rc) return rc;
    rc = prep_guides(ctx, b, L, p->patch, src_guide, 1, 0, st);
    if (rc) return rc;
    rc = prep_guides(ctx, b, L, p->patch, tgt_guide, 1, 1, st);
    if (rc) return rc;
    uint32_t *F = nullptr, *E = nullptr;
    rc = run_nnf(ctx, b, L, p, 0, 1, init_nnf, st, &F, &E);
    if (rc) return rc;
    FB_LAUNCH(ctx, st, FB_K_UNPACK, fb::launch_nnf_unpack(F, E, npx0, nnf_out, err_out, st));
    return FB_OK;
}

int fb_nnf_step(fb_ctx* ctx, const uint8_t* src_guide, const uint8_t* tgt_guide, int H, int W,
                const fb_params* p, int it, const int32_t* nnf_in, const uint32_t* err_in,
                int32_t* nnf_out, uint32_t* err_out, void* stream) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    ctx->err.clear();
    int rc = check_params(ctx, p, H, W);
    if (rc) return rc;
    if (p->levels != 1) return fail(ctx, FB_ERR_ARG, "fb_nnf_step works on one level: levels must be 1");
    if (p->flags != 0) return fail(ctx, FB_ERR_ARG, "fb_nnf_step takes the plain loss only: flags must be 0");
    if (it < 0 || it > 65534) return fail(ctx, FB_ERR_ARG, "it must be in [0, 65534], got %d", it);
    if (!src_guide || !tgt_guide || !nnf_in || !err_in || !nnf_out || !err_out)
        return fail(ctx, FB_ERR_ARG, "fb_nnf_step takes six non-NULL arrays");
    DeviceGuard dg(ctx->device);
    for (const void* q : {static_cast<const void*>(src_guide), static_cast<const void*>(tgt_guide),
                          static_cast<const void*>(nnf_in), static_cast<const void*>(err_in),
                          static_cast<const void*>(nnf_out), static_cast<const void*>(err_out)})
        if (classify(ctx, q) != Mem::Device)
            return fail(ctx, FB_ERR_ARG, "fb_nnf_step takes device pointers of the context's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Levels L = level_dims(H, W, 1);
    const size_t npx = static_cast<size_t>(H) * W;

    Buffers b;
    Carver measure(nullptr);
    carve(measure, b, L, p->patch, 2, 0, 1, 1, 0, false, 0, 0, 0);
    rc = ensure_arena(ctx, measure.off);
    if (rc) return rc;
    Carver cv(ctx->arena);
    carve(cv, b, L, p->patch, 2, 0, 1, 1, 0, false, 0, 0, 0);

    std::vector<PairDesc> pairs(1);
    pairs[0] = PairDesc{0, 1, p->pair_tag, 0, 1u, {0, 0, 0}};
    rc = upload_tables(ctx, pairs, {}, b, st);
    if (rc) return rc;
    rc = prep_guides(ctx, b, L, p->patch, src_guide, 1, 0, st);
    if (rc) return rc;
    rc = prep_guides(ctx, b, L, p->patch, tgt_guide, 1, 1, st);
    if (rc) return rc;
    FB_LAUNCH(ctx, st, FB_K_PACK, fb::launch_nnf_pack(nnf_in, H, W, b.FA, st));
    FB_CUDA(ctx, cudaMemcpyAsync(b.EA, err_in, npx * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    const LevelGeom g{H, W, b.rec[0]};
    const int r0 = p->r0 > 0 ? p->r0 : (H > W ? H : W);
    FB_LAUNCH(ctx, st, FB_K_ITER, fb::launch_nnf_iter(p->patch, b.pairs, 0, 1, g, r0, p->seed, 0, it, b.FA, b.EA,
                                                      b.FB, b.EB, st));
    FB_LAUNCH(ctx, st, FB_K_UNPACK, fb::launch_nnf_unpack(b.FB, b.EB, npx, nnf_out, err_out, st));
    return FB_OK;
}

int fb_nnf_segment(fb_ctx* ctx, const uint8_t* guides, const uint8_t* key_styles, int n, int H, int W,
                   const fb_params* p, const int32_t* init, int32_t* nnf_out, uint32_t* err_out,
                   void* stream) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    ctx->err.clear();
    int rc = check_params(ctx, p, H, W);
    if (rc) return rc;
    if (p->levels != 1) return fail(ctx, FB_ERR_ARG, "fb_nnf_segment requires levels == 1");
    if (p->flags & ~(FB_FLAG_ALIGN | FB_FLAG_TRACKING))
        return fail(ctx, FB_ERR_ARG, "fb_nnf_segment takes FB_FLAG_ALIGN and FB_FLAG_TRACKING only");
    if (n < 1 || n > 32767) return fail(ctx, FB_ERR_ARG, "n must be in [1, 32767], got %d", n);
    if (!guides || !key_styles || !nnf_out)
        return fail(ctx, FB_ERR_ARG, "guides, key_styles and nnf_out must be non-NULL");
    if (err_out && (p->flags & FB_FLAG_ALIGN) && p->iters == 0)
        return fail(ctx, FB_ERR_ARG, "with FB_FLAG_ALIGN the coupled loss is reported after iters >= 1");
    DeviceGuard dg(ctx->device);
    for (const void* q : {static_cast<const void*>(guides), static_cast<const void*>(key_styles),
                          static_cast<const void*>(init), static_cast<const void*>(nnf_out),
                          static_cast<const void*>(err_out)})
        if (q && classify(ctx, q) != Mem::Device)
            return fail(ctx, FB_ERR_ARG, "fb_nnf_segment takes device pointers of the context's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Levels L = level_dims(H, W, 1);
    const size_t npx0 = static_cast<size_t>(H) * W;
    const int k = p->patch;

    // Left key's chain first, then the right key's: pair q - 1 and n + q - 1 target frame q.
    std::vector<PairDesc> pairs;
    for (int side = 0; side < 2; ++side) {
        const int key = side == 0 ? 0 : n + 1;
        for (int q = 1; q <= n; ++q) pairs.push_back(PairDesc{key, q, fb_pair_tag(key, q), side, 1u, {-1, -1, -1}});
    }
    if (p->flags & FB_FLAG_TRACKING) set_chain_neighbours(pairs);
    if (p->flags & FB_FLAG_ALIGN)
        for (int q = 0; q < n; ++q) {
            pairs[q].pad[2] = n + q;
            pairs[n + q].pad[2] = q;
        }
    const size_t n_pairs = pairs.size();

    Buffers b;
    Carver measure(nullptr);
    carve(measure, b, L, k, n + 2, 2, n_pairs, n_pairs, 0, false, 0, 0, 0, false, false, true);
    rc = ensure_arena(ctx, measure.off);
    if (rc) return rc;
    Carver cv(ctx->arena);
    carve(cv, b, L, k, n + 2, 2, n_pairs, n_pairs, 0, false, 0, 0, 0, false, false, true);
    rc = upload_tables(ctx, pairs, {}, b, st);
    if (rc) return rc;
    rc = prep_guides(ctx, b, L, k, guides, n + 2, 0, st);
    if (rc) return rc;
    FB_LAUNCH(ctx, st, FB_K_PREP, fb::launch_prep_guides(k, key_styles, 2, H, W, b.srec, st));
    uint32_t *F = nullptr, *E = nullptr;
    rc = run_nnf(ctx, b, L, p, 0, static_cast<int>(n_pairs), init, st, &F, &E);
    if (rc) return rc;
    FB_LAUNCH(ctx, st, FB_K_UNPACK, fb::launch_nnf_unpack(F, E, n_pairs * npx0, nnf_out, err_out, st));
    return FB_OK;
}

int fb_nnf_balanced(fb_ctx* ctx, const uint8_t* src_guide, const uint8_t* tgt_guide,
                    const uint8_t* src_style, int H, int W, const fb_params* p,
                    const int32_t* init_nnf, int32_t* nnf_out, uint32_t* err_out, uint8_t* shat_out,
                    void* stream) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    ctx->err.clear();
    if (!p) return fail(ctx, FB_ERR_ARG, "params is NULL");
    fb_params q = *p;
    q.flags = FB_FLAG_BALANCED;
    int rc = check_params(ctx, &q, H, W);
    if (rc) return rc;
    if (!src_guide || !tgt_guide || !src_style || !nnf_out)
        return fail(ctx, FB_ERR_ARG, "src_guide, tgt_guide, src_style and nnf_out must be non-NULL");
    DeviceGuard dg(ctx->device);
    for (const void* v : {static_cast<const void*>(src_guide), static_cast<const void*>(tgt_guide),
                          static_cast<const void*>(src_style), static_cast<const void*>(nnf_out),
                          static_cast<const void*>(init_nnf), static_cast<const void*>(err_out),
                          static_cast<const void*>(shat_out)})
        if (v && classify(ctx, v) != Mem::Device)
            return fail(ctx, FB_ERR_ARG, "fb_nnf_balanced takes device pointers of the context's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Levels L = level_dims(H, W, 1);
    const size_t npx0 = static_cast<size_t>(H) * W;

    Buffers b;
    Carver measure(nullptr);
    carve(measure, b, L, q.patch, 2, 1, 1, 1, 0, false, 0, 0, 0, false, true);
    rc = ensure_arena(ctx, measure.off);
    if (rc) return rc;
    Carver cv(ctx->arena);
    carve(cv, b, L, q.patch, 2, 1, 1, 1, 0, false, 0, 0, 0, false, true);

    std::vector<PairDesc> pairs(1);
    pairs[0] = PairDesc{0, 1, q.pair_tag, 0, 1u, {0, 0, 0}};
    rc = upload_tables(ctx, pairs, {}, b, st);
    if (rc) return rc;
    rc = prep_guides(ctx, b, L, q.patch, src_guide, 1, 0, st);
    if (rc) return rc;
    rc = prep_guides(ctx, b, L, q.patch, tgt_guide, 1, 1, st);
    if (rc) return rc;
    FB_LAUNCH(ctx, st, FB_K_STYLE, fb::launch_style_rgbx(src_style, npx0, b.styles, st));
    FB_LAUNCH(ctx, st, FB_K_PREP, fb::launch_prep_guides(q.patch, src_style, 1, H, W, b.srec, st));
    uint32_t *F = nullptr, *E = nullptr;
    rc = run_nnf_balanced(ctx, b, H, W, &q, 0, 1, init_nnf, st, &F, &E);
    if (rc) return rc;
    FB_LAUNCH(ctx, st, FB_K_UNPACK, fb::launch_nnf_unpack(F, E, npx0, nnf_out, err_out, st));
    if (shat_out)
        FB_CUDA(ctx, cudaMemcpyAsync(shat_out, b.shat_img, npx0 * 3, cudaMemcpyDeviceToDevice, st));
    return FB_OK;
}

int fb_remap(fb_ctx* ctx, const uint8_t* src_style, const int32_t* nnf, int H, int W, int patch,
             float* out, void* stream) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    ctx->err.clear();
    if (patch < 3 || patch > 9 || (patch & 1) == 0)
        return fail(ctx, FB_ERR_ARG, "patch must be odd in [3, 9], got %d", patch);
    if (H < patch || W < patch || H > 32767 || W > 32767)
        return fail(ctx, FB_ERR_ARG, "image %dx%d outside [patch, 32767]", H, W);
    if (!src_style || !nnf || !out)
        return fail(ctx, FB_ERR_ARG, "src_style, nnf and out must be non-NULL");
    DeviceGuard dg(ctx->device);
    for (const void* q : {static_cast<const void*>(src_style), static_cast<const void*>(nnf),
                          static_cast<const void*>(out)})
        if (classify(ctx, q) != Mem::Device)
            return fail(ctx, FB_ERR_ARG, "fb_remap takes device pointers of the context's device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Levels L = level_dims(H, W, 1);
    const size_t npx = static_cast<size_t>(H) * W;

    Buffers b;
    Carver measure(nullptr);
    carve(measure, b, L, patch, 0, 1, 1, 1, 1, false, 0, 0, 0);
    int rc = ensure_arena(ctx, measure.off);
    if (rc) return rc;
    Carver cv(ctx->arena);
    carve(cv, b, L, patch, 0, 1, 1, 1, 1, false, 0, 0, 0);

    std::vector<PairDesc> pairs(1);
    pairs[0] = PairDesc{0, 0, 0u, 0, 1u, {0, 0, 0}};
    std::vector<JobDesc> jobs(1);
    jobs[0] = JobDesc{0, -1, 0u, 0, 1, static_cast<uint32_t>(255 * patch * patch), {0, 0}};
    rc = upload_tables(ctx, pairs, jobs, b, st);
    if (rc) return rc;
    FB_LAUNCH(ctx, st, FB_K_STYLE, fb::launch_style_rgbx(src_style, npx, b.styles, st));
    FB_LAUNCH(ctx, st, FB_K_PACK, fb::launch_nnf_pack(nnf, H, W, b.FA, st));
    FB_LAUNCH(ctx, st, FB_K_COMBINE, fb::launch_combine(patch, b.jobs, 0, 1, b.pairs, 0, b.FA, b.styles, H, W, out, st));
    return FB_OK;
}

int fb_blend_window(fb_ctx* ctx, const uint8_t* guides, const uint8_t* styles, int N, int H, int W,
                    int window, const fb_params* p, float* out, void* stream) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    ctx->err.clear();
    int rc = check_params(ctx, p, H, W);
    if (rc) return rc;
    if (N < 1 || N > 65535) return fail(ctx, FB_ERR_ARG, "N must be in [1, 65535], got %d", N);
    if (window < 1 || (window & 1) == 0)
        return fail(ctx, FB_ERR_ARG, "window must be odd and >= 1, got %d", window);
    if (!guides || !styles || !out)
        return fail(ctx, FB_ERR_ARG, "guides, styles and out must be non-NULL");
    if (p->flags & FB_FLAG_ALIGN) return fail(ctx, FB_ERR_ARG, "FB_FLAG_ALIGN applies to fb_interpolate only");
    const int k = p->patch;
    if (p->flags & FB_FLAG_FAST) {
        const uint64_t k4 = static_cast<uint64_t>(k) * k * k * k;
        if (k4 * 255u * static_cast<uint64_t>(window) >= (1ull << 32))
            return fail(ctx, FB_ERR_ARG, "fast mode: window %d with patch %d overflows the exact sums", window, k);
        FastPlan plan;
        plan_fast(N, window, plan);
        DeviceGuard dg(ctx->device);
        return run_fast_pipeline(ctx, guides, styles, N, H, W, plan, p, out, static_cast<cudaStream_t>(stream));
    }

    std::vector<PairDesc> pairs;
    std::vector<JobDesc> jobs;
    blend_pairs(N, k, window, p->flags, pairs, jobs);
    DeviceGuard dg(ctx->device);
    return run_pipeline(ctx, guides, N, H, W, styles, N, pairs, jobs, p, out,
                        static_cast<cudaStream_t>(stream));
}

int fb_interpolate(fb_ctx* ctx, const uint8_t* guides, int N, int H, int W, const int32_t* key_idx,
                   const uint8_t* key_styles, int n_keys, const fb_params* p, float* out,
                   void* stream) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    ctx->err.clear();
    int rc = check_params(ctx, p, H, W);
    if (rc) return rc;
    if (p->flags & (FB_FLAG_BALANCED | FB_FLAG_FAST | FB_FLAG_ACCURATE))
        return fail(ctx, FB_ERR_ARG, "the blending modes apply to fb_blend_window only");
    if (N < 1 || N > 65535) return fail(ctx, FB_ERR_ARG, "N must be in [1, 65535], got %d", N);
    if (!guides || !key_idx || !key_styles || !out)
        return fail(ctx, FB_ERR_ARG, "guides, key_idx, key_styles and out must be non-NULL");
    if (n_keys < 1 || n_keys > N)
        return fail(ctx, FB_ERR_ARG, "n_keys must be in [1, N], got %d", n_keys);
    for (int m = 0; m < n_keys; ++m) {
        if (key_idx[m] < 0 || key_idx[m] >= N)
            return fail(ctx, FB_ERR_ARG, "key_idx[%d] = %d outside [0, %d)", m, key_idx[m], N);
        if (m > 0 && key_idx[m] <= key_idx[m - 1])
            return fail(ctx, FB_ERR_ARG, "key_idx must be strictly increasing");
    }
    std::vector<PairDesc> pairs;
    std::vector<JobDesc> jobs;
    interp_pairs(N, p->patch, key_idx, n_keys, p->flags, pairs, jobs);
    DeviceGuard dg(ctx->device);
    return run_pipeline(ctx, guides, N, H, W, key_styles, n_keys, pairs, jobs, p, out,
                        static_cast<cudaStream_t>(stream));
}

// Modes whose pairs couple output frames across the whole clip cannot be cut into
// output-frame ranges: the fast mode's tables span the clip (Algs. 3-5) and tracking's
// chains run through the targets of one source (Sec. 3.5.1).
static int check_range_flags(fb_ctx* ctx, const fb_params* p) {
    if (p->flags & (FB_FLAG_FAST | FB_FLAG_TRACKING))
        return fail(ctx, FB_ERR_UNSUPPORTED,
                    "FB_FLAG_FAST and FB_FLAG_TRACKING couple output frames across the clip; "
                    "a range call cannot reproduce them");
    return FB_OK;
}

int fb_blend_window_range(fb_ctx* ctx, const uint8_t* guides, const uint8_t* styles, int n_in, int H, int W,
                          int window, const fb_params* p, int n_total, int frame_base, int out_first, int n_out,
                          float* out, void* stream) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    ctx->err.clear();
    int rc = check_params(ctx, p, H, W);
    if (rc) return rc;
    if (n_total < 1 || n_total > 65535) return fail(ctx, FB_ERR_ARG, "n_total must be in [1, 65535], got %d", n_total);
    if (window < 1 || (window & 1) == 0)
        return fail(ctx, FB_ERR_ARG, "window must be odd and >= 1, got %d", window);
    if (!guides || !styles || !out)
        return fail(ctx, FB_ERR_ARG, "guides, styles and out must be non-NULL");
    if (p->flags & FB_FLAG_ALIGN) return fail(ctx, FB_ERR_ARG, "FB_FLAG_ALIGN applies to fb_interpolate only");
    if (frame_base < 0 || n_in < 1 || frame_base + n_in > n_total)
        return fail(ctx, FB_ERR_ARG, "input frames [%d, %d) are not inside the clip [0, %d)", frame_base,
                    frame_base + n_in, n_total);
    if (n_out < 1 || out_first < 0 || out_first + n_out > n_total)
        return fail(ctx, FB_ERR_ARG, "output frames [%d, %d) are not inside the clip [0, %d)", out_first,
                    out_first + n_out, n_total);
    const int M = (window - 1) / 2;
    const int need_lo = out_first - M < 0 ? 0 : out_first - M;
    const int need_hi = out_first + n_out + M > n_total ? n_total : out_first + n_out + M;
    if (need_lo < frame_base || need_hi > frame_base + n_in)
        return fail(ctx, FB_ERR_ARG,
                    "output frames [%d, %d) with window %d need input frames [%d, %d); the call holds [%d, %d)",
                    out_first, out_first + n_out, window, need_lo, need_hi, frame_base, frame_base + n_in);
    rc = check_range_flags(ctx, p);
    if (rc) return rc;
    std::vector<PairDesc> pairs;
    std::vector<JobDesc> jobs;
    blend_pairs(n_total, p->patch, window, p->flags, pairs, jobs, out_first, out_first + n_out, frame_base);
    DeviceGuard dg(ctx->device);
    return run_pipeline(ctx, guides, n_in, H, W, styles, n_in, pairs, jobs, p, out,
                        static_cast<cudaStream_t>(stream));
}

int fb_interpolate_range(fb_ctx* ctx, const uint8_t* guides, int N, int H, int W, const int32_t* key_idx,
                         const uint8_t* key_styles, int n_keys, const fb_params* p, int out_first, int n_out,
                         float* out, void* stream) {
    if (!ctx) return fail(nullptr, FB_ERR_ARG, "ctx is NULL");
    ctx->err.clear();
    int rc = check_params(ctx, p, H, W);
    if (rc) return rc;
    if (p->flags & (FB_FLAG_BALANCED | FB_FLAG_FAST | FB_FLAG_ACCURATE))
        return fail(ctx, FB_ERR_ARG, "the blending modes apply to fb_blend_window only");
    if (N < 1 || N > 65535) return fail(ctx, FB_ERR_ARG, "N must be in [1, 65535], got %d", N);
    if (!guides || !key_idx || !key_styles || !out)
        return fail(ctx, FB_ERR_ARG, "guides, key_idx, key_styles and out must be non-NULL");
    if (n_keys < 1 || n_keys > N)
        return fail(ctx, FB_ERR_ARG, "n_keys must be in [1, N], got %d", n_keys);
    for (int m = 0; m < n_keys; ++m) {
        if (key_idx[m] < 0 || key_idx[m] >= N)
            return fail(ctx, FB_ERR_ARG, "key_idx[%d] = %d outside [0, %d)", m, key_idx[m], N);
        if (m > 0 && key_idx[m] <= key_idx[m - 1])
            return fail(ctx, FB_ERR_ARG, "key_idx must be strictly increasing");
    }
    if (n_out < 1 || out_first < 0 || out_first + n_out > N)
        return fail(ctx, FB_ERR_ARG, "output frames [%d, %d) are not inside the clip [0, %d)", out_first,
                    out_first + n_out, N);
    rc = check_range_flags(ctx, p);
    if (rc) return rc;
    std::vector<PairDesc> pairs;
    std::vector<JobDesc> jobs;
    interp_pairs(N, p->patch, key_idx, n_keys, p->flags, pairs, jobs, out_first, out_first + n_out);
    DeviceGuard dg(ctx->device);
    return run_pipeline(ctx, guides, N, H, W, key_styles, n_keys, pairs, jobs, p, out,
                        static_cast<cudaStream_t>(stream));
}

}  // extern "C"
