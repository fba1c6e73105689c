// fb_noalloc.cu -- fb_blend_window_noalloc: fb_blend_window without a context or any
// device allocation, for callers that cannot allocate device memory themselves.
//
// Some callers may not call cudaMalloc (or any allocator) at the point where they
// blend: code running inside a host callback or a stream-ordered pipeline that must
// not synchronise the device, plug-ins whose host application owns every allocation,
// or processes that run under a fixed device-memory budget fixed at start-up.  For
// them this entry point takes no context and allocates nothing: its scratch is the
// file-scope device array below, of a fixed size, which every GPU that loads this
// library holds until the process exits.  The caller still passes its own inputs and
// outputs.
#include <cstdio>

#include "fb.h"
#include "fb_internal.h"

namespace fb {
void set_null_ctx_error(const char* msg);
}

namespace {

using fb::JobDesc;
using fb::LevelGeom;
using fb::PairDesc;

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // FB_NOALLOC_SCRATCH_BYTES
static_assert(kStaticScratchBytes == FB_NOALLOC_SCRATCH_BYTES, "header and file disagree");

// The scratch.  In host code this name is only a host-side stand-in for the device
// array; its device address comes from cudaGetSymbolAddress (scratch_address below).
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

int report(int status, const char* fmt, long long a = 0, long long b = 0) {
    char buf[256];
    std::snprintf(buf, sizeof buf, fmt, a, b);
    fb::set_null_ctx_error(buf);
    return status;
}

// The device address of the static scratch array on the current device, looked up on
// every call: a host-side lookup once the library's device code is loaded on the device
// (the first call on a device loads it), and never stale, even after the device's
// primary context was reset and the array moved.
int scratch_address(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return report(FB_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed (%lld)",
                      static_cast<long long>(e));
    }
    *out = static_cast<unsigned char*>(p);
    return FB_OK;
}

// Pair and job tables of the window blend, built on the device (no host staging buffer): output
// frame i owns the pairs (j -> i), j in [max(0, i-M), min(N-1, i+M)], j != i, in
// increasing j, after the pairs of frames 0 .. i-1.
__global__ void blend_tables_kernel(int N, int M, int k, PairDesc* __restrict__ pairs,
                                    JobDesc* __restrict__ jobs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int first = 0;
    for (int q = 0; q < i; ++q) first += min(N - 1, q + M) - max(0, q - M);
    const int lo = max(0, i - M), hi = min(N - 1, i + M);
    JobDesc jd;
    jd.out_frame = i;
    jd.self_style = i;
    jd.self_w = 1u;
    jd.first_pair = first;
    jd.n_pairs = hi - lo;
    jd.den = static_cast<uint32_t>(255 * k * k * (hi - lo + 1));
    jd.pad[0] = jd.pad[1] = 0;
    jobs[i] = jd;
    int n = first;
    for (int j = lo; j <= hi; ++j) {
        if (j == i) continue;
        PairDesc pd;
        pd.src = j;
        pd.tgt = i;
        pd.tag = (static_cast<uint32_t>(j) << 16) | static_cast<uint32_t>(i);
        pd.style = j;
        pd.weight = 1u;
        pd.pad[0] = pd.pad[1] = pd.pad[2] = -1;  // no chain neighbours, no partner
        pairs[n++] = pd;
    }
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

bool on_device(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}

}  // namespace

extern "C" int fb_blend_window_noalloc(const uint8_t* guides, const uint8_t* styles, int N, int H,
                                       int W, int window, const fb_params* p, float* out,
                                       void* stream) {
    fb::set_null_ctx_error("");  // a success leaves no message behind
    if (!p) return report(FB_ERR_ARG, "params is NULL");
    if (p->patch < 3 || p->patch > 9 || (p->patch & 1) == 0)
        return report(FB_ERR_ARG, "patch must be odd in [3, 9], got %lld", p->patch);
    if (p->iters < 0 || p->iters > 65534)
        return report(FB_ERR_ARG, "iters must be in [0, 65534], got %lld", p->iters);
    if (p->levels < 1 || p->levels > 16)
        return report(FB_ERR_ARG, "levels must be in [1, 16], got %lld", p->levels);
    if (p->r0 < 0 || p->r0 > (1 << 20)) return report(FB_ERR_ARG, "r0 must be in [0, 2^20], got %lld", p->r0);
    if (p->flags != 0) return report(FB_ERR_ARG, "flags must be 0 for the no-allocation blend");
    if (H < p->patch || W < p->patch || H > 32767 || W > 32767)
        return report(FB_ERR_ARG, "image %lldx%lld outside [patch, 32767]", H, W);
    if (N < 1 || N > 65535) return report(FB_ERR_ARG, "N must be in [1, 65535], got %lld", N);
    if (window < 1 || (window & 1) == 0)
        return report(FB_ERR_ARG, "window must be odd and >= 1, got %lld", window);
    if (!guides || !styles || !out) return report(FB_ERR_ARG, "guides, styles and out must be non-NULL");

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return report(FB_ERR_CUDA, "no current CUDA device");
    }
    if (!on_device(guides, device) || !on_device(styles, device) || !on_device(out, device))
        return report(FB_ERR_ARG, "guides, styles and out must be device memory of the current device");

    const int k = p->patch, M = (window - 1) / 2;
    int hs[16], ws[16];
    hs[0] = H;
    ws[0] = W;
    for (int l = 1; l < p->levels; ++l) {
        hs[l] = (hs[l - 1] + 1) / 2;
        ws[l] = (ws[l - 1] + 1) / 2;
    }
    long long n_pairs = 0;
    for (int i = 0; i < N; ++i) n_pairs += (i + M > N - 1 ? N - 1 : i + M) - (i - M < 0 ? 0 : i - M);
    if (n_pairs > 65535) return report(FB_ERR_ARG, "%lld NNFs exceed the 65535 of one launch", n_pairs);
    const size_t npx0 = static_cast<size_t>(H) * W;

    // Layout of the static scratch (256-byte aligned pieces).
    size_t off = 0, o_raw[16] = {}, o_rec[16];
    for (int l = 0; l < p->levels; ++l) {
        const size_t npx = static_cast<size_t>(hs[l]) * ws[l];
        if (l > 0) { o_raw[l] = off; off = align256(off + static_cast<size_t>(N) * npx * 3); }
        o_rec[l] = off; off = align256(off + static_cast<size_t>(N) * fb::rowpatch_frame_words(k, hs[l], ws[l]) * 4);
    }
    const size_t o_sty = off; off = align256(off + static_cast<size_t>(N) * npx0 * 4);
    size_t o_fe[4];
    for (int q = 0; q < 4; ++q) { o_fe[q] = off; off = align256(off + static_cast<size_t>(n_pairs) * npx0 * 4); }
    const size_t o_pairs = off; off = align256(off + static_cast<size_t>(n_pairs > 0 ? n_pairs : 1) * sizeof(PairDesc));
    const size_t o_jobs = off; off = align256(off + static_cast<size_t>(N) * sizeof(JobDesc));
    if (off > kStaticScratchBytes)
        return report(FB_ERR_ARG, "this blend needs %lld bytes of scratch; the static scratch holds %lld",
                      static_cast<long long>(off), static_cast<long long>(kStaticScratchBytes));

    unsigned char* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto u32 = [&](size_t o) { return reinterpret_cast<uint32_t*>(base + o); };
    PairDesc* pairs = reinterpret_cast<PairDesc*>(base + o_pairs);
    JobDesc* jobs = reinterpret_cast<JobDesc*>(base + o_jobs);

#define NA_CHECK(expr)                                                                   \
    do {                                                                                 \
        const cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess)                                                           \
            return report(FB_ERR_CUDA, #expr " failed (%lld)", static_cast<long long>(e_)); \
    } while (0)

    blend_tables_kernel<<<(N + 127) / 128, 128, 0, st>>>(N, M, k, pairs, jobs);
    NA_CHECK(cudaGetLastError());
    const uint8_t* cur = guides;
    for (int l = 0; l < p->levels; ++l) {
        if (l > 0) {
            uint8_t* dst = base + o_raw[l];
            NA_CHECK(fb::launch_downsample(cur, N, hs[l - 1], ws[l - 1], dst, st));
            cur = dst;
        }
        NA_CHECK(fb::launch_prep_guides(k, cur, N, hs[l], ws[l], u32(o_rec[l]), st));
    }
    NA_CHECK(fb::launch_style_rgbx(styles, static_cast<size_t>(N) * npx0, u32(o_sty), st));

    uint32_t* F = nullptr;
    if (n_pairs > 0) {
        const int np = static_cast<int>(n_pairs);
        uint32_t *Fc = u32(o_fe[0]), *Ec = u32(o_fe[1]), *Fo = u32(o_fe[2]), *Eo = u32(o_fe[3]);
        for (int l = p->levels - 1; l >= 0; --l) {
            LevelGeom g{hs[l], ws[l], u32(o_rec[l])};
            if (l == p->levels - 1) {
                NA_CHECK(fb::launch_nnf_init(k, pairs, 0, np, g, 0, nullptr, 0, 0, nullptr, p->seed, l,
                                             Fc, Ec, st));
            } else {
                NA_CHECK(fb::launch_nnf_init(k, pairs, 0, np, g, 1, Fc, hs[l + 1], ws[l + 1], nullptr,
                                             p->seed, l, Fo, Eo, st));
                std::swap(Fc, Fo);
                std::swap(Ec, Eo);
            }
            const int r0 = p->r0 > 0 ? p->r0 : (hs[l] > ws[l] ? hs[l] : ws[l]);
            for (int it = 0; it < p->iters; ++it) {
                NA_CHECK(fb::launch_nnf_iter(k, pairs, 0, np, g, r0, p->seed, l, it, Fc, Ec, Fo, Eo, st));
                std::swap(Fc, Fo);
                std::swap(Ec, Eo);
            }
        }
        F = Fc;
    }
    NA_CHECK(fb::launch_combine(k, jobs, 0, N, pairs, 0, F, u32(o_sty), H, W, out, st));
#undef NA_CHECK
    return FB_OK;
}
