// fb_batch.cu -- persistent kernels of the batched submission (fb_blend_batch): many
// clips of uneven size, window and patch in one pass.  Every pair of every clip is cut
// into 32-column tiles, and runs of consecutive tiles of one pair form the work units;
// a kernel of SMs x resident-blocks CTAs claims units of the flattened work list
// (unit -> pair, first tile) from a counter, so clips of different shapes share one
// launch per Jacobi iteration.  The per-pixel work is the same code as the per-call kernels
// (fb_device.cuh), so results are identical to fb_blend_window whatever tile shape the
// autotuner picks.
#include <type_traits>

#include "fb_device.cuh"

namespace fb {
namespace {

using namespace dev;

// Variant v: tile height and the resident 32 x TH-thread blocks per SM the iteration
// kernel is compiled for (the same ~1280 threads per SM for k = 5).
template <int V>
struct Variant;
template <> struct Variant<0> { static constexpr int TH = 8, MINB = 5; };   // 32x8,  5 blocks
template <> struct Variant<1> { static constexpr int TH = 4, MINB = 10; };  // 32x4, 10 blocks
template <> struct Variant<2> { static constexpr int TH = 16, MINB = 2; };  // 32x16, 2 blocks
template <> struct Variant<3> { static constexpr int TH = 8, MINB = 4; };   // 32x8,  4 blocks

// Work distribution: every CTA claims the next unprocessed item from a counter that is
// zeroed before the launch, so items (pair-major) are processed close to their global
// order and only about one resident wave of pairs shares the L2 at a time (a static
// round-robin lets fast and slow CTAs drift apart and spreads the working set).  The
// claim for the following item is issued before the current one is processed, so its
// latency is hidden behind the work.
struct ItemQueue {
    int* counter;
    int* slot;    // shared: [2]
    int buf = 0;
    int pending = 0;
    __device__ __forceinline__ bool lead() const { return threadIdx.x == 0 && threadIdx.y == 0; }
    __device__ __forceinline__ int first() {
        if (lead()) slot[0] = atomicAdd(counter, 1);
        __syncthreads();
        return slot[0];
    }
    __device__ __forceinline__ void prefetch() {
        if (lead()) pending = atomicAdd(counter, 1);
    }
    __device__ __forceinline__ int next() {
        if (lead()) slot[buf ^ 1] = pending;
        __syncthreads();  // the claim is visible and every thread is done with the item
        buf ^= 1;
        return slot[buf];
    }
};

// Block-uniform descriptor loads the compiler may not hoist out of a tile loop: every
// thread re-reads them per tile (L1 broadcast hits), so they need not stay live in
// registers across the pixel work, which would spill at 5 blocks per SM.
__device__ __forceinline__ int4 ld_uniform(const void* p) {
    int4 v;
    asm volatile("ld.global.nc.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ const uint32_t* as_ptr(int lo, int hi) {
    return reinterpret_cast<const uint32_t*>((static_cast<uint64_t>(static_cast<uint32_t>(hi)) << 32) |
                                             static_cast<uint32_t>(lo));
}

// Larger patches keep more target words in registers: fewer resident warps (k = 7: 28
// warps per SM, as the per-call kernel, in as many whole blocks as fit).
template <int K, int V>
struct BatchOcc {
    static constexpr int base = Variant<V>::MINB;
    static constexpr int k7 = 28 / Variant<V>::TH > 0 ? 28 / Variant<V>::TH : 1;
    static constexpr int value = K <= 5 ? base : K <= 7 ? k7 : (base * 2 + 4) / 5;
};

template <int K, int V>
__global__ void __launch_bounds__(32 * Variant<V>::TH, BatchOcc<K, V>::value)
    batch_iter_kernel(const BatchPair* __restrict__ pairs, const BatchClip* __restrict__ clips,
                      const int32_t* __restrict__ item_pair, const int32_t* __restrict__ item_tile,
                      int n_items, int per_claim, int* __restrict__ counter, uint32_t key0,
                      uint32_t key1, uint32_t ctr_word, const uint32_t* __restrict__ Fp,
                      const uint32_t* __restrict__ Ep, uint32_t* __restrict__ Fn,
                      uint32_t* __restrict__ En) {
    using G = Geo<K>;
    constexpr int TH = Variant<V>::TH;
    __shared__ int s_slot[2];
    ItemQueue q{counter, s_slot};
    for (int item = q.first(); item < n_items; item = q.next()) {
        q.prefetch();
        const int ip = item_pair[item];
        const int t0 = item_tile[item];
        int t1;
        {
            const int4 cg = ld_uniform(clips + ld_uniform(pairs + ip).x);  // H, W, N, r0
            t1 = min(t0 + per_claim, ((cg.y + 31) / 32) * ((cg.x + TH - 1) / TH));
        }
        // No barrier inside the unit: each thread runs through its pixels of the unit's
        // tiles and rejoins the block at q.next().
        for (int tile = t0; tile < t1; ++tile) {
            const int4 p0 = ld_uniform(pairs + ip);              // clip, src, tgt, style
            const int4 p1 = ld_uniform(&pairs[ip].tag);          // tag, weight, fe_off
            const int4 cg = ld_uniform(clips + p0.x);            // H, W, N, r0
            const int4 cp = ld_uniform(&clips[p0.x].rp);         // rp, styles
            const int H = cg.x, W = cg.y, tiles_x = (W + 31) / 32;
            const int r = (tile / tiles_x) * TH + static_cast<int>(threadIdx.y);
            const int c = (tile % tiles_x) * 32 + static_cast<int>(threadIdx.x);
            if (r >= H || c >= W) continue;
            const uint32_t* rp = as_ptr(cp.x, cp.y);
            const uint64_t fe = (static_cast<uint64_t>(static_cast<uint32_t>(p1.w)) << 32) |
                                static_cast<uint32_t>(p1.z);
            iterate_pixel<K>(frame_rows<K>(rp, p0.y, H, W), frame_rows<K>(rp, p0.z, H, W), H, W, r, c,
                             static_cast<uint32_t>(p1.x), cg.w, key0, key1, ctr_word, Fp + fe,
                             Ep + fe, Fn + fe, En + fe);
        }
    }
}

template <int K, int V>
__global__ void __launch_bounds__(32 * Variant<V>::TH)
    batch_init_kernel(const BatchPair* __restrict__ pairs, const BatchClip* __restrict__ clips,
                      const int32_t* __restrict__ item_pair, const int32_t* __restrict__ item_tile,
                      int n_items, int* __restrict__ counter, uint32_t key0, uint32_t key1,
                      uint32_t* __restrict__ F, uint32_t* __restrict__ E) {
    using G = Geo<K>;
    constexpr int TH = Variant<V>::TH;
    __shared__ int s_slot[2];
    ItemQueue q{counter, s_slot};
    for (int item = q.first(); item < n_items; item = q.next()) {
        q.prefetch();
        const BatchPair bp = pairs[item_pair[item]];
        const BatchClip cl = clips[bp.clip];
        const int tiles_x = (cl.W + 31) / 32;
        const int t0 = item_tile[item];
        const int t1 = min(t0 + kInitTilesPerClaim, tiles_x * ((cl.H + TH - 1) / TH));
        for (int tile = t0; tile < t1; ++tile) {
            const int r = (tile / tiles_x) * TH + static_cast<int>(threadIdx.y);
            const int c = (tile % tiles_x) * 32 + static_cast<int>(threadIdx.x);
            if (r >= cl.H || c >= cl.W) continue;
            init_pixel<K>(frame_rows<K>(cl.rp, bp.src, cl.H, cl.W),
                          frame_rows<K>(cl.rp, bp.tgt, cl.H, cl.W), cl.H, cl.W, r, c,
                          bp.tag, 0, nullptr, 0, 0, nullptr, key0, key1, 0u, F + bp.fe_off,
                          E + bp.fe_off);
        }
    }
}

// Alg. 2 + Eq. 2 for the output frames of a chunk: units are (job, kCombineTilesPerClaim
// consecutive 32x8 tiles).
template <int K>
__global__ void __launch_bounds__(256)
    batch_combine_kernel(const BatchJob* __restrict__ jobs, const BatchPair* __restrict__ pairs,
                         const BatchClip* __restrict__ clips, const int32_t* __restrict__ item_job,
                         const int32_t* __restrict__ item_tile, int n_items,
                         int* __restrict__ counter, const uint32_t* __restrict__ F) {
    __shared__ int s_slot[2];
    ItemQueue q{counter, s_slot};
    for (int item = q.first(); item < n_items; item = q.next()) {
        q.prefetch();
        const int ij = item_job[item];
        const int t0 = item_tile[item];
        int t1;
        {
            const int4 cg = ld_uniform(clips + ld_uniform(jobs + ij).x);  // H, W, N, r0
            t1 = min(t0 + kCombineTilesPerClaim, ((cg.y + 31) / 32) * ((cg.x + 7) / 8));
        }
        for (int tile = t0; tile < t1; ++tile) {
            const int4 j0 = ld_uniform(jobs + ij);        // clip, frame, first_pair, n_pairs
            const int4 cg = ld_uniform(clips + j0.x);     // H, W, N, r0
            const int H = cg.x, W = cg.y, tiles_x = (W + 31) / 32;
            const int r = (tile / tiles_x) * 8 + static_cast<int>(threadIdx.y);
            const int c = (tile % tiles_x) * 32 + static_cast<int>(threadIdx.x);
            if (r >= H || c >= W) continue;
            const int4 cp = ld_uniform(&clips[j0.x].rp);  // rp, styles
            const uint32_t* styles = as_ptr(cp.z, cp.w);
            const size_t npx = static_cast<size_t>(H) * W;
            const size_t x = static_cast<size_t>(r) * W + c;
            const uint32_t s = __ldg(styles + static_cast<size_t>(j0.y) * npx + x);
            const uint32_t w = static_cast<uint32_t>(K * K);
            uint32_t a0 = w * (s & 0xFFu), a1 = w * ((s >> 8) & 0xFFu), a2 = w * ((s >> 16) & 0xFFu);
            for (int p = 0; p < j0.w; ++p) {
                const BatchPair bp = pairs[j0.z + p];
                uint32_t v0, v1, v2;
                remap_votes<K>(F + bp.fe_off, styles + static_cast<size_t>(bp.style) * npx, H, W, r,
                               c, v0, v1, v2);
                a0 += bp.weight * v0;
                a1 += bp.weight * v1;
                a2 += bp.weight * v2;
            }
            const BatchJob job = jobs[ij];
            const BatchClip* cl = clips + job.clip;
            write_output(cl->out + (static_cast<size_t>(job.frame) * npx + x) * 3, a0, a1, a2,
                         job.den);
        }
    }
}

template <int K, int V>
cudaError_t launch_iter_kv(const BatchPair* pairs, const BatchClip* clips, const int32_t* ip,
                           const int32_t* it_, int n, int per_claim, int* counter, uint32_t k0,
                           uint32_t k1, uint32_t cw, const uint32_t* Fp, const uint32_t* Ep,
                           uint32_t* Fn, uint32_t* En, int grid, cudaStream_t st) {
    batch_iter_kernel<K, V><<<grid, dim3(32, Variant<V>::TH), 0, st>>>(pairs, clips, ip, it_, n, per_claim,
                                                                       counter, k0, k1, cw, Fp, Ep, Fn, En);
    return cudaGetLastError();
}

template <int K, int V>
cudaError_t launch_init_kv(const BatchPair* pairs, const BatchClip* clips, const int32_t* ip,
                           const int32_t* it_, int n, int* counter, uint32_t k0, uint32_t k1,
                           uint32_t* F, uint32_t* E, int grid, cudaStream_t st) {
    batch_init_kernel<K, V><<<grid, dim3(32, Variant<V>::TH), 0, st>>>(pairs, clips, ip, it_, n, counter,
                                                                       k0, k1, F, E);
    return cudaGetLastError();
}

template <int K>
int occupancy_k(int v) {
    int nb = 0;
    switch (v) {
        case 0: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_iter_kernel<K, 0>, 32 * Variant<0>::TH, 0); break;
        case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_iter_kernel<K, 1>, 32 * Variant<1>::TH, 0); break;
        case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_iter_kernel<K, 2>, 32 * Variant<2>::TH, 0); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_iter_kernel<K, 3>, 32 * Variant<3>::TH, 0); break;
    }
    cudaGetLastError();
    return nb > 0 ? nb : 1;
}

#define FB_BATCH_DISPATCH(k, v, CALL)                                                     \
    switch ((k) * 10 + (v)) {                                                              \
        case 30: { constexpr int KK = 3, VV = 0; return CALL; }                            \
        case 31: { constexpr int KK = 3, VV = 1; return CALL; }                            \
        case 32: { constexpr int KK = 3, VV = 2; return CALL; }                            \
        case 33: { constexpr int KK = 3, VV = 3; return CALL; }                            \
        case 50: { constexpr int KK = 5, VV = 0; return CALL; }                            \
        case 51: { constexpr int KK = 5, VV = 1; return CALL; }                            \
        case 52: { constexpr int KK = 5, VV = 2; return CALL; }                            \
        case 53: { constexpr int KK = 5, VV = 3; return CALL; }                            \
        case 70: { constexpr int KK = 7, VV = 0; return CALL; }                            \
        case 71: { constexpr int KK = 7, VV = 1; return CALL; }                            \
        case 72: { constexpr int KK = 7, VV = 2; return CALL; }                            \
        case 73: { constexpr int KK = 7, VV = 3; return CALL; }                            \
        case 90: { constexpr int KK = 9, VV = 0; return CALL; }                            \
        case 91: { constexpr int KK = 9, VV = 1; return CALL; }                            \
        case 92: { constexpr int KK = 9, VV = 2; return CALL; }                            \
        case 93: { constexpr int KK = 9, VV = 3; return CALL; }                            \
        default: return cudaErrorInvalidValue;                                             \
    }

}  // namespace

const char* batch_variant_name(int v) {
    switch (v) {
        case 0: return "tile 32x8, 5 blocks/SM";
        case 1: return "tile 32x4, 10 blocks/SM";
        case 2: return "tile 32x16, 2 blocks/SM";
        case 3: return "tile 32x8, 4 blocks/SM";
        default: return "?";
    }
}

int batch_variant_tile_h(int variant) {
    switch (variant) {
        case 1: return Variant<1>::TH;
        case 2: return Variant<2>::TH;
        case 3: return Variant<3>::TH;
        default: return Variant<0>::TH;
    }
}

int batch_iter_blocks_per_sm(int k, int variant) {
    switch (k) {
        case 3: return occupancy_k<3>(variant);
        case 5: return occupancy_k<5>(variant);
        case 7: return occupancy_k<7>(variant);
        case 9: return occupancy_k<9>(variant);
        default: return 1;
    }
}

cudaError_t launch_batch_iter(int k, int variant, const BatchPair* pairs, const BatchClip* clips,
                              const int32_t* item_pair, const int32_t* item_tile, int n_items,
                              int per_claim, int* counter, uint64_t seed, int it, const uint32_t* Fp,
                              const uint32_t* Ep, uint32_t* Fn, uint32_t* En, int grid,
                              cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    if (per_claim < 1) return cudaErrorInvalidValue;
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    const uint32_t cw = static_cast<uint32_t>(it + 1) << 8;  // level 0
    FB_BATCH_DISPATCH(k, variant, (launch_iter_kv<KK, VV>(pairs, clips, item_pair, item_tile, n_items,
                                                         per_claim, counter, k0, k1, cw, Fp, Ep, Fn, En,
                                                         grid, st)));
}

cudaError_t launch_batch_init(int k, int variant, const BatchPair* pairs, const BatchClip* clips,
                              const int32_t* item_pair, const int32_t* item_tile, int n_items,
                              int* counter, uint64_t seed, uint32_t* F, uint32_t* E, int grid,
                              cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    FB_BATCH_DISPATCH(k, variant, (launch_init_kv<KK, VV>(pairs, clips, item_pair, item_tile, n_items,
                                                         counter, k0, k1, F, E, grid, st)));
}

cudaError_t launch_batch_combine(int k, const BatchJob* jobs, const BatchPair* pairs,
                                 const BatchClip* clips, const int32_t* item_job,
                                 const int32_t* item_tile, int n_items, int* counter,
                                 const uint32_t* F, int grid, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    const dim3 block(32, 8);
    switch (k) {
        case 3: batch_combine_kernel<3><<<grid, block, 0, st>>>(jobs, pairs, clips, item_job, item_tile, n_items, counter, F); break;
        case 5: batch_combine_kernel<5><<<grid, block, 0, st>>>(jobs, pairs, clips, item_job, item_tile, n_items, counter, F); break;
        case 7: batch_combine_kernel<7><<<grid, block, 0, st>>>(jobs, pairs, clips, item_job, item_tile, n_items, counter, F); break;
        case 9: batch_combine_kernel<9><<<grid, block, 0, st>>>(jobs, pairs, clips, item_job, item_tile, n_items, counter, F); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

#ifdef FB_CHECKED
cudaError_t check_read_batch(unsigned long long out[3], bool reset) {
    return dev::check_read_unit(out, reset);
}
#endif

}  // namespace fb
