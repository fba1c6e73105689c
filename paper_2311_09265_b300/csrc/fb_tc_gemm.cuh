// fb_tc_gemm.cuh -- a BF16 GEMM on the 5th-generation tensor cores (tcgen05) whose
// operands are gathered by the CTA's threads, used by the 3x3 convolutions of the
// learned NNF initialiser where the TMA-staged kernels (fb_tc_tma.cuh) do not apply: the
// layers whose output rows do not tile 128-pixel blocks, and the input gradients of
// stride-2 layers with odd inputs.
//
//   D[M x N] (+)= A[M x K] . B[N x K]^T,  bf16 inputs, fp32 accumulation in TMEM.
//
// A CTA of 128 threads owns an M = 128 by BN tile.  K advances in chunks of 64: the
// threads gather the chunk's A and B tiles into shared memory in the no-swizzle
// K-major layout (8-row x 16-byte core matrices; consecutive core matrices along K
// LBO = 128 bytes apart, along M/N SBO = 1024 bytes apart), one elected thread issues
// four tcgen05.mma (K = 16 each) and commits them to the stage's mbarrier, and the
// threads move on to gather the next chunk into the other stage.  The epilogue reads
// the accumulator from TMEM with tcgen05.ld (warp w owns rows 32w .. 32w+31).  Every
// mbarrier wait is bounded; on expiry the kernel records an error code and skips its
// epilogue, and TMEM is always released.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

namespace fb {
namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;              // K per stage: 8 core-matrix columns, 4 MMAs
constexpr int LBO = 128;            // bytes between core matrices along K
constexpr int SBO = 1024;           // bytes between 8-row groups (BK / 8 * 128)
constexpr long kWaitLimit = 1L << 26;
// Polls a PROGRESS wait (one that gates further work: operands landed, a stage free, the
// accumulator complete) makes before the kernel gives up and reports a timeout.  Host code
// may lower it (fb_debug_set_wait_limit) to exercise the timeout path; DRAIN waits (for
// MMAs already committed and copies already issued, before the CTA releases TMEM and
// shared memory) always use kWaitLimit.
static __device__ long g_progress_wait_limit = kWaitLimit;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start >> 4, LBO >> 4 at bit 16, SBO >> 4 at bit 32,
// descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) |
           (static_cast<uint64_t>((LBO >> 4) & 0x3FFFu) << 16) |
           (static_cast<uint64_t>((SBO >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: fp32 D, bf16 A and B, both K-major, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
           (static_cast<uint32_t>(BM >> 4) << 24);
}

// Byte offset of element (row, k) of a 64-wide K chunk in the core-matrix layout.
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
    return static_cast<uint32_t>((row >> 3) * SBO + (k >> 3) * LBO + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long limit = kWaitLimit) {
    uint32_t done = 0;
    for (long it = 0; it < limit && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity));
    }
    return done != 0;
}

// The progress-wait limit, read once by a kernel (the host sets it between launches).
__device__ __forceinline__ long progress_limit() { return g_progress_wait_limit; }

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar)));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
        "%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

template <int BN>
struct TmemCols {
    static constexpr int value = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
};

// Gather contract: Gather::load(stage_a, stage_b, k0, m0, n0) fills the 128 x 64 A tile
// and the BN x 64 B tile of K chunk [k0, k0 + 64) with tile_off() addressing (zeros
// outside the matrices); Epi::store(row, col0, v[16]) consumes 16 accumulator columns
// of one row.  Every thread of the CTA calls both.
template <int BN, class Gather, class Epi>
__global__ void __launch_bounds__(128) tc_gemm_kernel(Gather gather, Epi epi, int M, int N,
                                                      int K, int k_chunks_per_split,
                                                      int* status) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 128, "tile N");
    constexpr int A_BYTES = BM * BK * 2;   // 16 KB
    constexpr int B_BYTES = BN * BK * 2;
    constexpr int STAGE = A_BYTES + B_BYTES;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tmem_base;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int n_chunks_total = (K + BK - 1) / BK;
    const int c_begin = blockIdx.z * k_chunks_per_split;
    const int c_end = min(n_chunks_total, c_begin + k_chunks_per_split);

    if (threadIdx.x == 0) {
        mbar_init(&bars[0]);
        mbar_init(&bars[1]);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TmemCols<BN>::value));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = instr_desc(BN);

    bool ok = true;
    int issued = 0;
    int last_commit = -1;  // thread 0: last chunk (relative) whose MMAs it committed
    const long lim = progress_limit();
    for (int c = c_begin; c < c_end; ++c) {
        const int s = (c - c_begin) & 1;
        const int use = (c - c_begin) >> 1;  // how many times stage s was used before
        unsigned char* sa = smem + s * STAGE;
        unsigned char* sb = sa + A_BYTES;
        if (use > 0 && ok) ok = mbar_wait(&bars[s], (use - 1) & 1, lim);  // MMAs of that stage done
        gather.load(sa, sb, c * BK, m0, n0);
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (threadIdx.x == 0 && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int j = 0; j < BK / 16; ++j) {
                mma_bf16(tmem, smem_desc(smem_u32(sa) + j * 2 * LBO), smem_desc(smem_u32(sb) + j * 2 * LBO),
                         idesc, (c > c_begin || j > 0) ? 1u : 0u);
            }
            mma_commit(&bars[s]);
            last_commit = c - c_begin;
        }
        ++issued;
    }
    if (issued > 0 && ok) {
        const int last = issued - 1;
        ok = mbar_wait(&bars[last & 1], (last >> 1) & 1, lim);
    }
    if (!ok && lane == 0) atomicExch(status, 1);
    // After a timeout, let the MMAs already committed finish before TMEM is released (they
    // complete in issue order, so the last commit's phase covers them all).
    if (!ok && threadIdx.x == 0 && last_commit >= 0)
        mbar_wait(&bars[last_commit & 1], (last_commit >> 1) & 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && issued > 0) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
            if (row < M && n0 + c0 < N) epi.store(row, n0 + c0, v);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TmemCols<BN>::value));
}

template <int BN>
constexpr int gemm_smem_bytes() {
    return 2 * (BM * BK * 2 + BN * BK * 2);
}

// ---- asynchronous-copy variant ------------------------------------------------------
// 16-byte global -> shared copy that does not pass through registers (cp.async, L2 only);
// src_bytes = 0 writes zeros (the convolution's padding) and reads nothing.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Same GEMM with an S-stage pipeline: the threads issue the asynchronous copies of the
// chunks S-1 ahead of the one being multiplied, so several chunks of operand loads are
// in flight while the tensor cores work.  The gather decides the K order:
//   Gather::State st = gather.thread_state(m0)   per-thread set-up, once per CTA
//   gather.chunks()                              number of K chunks
//   gather.k_steps(c)                            K = 16 MMAs chunk c needs (1..4)
//   gather.load_async(st, sa, sb, c, n0)         issues (without waiting) the copies of
//                                                chunk c into shared addresses sa (A) /
//                                                sb (B), tile_off() layout, zeros where
//                                                the chunk has no data
// Stage s is refilled only after the mbarrier of its previous MMAs has fired.  Waits are
// bounded as above.
template <int BN, int S, class Gather, class Epi, int LA = S - 1>
__global__ void __launch_bounds__(128) tc_gemm_async_kernel(Gather gather, Epi epi, int M, int N,
                                                            int K, int* status) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 128, "tile N");
    static_assert(S >= 2 && S <= 8 && LA >= 1 && LA <= S - 1, "stages / lookahead");
    constexpr int A_BYTES = BM * BK * 2;
    constexpr int B_BYTES = BN * BK * 2;
    constexpr int STAGE = A_BYTES + B_BYTES;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[S];
    __shared__ uint32_t tmem_base;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int n_chunks = gather.chunks();
    (void)K;
    const typename Gather::State gst = gather.thread_state(m0);

    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) mbar_init(&bars[s]);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TmemCols<BN>::value));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = instr_desc(BN);
    const uint32_t s0 = smem_u32(smem);

    // Chunks are loaded LA ahead; chunk i + LA reuses the stage of chunk i + LA - S,
    // whose MMAs were issued S - LA iterations earlier.
#pragma unroll
    for (int i = 0; i < LA; ++i) {
        if (i < n_chunks) gather.load_async(gst, s0 + i * STAGE, s0 + i * STAGE + A_BYTES, i, n0);
        cp_async_commit();
    }
    bool ok = true;
    int last_commit = -1;  // thread 0: last chunk whose MMAs it committed
    const long lim = progress_limit();
    for (int i = 0; i < n_chunks; ++i) {
        const int s = i % S;
        cp_async_wait<LA - 1>();  // this thread's copies of chunk i have landed
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();         // ... and every thread's
        if (threadIdx.x == 0 && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = s0 + s * STAGE, sb = sa + A_BYTES;
            const int steps = gather.k_steps(i);
            for (int j = 0; j < steps; ++j)
                mma_bf16(tmem, smem_desc(sa + j * 2 * LBO), smem_desc(sb + j * 2 * LBO), idesc,
                         (i > 0 || j > 0) ? 1u : 0u);
            mma_commit(&bars[s]);
            last_commit = i;
        }
        const int nxt = i + LA;
        const int prev = nxt - S;  // the chunk that last used nxt's stage
        if (nxt < n_chunks) {
            if (prev >= 0 && ok) ok = mbar_wait(&bars[prev % S], (prev / S) & 1, lim);
            if (ok) {
                const uint32_t sa = s0 + (nxt % S) * STAGE;
                gather.load_async(gst, sa, sa + A_BYTES, nxt, n0);
            }
        }
        cp_async_commit();
    }
    cp_async_wait<0>();   // no copy of this thread is in flight past this point
    if (n_chunks > 0 && ok) ok = mbar_wait(&bars[(n_chunks - 1) % S], ((n_chunks - 1) / S) & 1, lim);
    if (!ok && lane == 0) atomicExch(status, 1);
    // After a timeout, let the MMAs already committed finish before TMEM is released.
    if (!ok && threadIdx.x == 0 && last_commit >= 0)
        mbar_wait(&bars[last_commit % S], (last_commit / S) & 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok && n_chunks > 0) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
            if (row < M && n0 + c0 < N) epi.store(row, n0 + c0, v);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TmemCols<BN>::value));
}

template <int BN, int S>
constexpr int gemm_async_smem_bytes() {
    return S * (BM * BK * 2 + BN * BK * 2);
}

}  // namespace tc
}  // namespace fb
