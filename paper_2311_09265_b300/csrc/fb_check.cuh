// fb_check.cuh -- device-side invariant checks of the checked build.
//
// Checked builds (-DFB_CHECKED, libfb_checked.so) test on the device the index and data
// invariants of the NNF path at the FB_CHECK_* sites of fb.h.  FB_CHECK(ok, site, a, b)
// evaluates to ok; when ok is false it also records (site, a, b) as the translation
// unit's first failure (if none is recorded yet) and counts the failure.  Callers skip
// the access or candidate the check guards, so a failed check never faults, traps or
// stops the kernel; the host reads the words with fb_check_status.  Product builds
// compile FB_CHECK to `true` without evaluating its arguments, and FB_CHECK_TALLY and
// FB_CHECKED_ONLY to nothing.
//
// The words are static, one set per translation unit that includes this header
// (libfb.so is built without relocatable device code); each such unit exposes a host
// reader (fb_internal.h: check_read_kernels, check_read_batch).
#pragma once

#include <cstdint>

#include "fb_internal.h"

namespace fb {
namespace dev {

#ifdef FB_CHECKED

struct CheckWords {
    unsigned long long first;      // (site << 56) | (a << 28) | b of the first failure, or 0
    unsigned long long failed;     // failed checks
    unsigned long long evaluated;  // pixel visits that ran the checks
};
static __device__ CheckWords g_check;

static __device__ __noinline__ void check_record(uint32_t site, uint32_t a, uint32_t b) {
    const unsigned long long w = (static_cast<unsigned long long>(site) << 56) |
                                 (static_cast<unsigned long long>(a & 0xFFFFFFFu) << 28) |
                                 static_cast<unsigned long long>(b & 0xFFFFFFFu);
    atomicCAS(&g_check.first, 0ull, w);
    atomicAdd(&g_check.failed, 1ull);
}

__device__ __forceinline__ bool check(bool ok, uint32_t site, uint32_t a, uint32_t b) {
    if (!ok) check_record(site, a, b);
    return ok;
}

// Adds n visits per calling thread, one atomic per warp.
__device__ __forceinline__ void check_tally(uint32_t n) {
    const unsigned mask = __activemask();
    const unsigned total = __reduce_add_sync(mask, n);
    unsigned lane;
    asm("mov.u32 %0, %%laneid;" : "=r"(lane));
    if (lane == static_cast<unsigned>(__ffs(mask) - 1))
        atomicAdd(&g_check.evaluated, static_cast<unsigned long long>(total));
}

// Host reader of this translation unit's words; zeroes them after reading if reset.
static cudaError_t check_read_unit(unsigned long long out[3], bool reset) {
    CheckWords w{};
    cudaError_t e = cudaMemcpyFromSymbol(&w, g_check, sizeof(w));
    if (e != cudaSuccess) return e;
    out[0] = w.first;
    out[1] = w.failed;
    out[2] = w.evaluated;
    if (reset) {
        const CheckWords zero{};
        e = cudaMemcpyToSymbol(g_check, &zero, sizeof(zero));
    }
    return e;
}

#define FB_CHECK(ok, site, a, b) \
    ::fb::dev::check((ok), (site), static_cast<uint32_t>(a), static_cast<uint32_t>(b))
#define FB_CHECK_TALLY(n) ::fb::dev::check_tally(n)
#define FB_CHECKED_ONLY(...) __VA_ARGS__

#else

#define FB_CHECK(ok, site, a, b) true
#define FB_CHECK_TALLY(n) ((void)0)
#define FB_CHECKED_ONLY(...)

#endif

// A packed match (row << 16) | col lies inside an H x W image.
__device__ __forceinline__ bool match_inside(uint32_t f, int H, int W) {
    return static_cast<int>(f >> 16) < H && static_cast<int>(f & 0xFFFFu) < W;
}

}  // namespace dev
}  // namespace fb
