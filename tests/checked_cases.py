"""Cases of the checked-build test (test_gpu_checked.py): every kernel family of the NNF
path -- initial fields at every mode, the Jacobi step of each loss, tracking, the
batched kernels, the remap and the combines -- on small seeded inputs.  run(fbp, ctx,
name) calls the library that `fbp` has loaded and returns the case's outputs as numpy
arrays; the test runs every case through libfb_checked.so in a child process and
through libfb.so in its own, and compares.
"""
import ctypes

import numpy as np

import synth

# name -> (kind, arguments)
CASES = {
    # fb_nnf: H, W, k, iters, levels, r0
    "nnf_k3": ("nnf", (64, 70, 3, 3, 1, 0)),
    "nnf_k5_pyramid": ("nnf", (61, 77, 5, 2, 3, 0)),
    "nnf_k5_one_tile_row": ("nnf", (5, 300, 5, 2, 1, 0)),
    "nnf_k7": ("nnf", (41, 45, 7, 2, 1, 0)),
    "nnf_k9_r0": ("nnf", (30, 33, 9, 2, 1, 4)),
    "nnf_user_init": ("nnf_init", (48, 52, 5, 2)),
    "remap_out_of_range_field": ("remap", (29, 71, 7)),
    # fb_blend_window: N, H, W, k, window, iters, levels, flags name
    "blend_plain": ("blend", (6, 40, 52, 5, 3, 2, 2, "")),
    "blend_balanced": ("blend", (5, 36, 40, 5, 3, 2, 1, "BALANCED")),
    "blend_accurate": ("blend", (5, 36, 40, 5, 3, 2, 1, "ACCURATE")),
    "blend_fast": ("blend", (7, 33, 35, 5, 5, 2, 1, "FAST")),
    "blend_tracking": ("blend", (6, 34, 38, 5, 5, 2, 1, "TRACKING")),
    "blend_k9": ("blend", (4, 33, 35, 9, 3, 1, 1, "")),
    # fb_interpolate: N, H, W, k, iters, keys, flags name
    "interp_plain": ("interp", (7, 36, 44, 7, 2, (0, 6), "")),
    "interp_tracking": ("interp", (7, 36, 44, 5, 2, (0, 6), "TRACKING")),
    "interp_align": ("interp", (7, 36, 44, 5, 2, (1, 5), "ALIGN")),
    "interp_align_tracking": ("interp", (6, 32, 40, 5, 2, (0, 5), "ALIGN|TRACKING")),
    "segment_align_tracking": ("segment", (4, 30, 34, 5, 2)),
    "batch_two_clips": ("batch", ()),
    "blend_range": ("range", (10, 30, 36, 5, 5, 2)),
    "noalloc": ("noalloc", (5, 32, 40, 5, 3, 2)),
}

SEED = 20231115


def _flags(fbp, names: str) -> int:
    v = 0
    for n in filter(None, names.split("|")):
        v |= getattr(fbp, "FB_FLAG_" + n)
    return v


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def nnf_visits(H: int, W: int, iters: int, levels: int) -> int:
    """Pixel visits of one fb_nnf call in a checked build: at every level one by the
    initial-field kernel and one per iteration."""
    total, h, w = 0, H, W
    for _ in range(levels):
        total += (1 + iters) * h * w
        h, w = (h + 1) // 2, (w + 1) // 2
    return total


def expected_visits(name: str):
    """The exact visit count of a case, where it has a closed form; else None."""
    kind, a = CASES[name]
    if kind == "nnf":
        H, W, k, iters, levels, r0 = a
        return nnf_visits(H, W, iters, levels)
    if kind == "nnf_init":
        H, W, k, iters = a
        return nnf_visits(H, W, iters, 1)
    if kind == "remap":
        H, W, k = a
        return H * W
    return None


def run(fbp, ctx, name: str):
    import torch
    kind, a = CASES[name]
    if kind == "nnf":
        H, W, k, iters, levels, r0 = a
        g, _ = synth.small_clip(2, H, W, seed=H * 1000 + W + k, motion="affine")
        p = fbp.Params.make(k, iters, levels, r0, SEED, fbp.fb_pair_tag(1, 0))
        F, E = fbp.fb_nnf(ctx, _cuda(g[1]), _cuda(g[0]), p)
        return [_host(F), _host(E)]
    if kind == "nnf_init":
        H, W, k, iters = a
        g, _ = synth.shift_clip(2, H, W, seed=5)
        rng = np.random.default_rng(0)
        init = np.stack([rng.integers(-5, H + 8, (H, W)), rng.integers(-5, W + 8, (H, W))], -1)
        p = fbp.Params.make(k, iters, 1, 0, SEED, 77)
        F, E = fbp.fb_nnf(ctx, _cuda(g[0]), _cuda(g[1]), p, init_nnf=_cuda(init.astype(np.int32)))
        return [_host(F), _host(E)]
    if kind == "remap":
        H, W, k = a
        rng = np.random.default_rng(H + W + k)
        S = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
        F = np.stack([rng.integers(-3, H + 3, (H, W)), rng.integers(-3, W + 3, (H, W))], -1)
        return [_host(fbp.fb_remap(ctx, _cuda(S), _cuda(F.astype(np.int32)), k))]
    if kind == "blend":
        N, H, W, k, window, iters, levels, fl = a
        g, s = synth.small_clip(N, H, W, seed=N * 100 + H + W, motion="affine")
        p = fbp.Params.make(k, iters, levels, 0, SEED, flags=_flags(fbp, fl), alpha=4)
        return [_host(fbp.fb_blend_window(ctx, _cuda(g), _cuda(s), window, p))]
    if kind == "interp":
        N, H, W, k, iters, keys, fl = a
        g, s = synth.small_clip(N, H, W, seed=N * 10 + H + W, motion="affine")
        p = fbp.Params.make(k, iters, 1, 0, SEED, flags=_flags(fbp, fl), alpha=4)
        return [_host(fbp.fb_interpolate(ctx, _cuda(g), list(keys), _cuda(s[list(keys)]), p))]
    if kind == "segment":
        n, H, W, k, iters = a
        g, s = synth.small_clip(n + 2, H, W, seed=7, motion="affine")
        p = fbp.Params.make(k, iters, 1, 0, SEED, flags=fbp.FB_FLAG_ALIGN | fbp.FB_FLAG_TRACKING, alpha=4)
        F, E = fbp.fb_nnf_segment(ctx, _cuda(g), _cuda(s[[0, n + 1]]), p)
        return [_host(F), _host(E)]
    if kind == "batch":
        g1, s1 = synth.small_clip(6, 40, 52, seed=31, motion="affine")
        g2, s2 = synth.small_clip(5, 33, 47, seed=32, motion="shift")
        p = fbp.Params.make(5, 2, 1, 0, SEED)
        outs = fbp.fb_blend_batch(ctx, [(_cuda(g1), _cuda(s1), 3, 5), (_cuda(g2), _cuda(s2), 5, 7)], p)
        return [_host(o) for o in outs]
    if kind == "range":
        N, H, W, k, window, iters = a
        g, s = synth.small_clip(N, H, W, seed=41, motion="affine")
        M = window // 2
        out_first, n_out = 3, 4
        base, end = max(0, out_first - M), min(N, out_first + n_out + M)
        p = fbp.Params.make(k, iters, 1, 0, SEED)
        out = fbp.fb_blend_window_range(ctx, _cuda(g[base:end]), _cuda(s[base:end]), window, p, N, base,
                                        out_first, n_out)
        return [_host(out)]
    if kind == "noalloc":
        N, H, W, k, window, iters = a
        g, s = synth.small_clip(N, H, W, seed=51, motion="affine")
        gd, sd = _cuda(g), _cuda(s)
        out = torch.full((N, H, W, 3), -1.0, dtype=torch.float32, device="cuda")
        p = fbp.Params.make(k, iters, 1, 0, SEED)
        rc = fbp.lib().fb_blend_window_noalloc(gd.data_ptr(), sd.data_ptr(), N, H, W, window, ctypes.byref(p),
                                               out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert rc == fbp.FB_OK, fbp.lib().fb_last_error(None).decode()
        return [_host(out)]
    raise KeyError(name)
