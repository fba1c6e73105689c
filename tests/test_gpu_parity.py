"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

NNFs and patch errors must be bit-exact; blended / interpolated pixels must agree to
0.5/255 in float32 (the path is exact integer arithmetic plus one IEEE division per
value, so in practice they agree bit for bit, which is also checked).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 0.5 / 255.0


@pytest.fixture(scope="module")
def fbp():
    import paper_2311_09265_b300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def ctx(fbp):
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    c = fbp.Context(0)
    yield c
    c.close()


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def gpu_nnf(fbp, ctx, s, t, patch, iters, levels=1, r0=0, seed=0, tag=0, init=None):
    p = fbp.Params.make(patch, iters, levels, r0, seed, tag)
    F, E = fbp.fb_nnf(ctx, cuda(s), cuda(t), p, init_nnf=None if init is None else cuda(init))
    return host(F), host(E).view(np.uint32)


# ----------------------------------------------------------------------------------
# Alg. 1 NNF: bit-exact F and E
# ----------------------------------------------------------------------------------
NNF_CASES = [
    # H, W, k, iters, levels, r0, motion
    (37, 53, 5, 0, 1, 0, "shift"),
    (37, 53, 5, 1, 1, 0, "shift"),
    (96, 96, 5, 4, 1, 0, "shift"),
    (64, 70, 3, 3, 1, 0, "affine"),
    (41, 45, 7, 2, 1, 0, "affine"),
    (30, 33, 9, 2, 1, 0, "affine"),
    (61, 77, 5, 2, 2, 0, "shift"),
    (50, 47, 5, 2, 3, 0, "affine"),
    (40, 44, 5, 3, 1, 4, "affine"),
    (9, 9, 9, 3, 1, 0, "affine"),     # smallest image for the largest patch
    (5, 300, 5, 2, 1, 0, "affine"),   # one tile row, ragged width
]


@pytest.mark.parametrize("H,W,k,iters,levels,r0,motion", NNF_CASES)
def test_nnf_bit_exact(fbp, ctx, H, W, k, iters, levels, r0, motion):
    g, _ = synth.small_clip(3, H, W, seed=H * 1000 + W + k, motion=motion)
    tag = oracle.pair_tag(2, 0)
    Fg, Eg = gpu_nnf(fbp, ctx, g[2], g[0], k, iters, levels, r0, seed=1234, tag=tag)
    Fo, Eo = oracle.nnf(g[2], g[0], k, iters, levels=levels, r0=r0, seed=1234, pair_tag=tag)
    assert (Fg == Fo).all(), np.argwhere((Fg != Fo).any(-1))[:5]
    assert (Eg == Eo).all()


def test_nnf_bit_exact_with_user_init(fbp, ctx):
    g, sh = synth.shift_clip(2, 48, 52, seed=5)
    rng = np.random.default_rng(0)
    init = np.stack([rng.integers(-5, 60, (48, 52)), rng.integers(-5, 60, (48, 52))], -1).astype(np.int32)
    Fg, Eg = gpu_nnf(fbp, ctx, g[0], g[1], 5, 2, seed=9, tag=77, init=init)
    Fo, Eo = oracle.nnf(g[0], g[1], 5, 2, seed=9, pair_tag=77, init=init)
    assert (Fg == Fo).all() and (Eg == Eo).all()


@pytest.mark.parametrize("H,W,k,iters,r0", [(37, 53, 3, 3, 0), (61, 77, 5, 3, 0), (41, 45, 7, 2, 0),
                                            (30, 33, 9, 2, 5), (5, 300, 5, 2, 0)])
def test_nnf_step_chain_reproduces_the_oracle_iterations(fbp, ctx, H, W, k, iters, r0):
    """fb_nnf_step from the oracle's initial field, stepped `iters` times, gives the
    oracle's field and errors after each iteration (Sec. 3.2 Jacobi schedule, one
    launch per step)."""
    g, _ = synth.small_clip(2, H, W, seed=H + 7 * W + k, motion="affine")
    tag = oracle.pair_tag(1, 0)
    F, E = oracle.nnf(g[1], g[0], k, 0, r0=r0, seed=77, pair_tag=tag)
    src, tgt = cuda(g[1]), cuda(g[0])
    p = fbp.Params.make(k, 0, 1, r0, 77, tag)
    Fd, Ed = cuda(F), cuda(E.view(np.int32))
    for it in range(iters):
        Fd, Ed = fbp.fb_nnf_step(ctx, src, tgt, p, it, Fd, Ed)
        Fo, Eo = oracle.nnf(g[1], g[0], k, it + 1, r0=r0, seed=77, pair_tag=tag)
        assert (host(Fd) == Fo).all() and (host(Ed).view(np.uint32) == Eo).all(), it


def test_nnf_step_rejects_what_it_does_not_compute(fbp, ctx):
    g, _ = synth.small_clip(2, 24, 24, seed=1)
    src, tgt = cuda(g[1]), cuda(g[0])
    F = cuda(np.zeros((24, 24, 2), np.int32))
    E = cuda(np.zeros((24, 24), np.int32))
    for p, it in [(fbp.Params.make(5, 1, 2), 0), (fbp.Params.make(5, 1, flags=fbp.FB_FLAG_TRACKING), 0),
                  (fbp.Params.make(5, 1), -1), (fbp.Params.make(5, 1), 65535)]:
        with pytest.raises(fbp.FastBlendError) as e:
            fbp.fb_nnf_step(ctx, src, tgt, p, it, F, E)
        assert e.value.status == fbp.FB_ERR_ARG


def test_nnf_seed_and_tag_change_the_stream(fbp, ctx):
    g, _ = synth.small_clip(2, 32, 32, seed=3)
    a = gpu_nnf(fbp, ctx, g[0], g[1], 5, 1, seed=1, tag=1)[0]
    b = gpu_nnf(fbp, ctx, g[0], g[1], 5, 1, seed=1, tag=2)[0]
    c = gpu_nnf(fbp, ctx, g[0], g[1], 5, 1, seed=1, tag=1)[0]
    assert (a != b).any() and (a == c).all()


# ----------------------------------------------------------------------------------
# Alg. 2 remap
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("H,W,k", [(33, 47, 3), (64, 64, 5), (29, 71, 7), (18, 19, 9)])
def test_remap_bit_exact(fbp, ctx, H, W, k):
    rng = np.random.default_rng(H + W + k)
    S = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    F = np.stack([rng.integers(-3, H + 3, (H, W)), rng.integers(-3, W + 3, (H, W))], -1).astype(np.int32)
    out = host(fbp.fb_remap(ctx, cuda(S), cuda(F), k))
    ref = oracle.remap(S, F, k)
    assert np.abs(out - ref).max() <= TOL
    assert (out == ref).all()


@pytest.mark.parametrize("H,W,k", [(9, 32760, 9), (32760, 9, 9), (9, 32761, 5), (32761, 9, 5)])
def test_remap_at_the_packed_clamp_bound(fbp, ctx, H, W, k):
    """The remap forms both clamped source coordinates of a vote with one per-halfword
    instruction on the packed field word for frames up to 32760 pixels a side (the largest
    side at which no half leaves the signed 16-bit range, with the largest patch), and with
    scalar clamps above that: both sides of the bound, fields running past every edge."""
    rng = np.random.default_rng(H + 3 * W + k)
    S = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    F = np.stack([rng.integers(-6, H + 6, (H, W)), rng.integers(-6, W + 6, (H, W))], -1).astype(np.int32)
    # the fields along the far edges point at the far edges, where the votes' offsets reach
    F[-2:, :, 0] = H - 1
    F[:, -2:, 1] = W - 1
    out = host(fbp.fb_remap(ctx, cuda(S), cuda(F), k))
    assert (out == oracle.remap(S, F, k)).all()


# ----------------------------------------------------------------------------------
# Eq. 2 window blend
# ----------------------------------------------------------------------------------
BLEND_CASES = [
    # N, H, W, k, window, iters, levels, motion
    (8, 96, 96, 5, 3, 4, 1, "shift"),      # the 8-frame 96x96 workload
    (7, 45, 61, 3, 5, 2, 1, "affine"),
    (5, 40, 36, 7, 3, 2, 1, "affine"),
    (6, 50, 42, 5, 7, 2, 2, "shift"),      # window larger than the clip, 2 levels
    (4, 33, 35, 9, 3, 1, 1, "affine"),
    (1, 20, 20, 5, 3, 2, 1, "shift"),      # single frame: no pairs
    (5, 20, 24, 5, 1, 2, 1, "shift"),      # window 1: output = style
]


@pytest.mark.parametrize("N,H,W,k,window,iters,levels,motion", BLEND_CASES)
def test_blend_window_matches_oracle(fbp, ctx, N, H, W, k, window, iters, levels, motion):
    g, s = synth.small_clip(N, H, W, seed=N * 100 + H + W, motion=motion)
    p = fbp.Params.make(k, iters, levels, 0, 4242)
    out = host(fbp.fb_blend_window(ctx, cuda(g), cuda(s), window, p))
    ref = oracle.blend_window(g, s, window, k, iters, levels=levels, seed=4242)
    assert np.abs(out - ref).max() <= TOL
    assert (out == ref).all()


def test_blend_window_host_buffers_equal_device_buffers(fbp, ctx):
    import torch
    g, s = synth.small_clip(6, 40, 52, seed=8)
    p = fbp.Params.make(5, 2, 1, 0, 11)
    dev = host(fbp.fb_blend_window(ctx, cuda(g), cuda(s), 3, p))
    gh = torch.from_numpy(g).pin_memory()
    sh = torch.from_numpy(s).pin_memory()
    hst = fbp.fb_blend_window(ctx, gh, sh, 3, p).numpy()
    assert (dev == hst).all()
    # pageable host memory works too
    assert (fbp.fb_blend_window(ctx, torch.from_numpy(g.copy()), torch.from_numpy(s.copy()), 3,
                                p).numpy() == dev).all()


def test_host_buffer_calls_split_into_chunks_give_the_device_results(fbp, ctx):
    """A host-buffer call whose pairs hold at least 4 x 2^21 pixels is cut into at least four
    chunks of output frames, so each chunk's frames leave while the next chunk's NNFs are
    computed; the device-buffer call of the same clip runs as one chunk.  Same results;
    more iteration launches for the host call show the cut."""
    import torch
    g, s = synth.small_clip(72, 256, 256, seed=31)
    ks = np.ascontiguousarray(s[[0, 71]])
    p = fbp.Params.make(5, 2, 1, 0, 17)
    n0 = ctx.launches
    a = host(fbp.fb_interpolate(ctx, cuda(g), [0, 71], cuda(ks), p))
    n_dev = ctx.launches - n0
    gh = torch.from_numpy(g).pin_memory()
    n0 = ctx.launches
    b = fbp.fb_interpolate(ctx, gh, [0, 71], torch.from_numpy(ks).pin_memory(), p).numpy()
    n_host = ctx.launches - n0
    assert (a == b).all()
    # 140 NNFs of 65,536 pixels: one chunk on the device, four from host buffers (2 more
    # iterations, an init and a combine per extra chunk; the combine split in groups)
    assert n_host >= n_dev + 3 * (p.iters + 2)
    assert (a[35] == oracle.interpolate_frame(g, [0, 71], ks, 35, 5, 2, seed=17)).all()
    g2, s2 = synth.small_clip(20, 256, 256, seed=32)
    d = host(fbp.fb_blend_window(ctx, cuda(g2), cuda(s2), 9, p))
    h = fbp.fb_blend_window(ctx, torch.from_numpy(g2).pin_memory(), torch.from_numpy(s2).pin_memory(), 9,
                            p).numpy()
    assert (d == h).all()


def test_host_buffers_in_chunks_and_modes_equal_device_buffers(fbp, ctx):
    """Host buffers move through a copy stream (styles in while the search runs, frames out
    in groups as their combine finishes): the results equal the device-buffer call for
    several chunks, for interpolation and for a mode that reads the styles early."""
    import torch
    g, s = synth.small_clip(8, 96, 96, seed=21)
    gh, sh = torch.from_numpy(g).pin_memory(), torch.from_numpy(s).pin_memory()
    p = fbp.Params.make(5, 2, 1, 0, 13)
    ctx.set_pair_budget(1 << 20)   # one to two output frames of 96x96 pairs per chunk
    try:
        dev = host(fbp.fb_blend_window(ctx, cuda(g), cuda(s), 7, p))
        hst = fbp.fb_blend_window(ctx, gh, sh, 7, p).numpy()
    finally:
        ctx.set_pair_budget(0)
    assert (dev == hst).all()
    assert (dev == oracle.blend_window(g, s, 7, 5, 2, seed=13)).all()
    ks = np.ascontiguousarray(s[[0, 7]])
    a = host(fbp.fb_interpolate(ctx, cuda(g), [0, 7], cuda(ks), p))
    b = fbp.fb_interpolate(ctx, gh, [0, 7], torch.from_numpy(ks).pin_memory(), p).numpy()
    assert (a == b).all()
    pb = fbp.Params.make(5, 2, 1, 0, 13, flags=fbp.FB_FLAG_BALANCED, alpha=10)
    a = host(fbp.fb_blend_window(ctx, cuda(g), cuda(s), 5, pb))
    b = fbp.fb_blend_window(ctx, gh, sh, 5, pb).numpy()
    assert (a == b).all()


def test_blend_window_is_deterministic_and_counts_launches(fbp, ctx):
    g, s = synth.small_clip(5, 32, 32, seed=2)
    p = fbp.Params.make(5, 3, 1, 0, 3)
    n0 = ctx.launches
    a = host(fbp.fb_blend_window(ctx, cuda(g), cuda(s), 3, p))
    n1 = ctx.launches
    b = host(fbp.fb_blend_window(ctx, cuda(g), cuda(s), 3, p))
    assert (a == b).all()
    # prep + style + init + 3 iterations + combine
    assert n1 - n0 == 1 + 1 + 1 + 3 + 1


# ----------------------------------------------------------------------------------
# Sec. 3.5.2 interpolation
# ----------------------------------------------------------------------------------
INTERP_CASES = [
    # N, H, W, k, keys, iters
    (9, 50, 40, 5, (0, 8), 3),
    (10, 36, 44, 7, (2, 5, 7), 2),
    (6, 30, 30, 5, (3,), 2),
    (5, 28, 31, 3, (0, 1, 2, 3, 4), 1),     # every frame a key
    (7, 33, 29, 9, (6,), 1),                # before the only key
]


@pytest.mark.parametrize("N,H,W,k,keys,iters", INTERP_CASES)
def test_interpolate_matches_oracle(fbp, ctx, N, H, W, k, keys, iters):
    g, s = synth.small_clip(N, H, W, seed=N + H * W, motion="affine")
    ks = np.ascontiguousarray(s[list(keys)])
    p = fbp.Params.make(k, iters, 1, 0, 99)
    out = host(fbp.fb_interpolate(ctx, cuda(g), list(keys), cuda(ks), p))
    ref = oracle.interpolate(g, list(keys), ks, k, iters, seed=99)
    assert np.abs(out - ref).max() <= TOL
    assert (out == ref).all()


# ----------------------------------------------------------------------------------
# Argument errors: FB_ERR_ARG before any launch
# ----------------------------------------------------------------------------------
def test_argument_errors(fbp, ctx):
    import torch
    g = torch.zeros((4, 16, 16, 3), dtype=torch.uint8, device="cuda")
    n0 = ctx.launches
    bad = [
        lambda: fbp.fb_blend_window(ctx, g, g, 3, fbp.Params.make(4, 2)),     # even patch
        lambda: fbp.fb_blend_window(ctx, g, g, 3, fbp.Params.make(11, 2)),    # patch > 9
        lambda: fbp.fb_blend_window(ctx, g, g, 2, fbp.Params.make(5, 2)),     # even window
        lambda: fbp.fb_blend_window(ctx, g, g, 3, fbp.Params.make(5, -1)),    # iters < 0
        lambda: fbp.fb_blend_window(ctx, g, g, 3, fbp.Params.make(5, 2, 0)),  # levels 0
        lambda: fbp.fb_interpolate(ctx, g, [2, 1], g[:2], fbp.Params.make(5, 2)),  # unsorted
        lambda: fbp.fb_interpolate(ctx, g, [0, 4], g[:2], fbp.Params.make(5, 2)),  # out of range
        lambda: fbp.fb_nnf(ctx, g[0], g[1], fbp.Params.make(5, 2, 2),
                           init_nnf=torch.zeros((16, 16, 2), dtype=torch.int32, device="cuda")),
        lambda: fbp.fb_nnf(ctx, g[0].cpu(), g[1], fbp.Params.make(5, 2)),       # host pointer
        lambda: fbp.fb_blend_window(ctx, g, g.cpu(), 3, fbp.Params.make(5, 2)),  # mixed memory
        lambda: fbp.fb_nnf(ctx, g[0, :3, :3].contiguous(), g[1, :3, :3].contiguous(),
                           fbp.Params.make(5, 2)),                               # H < patch
    ]
    for f in bad:
        with pytest.raises(fbp.FastBlendError) as ei:
            f()
        assert ei.value.status == fbp.FB_ERR_ARG
    assert ctx.launches == n0


# ----------------------------------------------------------------------------------
# Full-size workloads in the launch configuration bench.py times, checked on samples
# the oracle can compute one by one.
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("H,W", [(9, 32767), (32767, 9)])
def test_nnf_at_the_largest_image_side(fbp, ctx, H, W):
    """The packed NNF entries (row << 16 | col) at the largest supported side, odd sizes
    (the paired k = 5 row layout's last pair then holds a clamped row)."""
    g = synth.noise_pair(H, W, seed=77)
    Fg, Eg = gpu_nnf(fbp, ctx, g[0], g[1], 5, 1, seed=5, tag=oracle.pair_tag(0, 1))
    Fo, Eo = oracle.nnf(g[0], g[1], 5, 1, seed=5, pair_tag=oracle.pair_tag(0, 1))
    assert (Fg == Fo).all() and (Eg == Eo).all()
    assert Fg[..., 0].max() <= H - 1 and Fg[..., 1].max() <= W - 1


@pytest.mark.slow
def test_blend_512_full_size_sampled_frames(fbp, ctx):
    w = synth.WORKLOADS["blend_512"]
    g, s = synth.make_clip("blend_512")
    seed = w.seed
    p = fbp.Params.make(w.patch, w.iters, 1, 0, seed)
    out = host(fbp.fb_blend_window(ctx, cuda(g), cuda(s), w.window, p))
    for i in (0, 31):
        ref = oracle.blend_frame(g, s, w.window, i, w.patch, w.iters, seed=seed)
        assert np.abs(out[i] - ref).max() <= TOL
        assert (out[i] == ref).all()
    # one pair's NNF, bit-exact, through fb_nnf with that pair's tag
    tag = oracle.pair_tag(33, 31)
    Fg, Eg = gpu_nnf(fbp, ctx, g[33], g[31], w.patch, w.iters, seed=seed, tag=tag)
    Fo, Eo = oracle.nnf(g[33], g[31], w.patch, w.iters, seed=seed, pair_tag=tag)
    assert (Fg == Fo).all() and (Eg == Eo).all()


@pytest.mark.slow
def test_interp_1024x576_full_size_sampled_frame(fbp, ctx):
    w = synth.WORKLOADS["interp_1024x576"]
    g, ks = synth.make_clip("interp_1024x576")
    p = fbp.Params.make(w.patch, w.iters, 1, 0, w.seed)
    out = host(fbp.fb_interpolate(ctx, cuda(g), list(w.keys), cuda(ks), p))
    for i in (0, 23):
        ref = oracle.interpolate_frame(g, list(w.keys), ks, i, w.patch, w.iters, seed=w.seed)
        assert np.abs(out[i] - ref).max() <= TOL
        assert (out[i] == ref).all()
