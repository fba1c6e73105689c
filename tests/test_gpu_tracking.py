"""Tracking of Sec. 3.5.1 (FB_FLAG_TRACKING of fb_interpolate and fb_blend_window) on the GPU
against the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbp():
    import paper_2311_09265_b300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def ctx(fbp):
    c = fbp.Context(0)
    yield c
    c.close()


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


TRACK_CASES = [
    # N, H, W, k, keys, iters, motion
    (9, 50, 40, 5, (0, 8), 3, "affine"),       # two chains of 7 pairs
    (10, 36, 44, 7, (2, 5, 7), 2, "shift"),    # chains on both sides of inner keys
    (6, 30, 30, 5, (3,), 2, "affine"),         # one key, chains before and after it
    (7, 33, 29, 9, (6,), 1, "affine"),         # one chain ending at the key
    (6, 28, 31, 3, (0, 2, 4), 2, "shift"),     # chains of one pair: nothing to track
    (8, 21, 26, 5, (0, 7), 0, "affine"),       # no iterations: the random initialisation
]


@pytest.mark.parametrize("N,H,W,k,keys,iters,motion", TRACK_CASES)
def test_tracking_interpolation_matches_oracle(fbp, ctx, N, H, W, k, keys, iters, motion):
    g, s = synth.small_clip(N, H, W, seed=N * 7 + H, motion=motion)
    ks = np.ascontiguousarray(s[list(keys)])
    p = fbp.Params.make(k, iters, 1, 0, 31, flags=fbp.FB_FLAG_TRACKING)
    out = fbp.fb_interpolate(ctx, cuda(g), list(keys), cuda(ks), p).cpu().numpy()
    ref = oracle.interpolate_tracking(g, list(keys), ks, k, iters, seed=31)
    assert np.abs(out - ref).max() <= 0.5 / 255
    assert (out == ref).all()


def test_tracking_changes_the_result_where_chains_exist(fbp, ctx):
    # A guard that the flag reaches the kernel: with chains of several pairs the extra
    # candidates change some matches, so the output differs from the plain interpolation.
    g, s = synth.small_clip(9, 40, 40, seed=5, motion="affine")
    ks = np.ascontiguousarray(s[[0, 8]])
    plain = fbp.fb_interpolate(ctx, cuda(g), [0, 8], cuda(ks), fbp.Params.make(5, 2, 1, 0, 3))
    track = fbp.fb_interpolate(ctx, cuda(g), [0, 8], cuda(ks),
                               fbp.Params.make(5, 2, 1, 0, 3, flags=fbp.FB_FLAG_TRACKING))
    assert not np.array_equal(plain.cpu().numpy(), track.cpu().numpy())


BLEND_CASES = [
    # N, H, W, k, window, iters, motion
    (7, 40, 44, 5, 5, 2, "affine"),
    (9, 33, 37, 7, 7, 2, "shift"),
    (5, 24, 20, 3, 15, 3, "affine"),           # window wider than the clip
    (6, 21, 26, 9, 3, 2, "affine"),            # chains of one pair
    (4, 18, 19, 5, 5, 0, "shift"),             # no iterations
]


@pytest.mark.parametrize("N,H,W,k,window,iters,motion", BLEND_CASES)
def test_tracking_blend_matches_oracle(fbp, ctx, N, H, W, k, window, iters, motion):
    g, s = synth.small_clip(N, H, W, seed=N * 13 + W, motion=motion)
    p = fbp.Params.make(k, iters, 1, 0, 17, flags=fbp.FB_FLAG_TRACKING)
    out = fbp.fb_blend_window(ctx, cuda(g), cuda(s), window, p).cpu().numpy()
    ref = oracle.blend_window_tracking(g, s, window, k, iters, seed=17)
    assert np.abs(out - ref).max() <= 0.5 / 255
    assert (out == ref).all()


def test_tracking_blend_through_host_buffers(fbp, ctx):
    import torch
    g, s = synth.small_clip(6, 30, 34, seed=2, motion="affine")
    p = fbp.Params.make(5, 2, 1, 0, 8, flags=fbp.FB_FLAG_TRACKING)
    out = fbp.fb_blend_window(ctx, torch.from_numpy(g), torch.from_numpy(s), 5, p).numpy()
    assert (out == oracle.blend_window_tracking(g, s, 5, 5, 2, seed=8)).all()


def test_tracking_beyond_the_pair_budget_is_refused(fbp, ctx):
    # Tracking couples every NNF of the call; a budget that splits the call into chunks
    # is refused before any launch (the plain search runs it chunk by chunk).
    g, s = synth.small_clip(8, 96, 96, seed=6, motion="affine")
    gd, sd = cuda(g), cuda(s)
    p = fbp.Params.make(5, 1, 1, 0, 2, flags=fbp.FB_FLAG_TRACKING)
    ctx.set_pair_budget(1 << 20)     # the smallest budget: one output frame's 6 NNFs (864 KiB)
    try:
        n0 = ctx.launches
        with pytest.raises(fbp.FastBlendError) as ei:
            fbp.fb_blend_window(ctx, gd, sd, 7, p)
        assert ei.value.status == fbp.FB_ERR_UNSUPPORTED and ctx.launches == n0
        plain = fbp.fb_blend_window(ctx, gd, sd, 7, fbp.Params.make(5, 1, 1, 0, 2)).cpu().numpy()
        assert (plain == oracle.blend_window(g, s, 7, 5, 1, seed=2)).all()
    finally:
        ctx.set_pair_budget(0)


def test_tracking_argument_errors(fbp, ctx):
    import torch
    g = torch.zeros((4, 16, 16, 3), dtype=torch.uint8, device="cuda")
    T = fbp.FB_FLAG_TRACKING
    n0 = ctx.launches
    bad = [
        lambda: fbp.fb_interpolate(ctx, g, [0, 3], g[:2], fbp.Params.make(5, 2, 2, flags=T)),
        lambda: fbp.fb_interpolate(ctx, g, [0, 3], g[:2],
                                   fbp.Params.make(5, 2, 1, flags=T | fbp.FB_FLAG_LEARNED_INIT)),
        lambda: fbp.fb_blend_window(ctx, g, g, 3, fbp.Params.make(5, 2, 2, flags=T)),
        lambda: fbp.fb_blend_window(ctx, g, g, 3, fbp.Params.make(5, 2, 1, flags=T | fbp.FB_FLAG_BALANCED,
                                                                  alpha=3)),
        lambda: fbp.fb_blend_window(ctx, g, g, 3, fbp.Params.make(5, 2, 1, flags=T | fbp.FB_FLAG_FAST)),
        lambda: fbp.fb_blend_window(ctx, g, g, 3, fbp.Params.make(5, 2, 1, flags=T | fbp.FB_FLAG_ACCURATE,
                                                                  alpha=3)),
        lambda: fbp.fb_nnf(ctx, g[0], g[1], fbp.Params.make(5, 2, 1, flags=T)),
    ]
    for f in bad:
        with pytest.raises(fbp.FastBlendError) as ei:
            f()
        assert ei.value.status == fbp.FB_ERR_ARG
    assert ctx.launches == n0


@pytest.mark.slow
def test_tracking_interp_1024x576_full_size_sampled_frames(fbp, ctx):
    """The launch configuration bench.py times for tracking_1024x576; the oracle's
    tracking couples whole chains, so the sample is a shorter clip of the same frame size
    whose two chains the oracle finishes in seconds."""
    w = synth.WORKLOADS["interp_1024x576"]
    g, ks = synth.make_clip("interp_1024x576")
    g = np.ascontiguousarray(g[:6])
    ks = np.ascontiguousarray(np.stack([ks[0], ks[0]]))
    keys = [0, 5]
    p = fbp.Params.make(w.patch, 2, 1, 0, w.seed, flags=fbp.FB_FLAG_TRACKING)
    out = fbp.fb_interpolate(ctx, cuda(g), keys, cuda(ks), p).cpu().numpy()
    ref = oracle.interpolate_tracking(g, keys, ks, w.patch, 2, seed=w.seed)
    assert np.abs(out - ref).max() <= 0.5 / 255
    assert (out == ref).all()


@pytest.mark.slow
def test_tracking_blend_512_frame_size(fbp, ctx):
    """The 512x512 frame size of the headline blend at window 15, on a 9-frame clip whose
    tracked chains the oracle finishes in seconds."""
    w = synth.WORKLOADS["blend_512"]
    g, s = synth.make_clip("blend_512")
    g, s = np.ascontiguousarray(g[:9]), np.ascontiguousarray(s[:9])
    p = fbp.Params.make(w.patch, 2, 1, 0, w.seed, flags=fbp.FB_FLAG_TRACKING)
    out = fbp.fb_blend_window(ctx, cuda(g), cuda(s), w.window, p).cpu().numpy()
    ref = oracle.blend_window_tracking(g, s, w.window, w.patch, 2, seed=w.seed)
    assert (out == ref).all()


@pytest.mark.parametrize("H,W", [(9, 32767), (32767, 9)])
def test_tracking_blend_at_the_largest_image_side(fbp, ctx, H, W):
    g = np.stack([synth.noise_pair(H, W, seed=51 + q)[0] for q in range(3)])
    s = np.stack([synth.noise_pair(H, W, seed=61 + q)[1] for q in range(3)])
    p = fbp.Params.make(5, 1, 1, 0, 4, flags=fbp.FB_FLAG_TRACKING)
    out = fbp.fb_blend_window(ctx, cuda(g), cuda(s), 5, p).cpu().numpy()
    assert (out == oracle.blend_window_tracking(g, s, 5, 5, 1, seed=4)).all()
