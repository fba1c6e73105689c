"""Output-frame ranges of one clip on the GPU (the split that spreads a clip over GPUs).

Eq. 2 (Sec. 3.4) gives output frame i from the frames of its window alone, and an
interpolated frame from its keys alone (Sec. 3.5.2).  fb_blend_window_range and
fb_interpolate_range compute a range of output frames from the range plus its halo; each
NNF keeps the random stream of its clip frames.  Here ranges from fb_shard_plan, run one
after the other on one GPU and stitched together, must equal the whole-clip call bit for
bit, and sampled frames must equal the CPU oracle (0.5/255; in practice bit-exact).
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


def stitched_blend(fbp, ctx, g, s, window, p, n_shards, on_host=False):
    import torch
    N = g.shape[0]
    parts = []
    for r in range(n_shards):
        pl = fbp.fb_shard_plan(N, window, n_shards, r)
        lo, n_in = pl["frame_base"], pl["n_in"]
        gs, ss = g[lo:lo + n_in], s[lo:lo + n_in]
        if on_host:
            gt, st = torch.from_numpy(np.ascontiguousarray(gs)), torch.from_numpy(np.ascontiguousarray(ss))
        else:
            gt, st = cuda(gs), cuda(ss)
        o = fbp.fb_blend_window_range(ctx, gt, st, window, p, N, lo, pl["out_first"], pl["n_out"])
        parts.append(o.numpy() if on_host else host(o))
    return np.concatenate(parts, axis=0)


@pytest.mark.parametrize("N,H,W,k,window,iters,n_shards,levels", [
    (9, 48, 56, 5, 5, 3, 2, 1),
    (9, 48, 56, 5, 5, 3, 3, 1),
    (12, 40, 37, 3, 7, 2, 4, 1),
    (7, 33, 45, 7, 3, 2, 7, 1),
    (10, 64, 48, 5, 9, 2, 3, 2),
    (6, 30, 31, 5, 31, 1, 2, 1),
])
def test_blend_ranges_stitch_to_the_whole_clip(fbp, ctx, N, H, W, k, window, iters, n_shards, levels):
    g, s = synth.small_clip(N, H, W, seed=4100 + N * 7 + k)
    p = fbp.Params.make(k, iters, levels, 0, 97)
    whole = host(fbp.fb_blend_window(ctx, cuda(g), cuda(s), window, p))
    got = stitched_blend(fbp, ctx, g, s, window, p, n_shards)
    assert np.array_equal(got, whole)
    # a frame at a shard boundary against the oracle
    b = fbp.fb_shard_plan(N, window, n_shards, n_shards - 1)["out_first"]
    for i in sorted({b - 1, b}):
        ref = oracle.blend_frame(g, s, window, i, k, iters, levels, seed=97)
        assert np.abs(got[i] - ref).max() <= TOL


def test_blend_range_from_host_buffers(fbp, ctx):
    g, s = synth.small_clip(8, 40, 44, seed=4177)
    p = fbp.Params.make(5, 3, 1, 0, 5)
    whole = host(fbp.fb_blend_window(ctx, cuda(g), cuda(s), 5, p))
    got = stitched_blend(fbp, ctx, g, s, 5, p, 3, on_host=True)
    assert np.array_equal(got, whole)


@pytest.mark.parametrize("flag", ["balanced", "accurate"])
def test_two_image_loss_ranges(fbp, ctx, flag):
    """The improved and accurate losses couple only NNFs of the same output frame (its S^
    per pair, its mean frame per output frame), so they shard like the plain loss."""
    g, s = synth.small_clip(8, 36, 40, seed=4199, motion="affine")
    f = fbp.FB_FLAG_BALANCED if flag == "balanced" else fbp.FB_FLAG_ACCURATE
    p = fbp.Params.make(5, 3, 1, 0, 11, flags=f, alpha=10)
    whole = host(fbp.fb_blend_window(ctx, cuda(g), cuda(s), 5, p))
    got = stitched_blend(fbp, ctx, g, s, 5, p, 3)
    assert np.array_equal(got, whole)


@pytest.mark.parametrize("keys,flags", [((0, 11), 0), ((0, 11), 0x40), ((3, 7), 0x40), ((5,), 0)])
def test_interpolation_ranges_stitch_to_the_whole_clip(fbp, ctx, keys, flags):
    N = 12
    g, s = synth.small_clip(N, 40, 48, seed=4233)
    ks = np.ascontiguousarray(s[list(keys)])
    p = fbp.Params.make(5, 3, 1, 0, 23, flags=flags, alpha=10)
    whole = host(fbp.fb_interpolate(ctx, cuda(g), keys, cuda(ks), p))
    parts = []
    for r in range(4):
        pl = fbp.fb_shard_plan(N, 0, 4, r)
        parts.append(host(fbp.fb_interpolate_range(ctx, cuda(g), keys, cuda(ks), p, pl["out_first"],
                                                   pl["n_out"])))
    got = np.concatenate(parts, axis=0)
    assert np.array_equal(got, whole)
    if flags == 0:
        i = fbp.fb_shard_plan(N, 0, 4, 2)["out_first"]
        ref = oracle.interpolate_frame(g, list(keys), ks, i, 5, 3, seed=23)
        assert np.abs(got[i] - ref).max() <= TOL


def test_range_argument_errors(fbp, ctx):
    import paper_2311_09265_b300 as m
    g, s = synth.small_clip(8, 32, 32, seed=4300)
    p = fbp.Params.make(5, 2, 1, 0, 1)
    # output frames [3, 5) with window 5 need inputs [1, 7); frames [2, 7) are one short
    with pytest.raises(m.FastBlendError) as e:
        fbp.fb_blend_window_range(ctx, cuda(g[2:7]), cuda(s[2:7]), 5, p, 8, 2, 3, 2)
    assert e.value.status == m.FB_ERR_ARG
    ok = fbp.fb_blend_window_range(ctx, cuda(g[1:7]), cuda(s[1:7]), 5, p, 8, 1, 3, 2)
    whole = host(fbp.fb_blend_window(ctx, cuda(g), cuda(s), 5, p))
    assert np.array_equal(host(ok), whole[3:5])
    for flags in (m.FB_FLAG_TRACKING, m.FB_FLAG_FAST):
        q = fbp.Params.make(5, 2, 1, 0, 1, flags=flags)
        with pytest.raises(m.FastBlendError) as e:
            fbp.fb_blend_window_range(ctx, cuda(g), cuda(s), 5, q, 8, 0, 0, 8)
        assert e.value.status == m.FB_ERR_UNSUPPORTED


def test_headline_clip_in_two_shards(fbp, ctx):
    """The 60-frame 512x512 clip (window 15, k = 5, 6 iterations) split in two as on two
    GPUs: stitched, bit-identical to the whole call; the frames on either side of the cut
    equal the oracle's."""
    g, s = synth.make_clip("blend_512")
    w = synth.WORKLOADS["blend_512"]
    p = fbp.Params.make(w.patch, w.iters, 1, 0, w.seed)
    whole = host(fbp.fb_blend_window(ctx, cuda(g), cuda(s), w.window, p))
    got = stitched_blend(fbp, ctx, g, s, w.window, p, 2)
    assert np.array_equal(got, whole)
    b = fbp.fb_shard_plan(w.N, w.window, 2, 1)["out_first"]
    ref = oracle.blend_frame(g, s, w.window, b, w.patch, w.iters, seed=w.seed)
    assert np.abs(got[b] - ref).max() <= TOL
