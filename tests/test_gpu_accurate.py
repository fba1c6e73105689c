"""The accurate mode of Sec. 3.4 (FB_FLAG_ACCURATE) on the GPU against the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ACCURATE_ALPHA = 10


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


@pytest.mark.parametrize("N,H,W,k,window,iters,alpha,motion", [
    (5, 40, 44, 5, 3, 2, 10, "affine"), (6, 33, 37, 7, 5, 2, 2, "shift"),
    (4, 24, 20, 3, 7, 1, 0, "affine"), (7, 21, 26, 9, 3, 1, 255, "affine"),
    (3, 18, 19, 5, 5, 0, 4, "shift")])
def test_accurate_blend_matches_oracle(fbp, ctx, N, H, W, k, window, iters, alpha, motion):
    g, s = synth.small_clip(N, H, W, seed=N * 50 + W, motion=motion)
    p = fbp.Params.make(k, iters, 1, 0, 23, flags=fbp.FB_FLAG_ACCURATE, alpha=alpha)
    out = fbp.fb_blend_window(ctx, cuda(g), cuda(s), window, p).cpu().numpy()
    ref = oracle.blend_window_accurate(g, s, window, k, iters, alpha, seed=23)
    assert np.abs(out - ref).max() <= 0.5 / 255
    assert (out == ref).all()


def test_accurate_argument_errors(fbp, ctx):
    g, s = synth.small_clip(4, 20, 20, seed=1)
    gd, sd = cuda(g), cuda(s)
    for p in (fbp.Params.make(5, 1, 2, flags=fbp.FB_FLAG_ACCURATE, alpha=1),
              fbp.Params.make(5, 1, flags=fbp.FB_FLAG_ACCURATE, alpha=300),
              fbp.Params.make(5, 1, flags=fbp.FB_FLAG_ACCURATE | fbp.FB_FLAG_FAST, alpha=1)):
        with pytest.raises(fbp.FastBlendError) as ei:
            fbp.fb_blend_window(ctx, gd, sd, 3, p)
        assert ei.value.status == fbp.FB_ERR_ARG


@pytest.mark.slow
def test_accurate_blend_512_full_size_sampled_frame(fbp, ctx):
    w = synth.WORKLOADS["blend_512"]
    g, s = synth.make_clip("blend_512")
    p = fbp.Params.make(w.patch, w.iters, 1, 0, w.seed, flags=fbp.FB_FLAG_ACCURATE, alpha=ACCURATE_ALPHA)
    out = fbp.fb_blend_window(ctx, cuda(g), cuda(s), w.window, p)
    ref, _, _ = oracle.blend_frame_accurate(g, s, w.window, 31, w.patch, w.iters, ACCURATE_ALPHA, seed=w.seed)
    assert (out[31].cpu().numpy() == ref).all()


@pytest.mark.parametrize("H,W", [(9, 32767), (32767, 9)])
def test_accurate_mode_at_the_largest_image_side(fbp, ctx, H, W):
    g = np.stack([synth.noise_pair(H, W, seed=11 + q)[0] for q in range(3)])
    s = np.stack([synth.noise_pair(H, W, seed=21 + q)[1] for q in range(3)])
    p = fbp.Params.make(5, 1, 1, 0, 2, flags=fbp.FB_FLAG_ACCURATE, alpha=10)
    out = fbp.fb_blend_window(ctx, cuda(g), cuda(s), 3, p).cpu().numpy()
    assert (out == oracle.blend_window_accurate(g, s, 3, 5, 1, 10, seed=2)).all()
