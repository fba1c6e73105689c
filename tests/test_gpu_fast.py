"""The fast mode of Sec. 3.4 (FB_FLAG_FAST) on the GPU against the oracle, bit for bit."""
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


CASES = [
    # N, H, W, k, window, iters, levels, motion
    (9, 40, 44, 5, 5, 2, 1, "affine"),
    (13, 33, 37, 3, 7, 2, 1, "shift"),
    (16, 24, 28, 7, 15, 1, 1, "affine"),
    (23, 20, 21, 5, 31, 1, 1, "shift"),
    (6, 30, 33, 5, 3, 2, 2, "affine"),
    (5, 18, 19, 9, 5, 1, 1, "affine"),
    (7, 16, 17, 5, 1, 1, 1, "affine"),
]


@pytest.mark.parametrize("N,H,W,k,window,iters,levels,motion", CASES)
def test_fast_blend_matches_oracle(fbp, ctx, N, H, W, k, window, iters, levels, motion):
    g, s = synth.small_clip(N, H, W, seed=N * 31 + window, motion=motion)
    p = fbp.Params.make(k, iters, levels, 0, 17, flags=fbp.FB_FLAG_FAST)
    out = fbp.fb_blend_window(ctx, cuda(g), cuda(s), window, p).cpu().numpy()
    o = oracle.params(k, iters, levels, 0, 17)
    ref = np.stack([_oracle_frame(g, s, window, i, o) for i in range(N)])
    assert np.abs(out - ref).max() <= 0.5 / 255
    assert (out == ref).all()


def _oracle_frame(g, s, window, i, o):
    import ctypes
    N, H, W = g.shape[:3]
    out = np.zeros((H, W, 3), np.float32)
    rc = oracle.lib().fbref_blend_frame_fast(g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                             s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                             N, H, W, window, ctypes.byref(o), i,
                                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    assert rc == 0
    return out


def test_fast_blend_host_buffers_equal_device_buffers(fbp, ctx):
    import torch
    g, s = synth.small_clip(8, 24, 26, seed=3, motion="affine")
    p = fbp.Params.make(5, 2, 1, 0, 4, flags=fbp.FB_FLAG_FAST)
    a = fbp.fb_blend_window(ctx, cuda(g), cuda(s), 5, p).cpu().numpy()
    out = torch.empty((8, 24, 26, 3), dtype=torch.float32).pin_memory()
    fbp.fb_blend_window(ctx, torch.tensor(g).pin_memory(), torch.tensor(s).pin_memory(), 5, p, out=out)
    assert (out.numpy() == a).all()


def test_fast_flag_argument_errors(fbp, ctx):
    g, s = synth.small_clip(4, 20, 20, seed=1)
    gd, sd = cuda(g), cuda(s)
    for flags in (fbp.FB_FLAG_FAST | fbp.FB_FLAG_BALANCED, fbp.FB_FLAG_FAST | fbp.FB_FLAG_LEARNED_INIT):
        with pytest.raises(fbp.FastBlendError) as ei:
            fbp.fb_blend_window(ctx, gd, sd, 3, fbp.Params.make(5, 1, flags=flags, alpha=1))
        assert ei.value.status == fbp.FB_ERR_ARG
    with pytest.raises(fbp.FastBlendError):
        fbp.fb_nnf(ctx, gd[0], gd[1], fbp.Params.make(5, 1, flags=fbp.FB_FLAG_FAST))
    with pytest.raises(fbp.FastBlendError):
        fbp.fb_interpolate(ctx, gd, [0, 3], sd[[0, 3]].contiguous(), fbp.Params.make(5, 1, flags=fbp.FB_FLAG_FAST))


@pytest.mark.slow
def test_fast_blend_512_full_size_sampled_frame(fbp, ctx):
    """The headline clip in fast mode, one interior frame against the oracle bit for bit."""
    w = synth.WORKLOADS["blend_512"]
    g, s = synth.make_clip("blend_512")
    p = fbp.Params.make(w.patch, w.iters, 1, 0, w.seed, flags=fbp.FB_FLAG_FAST)
    out = fbp.fb_blend_window(ctx, cuda(g), cuda(s), w.window, p)
    ref = oracle.blend_frame_fast(g, s, w.window, 31, w.patch, w.iters, seed=w.seed)
    assert (out[31].cpu().numpy() == ref).all()


@pytest.mark.parametrize("H,W", [(9, 32767), (32767, 9)])
def test_fast_mode_at_the_largest_image_side(fbp, ctx, H, W):
    g = np.stack([synth.noise_pair(H, W, seed=81 + q)[0] for q in range(5)])
    s = np.stack([synth.noise_pair(H, W, seed=91 + q)[1] for q in range(5)])
    p = fbp.Params.make(5, 1, 1, 0, 6, flags=fbp.FB_FLAG_FAST)
    out = fbp.fb_blend_window(ctx, cuda(g), cuda(s), 5, p).cpu().numpy()
    assert (out == oracle.blend_window_fast(g, s, 5, 5, 1, seed=6)).all()
