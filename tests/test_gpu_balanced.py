"""The improved loss of Sec. 3.4 ("balanced mode") on the GPU against the oracle: fields,
losses and S^ bit for bit, blends bit for bit, and the argument checks."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

BALANCED_ALPHA = 10   # the guide weight the balanced benchmark uses


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


NNF_CASES = [
    # H, W, k, iters, alpha, motion
    (37, 53, 5, 0, 7, "affine"),
    (37, 53, 5, 1, 7, "affine"),
    (48, 48, 5, 3, 10, "shift"),
    (41, 45, 7, 2, 3, "affine"),
    (30, 33, 3, 2, 0, "shift"),
    (29, 31, 9, 2, 255, "affine"),
    (5, 300, 5, 2, 10, "affine"),
]


@pytest.mark.parametrize("H,W,k,iters,alpha,motion", NNF_CASES)
def test_nnf_balanced_bit_exact(fbp, ctx, H, W, k, iters, alpha, motion):
    g, s = synth.small_clip(2, H, W, seed=H * 7 + W, motion=motion)
    tag = oracle.pair_tag(0, 1)
    p = fbp.Params.make(k, iters, 1, 0, 11, tag, alpha=alpha)
    F, E, S = fbp.fb_nnf_balanced(ctx, cuda(g[0]), cuda(g[1]), cuda(s[0]), p)
    Fo, Eo, So = oracle.nnf_balanced(g[0], g[1], s[0], k, iters, alpha, seed=11, pair_tag=tag)
    assert (F.cpu().numpy() == Fo).all()
    assert (E.cpu().numpy().view(np.uint32) == Eo).all()
    assert (S.cpu().numpy() == So).all()


def test_nnf_balanced_with_user_init(fbp, ctx):
    g, s = synth.small_clip(2, 40, 44, seed=5, motion="affine")
    rng = np.random.default_rng(1)
    init = np.stack([rng.integers(-3, 43, (40, 44)), rng.integers(-3, 47, (40, 44))], -1).astype(np.int32)
    p = fbp.Params.make(5, 2, 1, 0, 3, 9, alpha=4)
    F, E, S = fbp.fb_nnf_balanced(ctx, cuda(g[0]), cuda(g[1]), cuda(s[0]), p, init_nnf=cuda(init))
    Fo, Eo, So = oracle.nnf_balanced(g[0], g[1], s[0], 5, 2, 4, seed=3, pair_tag=9, init=init)
    assert (F.cpu().numpy() == Fo).all() and (E.cpu().numpy().view(np.uint32) == Eo).all()


@pytest.mark.parametrize("N,H,W,k,window,iters,alpha", [(5, 40, 44, 5, 3, 2, 10), (4, 33, 37, 7, 5, 2, 2),
                                                        (3, 24, 20, 3, 3, 1, 0)])
def test_balanced_blend_matches_oracle(fbp, ctx, N, H, W, k, window, iters, alpha):
    g, s = synth.small_clip(N, H, W, seed=N * 100 + H, motion="affine")
    p = fbp.Params.make(k, iters, 1, 0, 21, flags=fbp.FB_FLAG_BALANCED, alpha=alpha)
    out = fbp.fb_blend_window(ctx, cuda(g), cuda(s), window, p).cpu().numpy()
    ref = oracle.blend_window_balanced(g, s, window, k, iters, alpha, seed=21)
    assert np.abs(out - ref).max() <= 0.5 / 255
    assert (out == ref).all()


def test_balanced_argument_errors(fbp, ctx):
    import torch
    g, s = synth.small_clip(3, 20, 20, seed=1)
    gd, sd = cuda(g), cuda(s)
    bad = [fbp.Params.make(5, 1, 2, 0, 0, flags=fbp.FB_FLAG_BALANCED, alpha=1),
           fbp.Params.make(5, 1, 1, 0, 0, flags=fbp.FB_FLAG_BALANCED, alpha=256),
           fbp.Params.make(5, 1, 1, 0, 0, flags=fbp.FB_FLAG_BALANCED | fbp.FB_FLAG_LEARNED_INIT, alpha=1)]
    for p in bad:
        with pytest.raises(fbp.FastBlendError) as ei:
            fbp.fb_blend_window(ctx, gd, sd, 3, p)
        assert ei.value.status == fbp.FB_ERR_ARG
    with pytest.raises(fbp.FastBlendError):
        fbp.fb_nnf(ctx, gd[0], gd[1], fbp.Params.make(5, 1, flags=fbp.FB_FLAG_BALANCED, alpha=1))
    with pytest.raises(fbp.FastBlendError):
        fbp.fb_interpolate(ctx, gd, [0, 2], sd[[0, 2]].contiguous(),
                           fbp.Params.make(5, 1, flags=fbp.FB_FLAG_BALANCED, alpha=1))
    with pytest.raises(fbp.FastBlendError):
        fbp.fb_nnf_balanced(ctx, gd[0], gd[1], sd[0], fbp.Params.make(5, 1, 2, alpha=1))
    torch.cuda.synchronize()


@pytest.mark.slow
def test_balanced_blend_512_full_size_sampled_frame(fbp, ctx):
    """The headline clip in the balanced benchmark's configuration, one interior frame
    against the oracle bit for bit."""
    w = synth.WORKLOADS["blend_512"]
    g, s = synth.make_clip("blend_512")
    p = fbp.Params.make(w.patch, w.iters, 1, 0, w.seed, flags=fbp.FB_FLAG_BALANCED, alpha=BALANCED_ALPHA)
    out = fbp.fb_blend_window(ctx, cuda(g), cuda(s), w.window, p)
    i = 31
    ref = oracle.blend_frame_balanced(g, s, w.window, i, w.patch, w.iters, BALANCED_ALPHA, seed=w.seed)
    assert (out[i].cpu().numpy() == ref).all()


@pytest.mark.parametrize("H,W", [(9, 32767), (32767, 9)])
def test_balanced_at_the_largest_image_side(fbp, ctx, H, W):
    """Improved loss with packed field entries at the largest supported side: fields,
    losses and S^ of one pair, and a short blend, bit-exact."""
    g0, g1 = synth.noise_pair(H, W, seed=5)
    s0 = synth.noise_pair(H, W, seed=6)[0]
    p = fbp.Params.make(5, 1, 1, 0, 3, pair_tag=17, alpha=10)
    F, E, S = fbp.fb_nnf_balanced(ctx, cuda(g0), cuda(g1), cuda(s0), p)
    Fo, Eo, So = oracle.nnf_balanced(g0, g1, s0, 5, 1, 10, seed=3, pair_tag=17)
    assert (F.cpu().numpy() == Fo).all() and (E.cpu().numpy().view(np.uint32) == Eo).all()
    assert (S.cpu().numpy() == So).all()
    g = np.stack([g0, g1, synth.noise_pair(H, W, seed=7)[0]])
    s = np.stack([s0, synth.noise_pair(H, W, seed=8)[0], synth.noise_pair(H, W, seed=9)[0]])
    pb = fbp.Params.make(5, 1, 1, 0, 3, flags=fbp.FB_FLAG_BALANCED, alpha=10)
    out = fbp.fb_blend_window(ctx, cuda(g), cuda(s), 3, pb).cpu().numpy()
    assert (out == oracle.blend_window_balanced(g, s, 3, 5, 1, 10, seed=3)).all()
