"""Alignment loss of Sec. 3.5.2 (Eq. 10, FB_FLAG_ALIGN of fb_interpolate), with and without
the tracking of Sec. 3.5.1, on the GPU against the oracle."""
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


ALIGN_CASES = [
    # N, H, W, k, keys, iters, alpha, tracking, motion
    (9, 40, 44, 5, (0, 8), 3, 10, False, "affine"),
    (9, 40, 44, 5, (0, 8), 3, 10, True, "affine"),
    (10, 33, 37, 7, (2, 5, 7), 2, 0, True, "shift"),     # inner keys, frames outside them
    (8, 24, 20, 3, (1, 6), 2, 255, False, "affine"),
    (7, 21, 26, 9, (0, 6), 1, 4, True, "affine"),
    (6, 28, 31, 5, (0, 1, 2, 5), 2, 7, False, "shift"),  # adjacent keys: no frame between
    (6, 30, 30, 5, (3,), 2, 10, True, "affine"),         # one key: no partner anywhere
    (5, 18, 19, 5, (0, 4), 0, 10, False, "affine"),      # no iterations
]


@pytest.mark.parametrize("N,H,W,k,keys,iters,alpha,tracking,motion", ALIGN_CASES)
def test_aligned_interpolation_matches_oracle(fbp, ctx, N, H, W, k, keys, iters, alpha, tracking, motion):
    g, s = synth.small_clip(N, H, W, seed=N * 11 + W, motion=motion)
    ks = np.ascontiguousarray(s[list(keys)])
    flags = fbp.FB_FLAG_ALIGN | (fbp.FB_FLAG_TRACKING if tracking else 0)
    p = fbp.Params.make(k, iters, 1, 0, 41, flags=flags, alpha=alpha)
    out = fbp.fb_interpolate(ctx, cuda(g), list(keys), cuda(ks), p).cpu().numpy()
    ref = oracle.interpolate_aligned(g, list(keys), ks, k, iters, alpha, tracking=tracking, seed=41)
    assert np.abs(out - ref).max() <= 0.5 / 255
    assert (out == ref).all()


SEGMENT_CASES = [
    # n, H, W, k, iters, alpha, align, tracking, with_init
    (3, 30, 34, 5, 3, 10, True, False, False),
    (4, 27, 25, 5, 2, 10, True, True, False),
    (2, 22, 31, 7, 2, 0, True, True, True),
    (3, 19, 20, 3, 1, 255, True, False, True),
    (2, 21, 23, 9, 2, 6, True, True, False),
    (3, 24, 26, 5, 2, 0, False, True, False),     # tracked chains, plain loss
    (2, 20, 21, 5, 2, 0, False, False, True),     # independent plain fields
]


@pytest.mark.parametrize("n,H,W,k,iters,alpha,align,tracking,with_init", SEGMENT_CASES)
def test_segment_fields_match_oracle(fbp, ctx, n, H, W, k, iters, alpha, align, tracking, with_init):
    """Field-level parity: every NNF and loss of a segment, bit-exact."""
    g, s = synth.small_clip(n + 2, H, W, seed=n * 31 + H, motion="affine")
    ks = np.ascontiguousarray(s[[0, n + 1]])
    tl = [oracle.pair_tag(0, q) for q in range(1, n + 1)]
    tr = [oracle.pair_tag(n + 1, q) for q in range(1, n + 1)]
    init = None
    if with_init:
        rng = np.random.default_rng(n + H)
        init = np.stack([rng.integers(-3, H + 3, (2 * n, H, W)), rng.integers(-3, W + 3, (2 * n, H, W))],
                        -1).astype(np.int32)
    flags = (fbp.FB_FLAG_ALIGN if align else 0) | (fbp.FB_FLAG_TRACKING if tracking else 0)
    p = fbp.Params.make(k, iters, 1, 0, 19, flags=flags, alpha=alpha)
    F, E = fbp.fb_nnf_segment(ctx, cuda(g), cuda(ks), p, init=None if init is None else cuda(init))
    F, E = F.cpu().numpy(), E.cpu().numpy().view(np.uint32)
    if align:
        Fo, Eo = oracle.nnf_segment(g[0], g[n + 1], ks[0], ks[1], g[1:n + 1], k, iters, alpha, tl, tr,
                                    tracking=tracking, seed=19,
                                    init=None if init is None else init.reshape(2, n, H, W, 2))
        Fo, Eo = Fo.reshape(2 * n, H, W, 2), Eo.reshape(2 * n, H, W)
    else:
        Fs, Es = [], []
        for side, src in enumerate((0, n + 1)):
            tags = tl if side == 0 else tr
            side_init = None if init is None else init[side * n:(side + 1) * n]
            if tracking:
                a, b = oracle.nnf_chain(g[src], g[1:n + 1], k, iters, tags, seed=19, init=side_init)
                Fs.append(a)
                Es.append(b)
            else:
                for q in range(n):
                    a, b = oracle.nnf(g[src], g[1 + q], k, iters, seed=19, pair_tag=tags[q],
                                      init=None if side_init is None else side_init[q])
                    Fs.append(a[None])
                    Es.append(b[None])
        Fo, Eo = np.concatenate(Fs), np.concatenate(Es)
    assert (F == Fo).all()
    assert (E == Eo).all()


def test_segment_argument_errors(fbp, ctx):
    import torch
    g = torch.zeros((4, 16, 16, 3), dtype=torch.uint8, device="cuda")
    A = fbp.FB_FLAG_ALIGN
    n0 = ctx.launches
    for p in (fbp.Params.make(5, 0, 1, flags=A, alpha=1),                         # loss needs an iteration
              fbp.Params.make(5, 2, 2, flags=A, alpha=1),                         # levels
              fbp.Params.make(5, 2, 1, flags=A | fbp.FB_FLAG_BALANCED, alpha=1),  # other modes
              fbp.Params.make(5, 2, 1, flags=A, alpha=300)):
        with pytest.raises(fbp.FastBlendError) as ei:
            fbp.fb_nnf_segment(ctx, g, g[:2], p)
        assert ei.value.status == fbp.FB_ERR_ARG
    with pytest.raises(fbp.FastBlendError) as ei:
        fbp.fb_nnf_segment(ctx, g[:2], g[:2], fbp.Params.make(5, 2))             # no frame between
    assert ei.value.status == fbp.FB_ERR_ARG
    assert ctx.launches == n0


def test_aligned_interpolation_through_host_buffers(fbp, ctx):
    import torch
    g, s = synth.small_clip(7, 26, 29, seed=3, motion="affine")
    ks = np.ascontiguousarray(s[[0, 6]])
    p = fbp.Params.make(5, 2, 1, 0, 5, flags=fbp.FB_FLAG_ALIGN, alpha=10)
    out = fbp.fb_interpolate(ctx, torch.from_numpy(g), [0, 6], torch.from_numpy(ks), p).numpy()
    assert (out == oracle.interpolate_aligned(g, [0, 6], ks, 5, 2, 10, seed=5)).all()


def test_aligned_interpolation_split_into_chunks(fbp, ctx):
    # Without tracking, the coupled pairs of a frame stay in one chunk of any budget.
    g, s = synth.small_clip(8, 96, 96, seed=9, motion="affine")
    ks = np.ascontiguousarray(s[[0, 7]])
    p = fbp.Params.make(5, 2, 1, 0, 5, flags=fbp.FB_FLAG_ALIGN, alpha=10)
    ctx.set_pair_budget(1 << 20)     # 7 pairs of 96x96: chunks of 3 frames (6 coupled pairs)
    try:
        out = fbp.fb_interpolate(ctx, cuda(g), [0, 7], cuda(ks), p).cpu().numpy()
    finally:
        ctx.set_pair_budget(0)
    assert (out == oracle.interpolate_aligned(g, [0, 7], ks, 5, 2, 10, seed=5)).all()


def test_align_argument_errors(fbp, ctx):
    import torch
    g = torch.zeros((4, 16, 16, 3), dtype=torch.uint8, device="cuda")
    A = fbp.FB_FLAG_ALIGN
    n0 = ctx.launches
    bad = [
        lambda: fbp.fb_interpolate(ctx, g, [0, 3], g[:2], fbp.Params.make(5, 2, 2, flags=A, alpha=1)),
        lambda: fbp.fb_interpolate(ctx, g, [0, 3], g[:2], fbp.Params.make(5, 2, 1, flags=A, alpha=256)),
        lambda: fbp.fb_interpolate(ctx, g, [0, 3], g[:2],
                                   fbp.Params.make(5, 2, 1, flags=A | fbp.FB_FLAG_REPORT_ENERGY, alpha=1)),
        lambda: fbp.fb_interpolate(ctx, g, [0, 3], g[:2],
                                   fbp.Params.make(5, 2, 1, flags=A | fbp.FB_FLAG_LEARNED_INIT, alpha=1)),
        lambda: fbp.fb_interpolate(ctx, g, [0, 3], g[:2],
                                   fbp.Params.make(5, 2, 1, flags=A | fbp.FB_FLAG_BALANCED, alpha=1)),
        lambda: fbp.fb_blend_window(ctx, g, g, 3, fbp.Params.make(5, 2, 1, flags=A, alpha=1)),
        lambda: fbp.fb_nnf(ctx, g[0], g[1], fbp.Params.make(5, 2, 1, flags=A, alpha=1)),
    ]
    for f in bad:
        with pytest.raises(fbp.FastBlendError) as ei:
            f()
        assert ei.value.status == fbp.FB_ERR_ARG
    assert ctx.launches == n0


@pytest.mark.slow
def test_aligned_tracking_interp_1024x576_frame_size(fbp, ctx):
    """The 576x1024 frames of the interpolation workload with tracking and alignment on
    (the launch configuration bench.py times for aligned_1024x576), on a 6-frame clip whose
    coupled chains the oracle finishes in seconds."""
    w = synth.WORKLOADS["interp_1024x576"]
    g, ks = synth.make_clip("interp_1024x576")
    g = np.ascontiguousarray(g[:6])
    ks = np.ascontiguousarray(np.stack([ks[0], ks[1]]))
    keys = [0, 5]
    p = fbp.Params.make(w.patch, 2, 1, 0, w.seed, flags=fbp.FB_FLAG_ALIGN | fbp.FB_FLAG_TRACKING,
                        alpha=10)
    out = fbp.fb_interpolate(ctx, cuda(g), keys, cuda(ks), p).cpu().numpy()
    ref = oracle.interpolate_aligned(g, keys, ks, w.patch, 2, 10, tracking=True, seed=w.seed)
    assert (out == ref).all()


@pytest.mark.parametrize("H,W", [(9, 32767), (32767, 9)])
def test_segment_at_the_largest_image_side(fbp, ctx, H, W):
    """Coupled and tracked fields with packed (row << 16 | col) entries at the largest
    supported side: every field and loss bit-exact."""
    g = np.stack([synth.noise_pair(H, W, seed=31 + q)[0] for q in range(4)])
    ks = np.stack([synth.noise_pair(H, W, seed=71)[1], synth.noise_pair(H, W, seed=72)[1]])
    n = 2
    p = fbp.Params.make(5, 1, 1, 0, 9, flags=fbp.FB_FLAG_ALIGN | fbp.FB_FLAG_TRACKING, alpha=10)
    F, E = fbp.fb_nnf_segment(ctx, cuda(g), cuda(ks), p)
    F, E = F.cpu().numpy(), E.cpu().numpy().view(np.uint32)
    tl = [oracle.pair_tag(0, q) for q in range(1, n + 1)]
    tr = [oracle.pair_tag(n + 1, q) for q in range(1, n + 1)]
    Fo, Eo = oracle.nnf_segment(g[0], g[n + 1], ks[0], ks[1], g[1:n + 1], 5, 1, 10, tl, tr,
                                tracking=True, seed=9)
    assert (F == Fo.reshape(2 * n, H, W, 2)).all() and (E == Eo.reshape(2 * n, H, W)).all()
    assert F[..., 0].max() <= H - 1 and F[..., 1].max() <= W - 1
