"""Pins of the oracle's accurate mode (Sec. 3.4, quality improvement): the window's NNFs
of output frame i computed together under alpha ||G_j[F] - G_i||^2 + ||S_j[F] - Tbar_i||^2,
Tbar_i the rounded mean remapped frame refreshed at the start of every iteration."""
import numpy as np

import oracle
import synth


def test_styles_constant_per_frame_give_the_fields_of_the_plain_search():
    # Each frame's style is one colour, so the style term is the same for every candidate
    # of a pair and every pair's field is that of the plain search (same stream).
    g, _ = synth.small_clip(5, 22, 25, seed=6, motion="affine")
    s = np.stack([np.full(g.shape[1:], 30 + 40 * t, np.uint8) for t in range(5)])
    s[..., 1] = 200 - s[..., 1]
    for i in (0, 2, 4):
        js = [j for j in range(max(0, i - 2), min(4, i + 2) + 1) if j != i]
        for alpha, iters in ((3, 3), (0, 0)):
            out, _, F = oracle.blend_frame_accurate(g, s, 5, i, 5, 3, alpha, seed=7)
            for m, j in enumerate(js):
                # alpha = 0: every candidate ties, so the random start is kept
                Fp, _ = oracle.nnf(g[j], g[i], 5, iters, seed=7, pair_tag=oracle.pair_tag(j, i))
                assert (F[m] == Fp).all(), (i, j, alpha)
            assert (out == oracle.blend_frame(g, s, 5, i, 5, 3, seed=7)).all()


def test_tbar_is_the_rounded_mean_remap_of_the_fields_entering_the_iteration():
    # After one iteration Tbar_i was built from the random start of every pair (j -> i).
    N, H, W, k, window, i = 5, 18, 21, 5, 5, 2
    g, s = synth.small_clip(N, H, W, seed=9, motion="affine")
    _, tbar, _ = oracle.blend_frame_accurate(g, s, window, i, k, 1, 4, seed=3)
    num = (k * k) * s[i].astype(np.int64)
    for j in range(N):
        if j == i:
            continue
        F0, _ = oracle.nnf(g[j], g[i], k, 0, seed=3, pair_tag=oracle.pair_tag(j, i))
        num += oracle.remap_sum(s[j], F0, k).astype(np.int64)
    den = k * k * N
    assert (tbar == (num + den // 2) // den).all()


def test_constant_style_is_constant():
    g, _ = synth.shift_clip(6, 16, 18, seed=2)
    s = np.full(g.shape, 77, np.uint8)
    out = oracle.blend_window_accurate(g, s, 3, 5, 2, 6, seed=1)
    assert np.abs(out - 77 / 255).max() <= 1e-6
