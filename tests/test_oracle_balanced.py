"""Pins of the oracle's improved-loss ("balanced") mode, Sec. 3.4:
L = alpha ||G_j[F(x)] - G_i[x]||^2 + ||S_j[F(x)] - S^_i[x]||^2, S^_i the rounded remap of
S_j through the field, refreshed at the beginning of every iteration."""
import numpy as np
import pytest

import oracle
import synth


def _true_field(H, W, d):
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return np.stack([np.clip(rr + d[0], 0, H - 1), np.clip(cc + d[1], 0, W - 1)], -1).astype(np.int32)


def test_constant_styles_reduce_to_the_plain_search_scaled_by_alpha():
    # A constant style is its own remap, so the style term vanishes and L = alpha E_plain:
    # the same strict comparisons, the same field.
    g, _ = synth.shift_clip(2, 30, 33, seed=3)
    s = np.full_like(g[0], 93)
    tag = oracle.pair_tag(0, 1)
    Fp, Ep = oracle.nnf(g[0], g[1], 5, 3, seed=7, pair_tag=tag)
    Fb, Eb, S = oracle.nnf_balanced(g[0], g[1], s, 5, 3, 4, seed=7, pair_tag=tag)
    assert (Fb == Fp).all() and (Eb == 4 * Ep.astype(np.int64)).all() and (S == 93).all()
    # alpha = 0: every candidate ties at zero, so the random start is kept
    F0, _ = oracle.nnf(g[0], g[1], 5, 0, seed=7, pair_tag=tag)
    Fz, Ez, _ = oracle.nnf_balanced(g[0], g[1], s, 5, 3, 0, seed=7, pair_tag=tag)
    assert (Fz == F0).all() and (Ez == 0).all()


def test_true_field_is_a_fixed_point_when_styles_follow_the_guides():
    # S = G and a known shift d: the remap of S_j through F* reproduces G_i away from the
    # borders, so both terms vanish there and F* stays.
    g, sh = synth.shift_clip(2, 36, 40, seed=8)
    d = sh[1] - sh[0]
    Fstar = _true_field(36, 40, d)
    F, E, S = oracle.nnf_balanced(g[0], g[1], g[0], 5, 2, 3, seed=2, init=Fstar)
    m = 2 * 2 + int(np.abs(d).max()) + 1
    inner = (slice(m, 36 - m), slice(m, 40 - m))
    assert (E[inner] == 0).all() and (F[inner] == Fstar[inner]).all()
    assert (S[inner] == g[1][inner]).all()


def test_shat_rounds_the_vote_mean_to_nearest():
    # k = 3, every match at the centre (1, 1): the votes for x = (1, 1) are the nine pixels
    # (2, 2) - q, i.e. the whole 3x3 style, so V = its sum.  Sums 94 and 95 over nine votes
    # round to 10 and 11.
    F = np.ones((3, 3, 2), np.int32)
    for total, want in ((94, 10), (95, 11), (9 * 255, 255)):
        s = np.zeros((3, 3, 3), np.uint8)
        vals = np.full(9, total // 9)
        vals[: total % 9] += 1
        s[..., 0] = vals.reshape(3, 3)
        assert oracle.shat(s, F, 3)[1, 1, 0] == want


def test_returned_error_is_the_loss_of_the_returned_field_against_the_returned_shat():
    g, _ = synth.small_clip(2, 20, 23, seed=5, motion="affine")
    _, s = synth.small_clip(2, 20, 23, seed=6, motion="shift")
    for iters in (0, 1, 3):
        F, E, S = oracle.nnf_balanced(g[0], g[1], s[0], 5, iters, 7, seed=3, pair_tag=9)
        for r in range(20):
            for c in range(23):
                want = 7 * oracle.ssd(g[0], g[1], 5, F[r, c], (r, c)) + oracle.ssd(s[0], S, 5, F[r, c], (r, c))
                assert E[r, c] == want, (iters, r, c)


def test_shat_is_refreshed_from_the_field_entering_each_iteration():
    g, _ = synth.small_clip(2, 24, 26, seed=11, motion="affine")
    _, s = synth.small_clip(2, 24, 26, seed=12, motion="shift")
    F1, _, _ = oracle.nnf_balanced(g[0], g[1], s[0], 5, 1, 5, seed=4, pair_tag=3)
    F2, _, S2 = oracle.nnf_balanced(g[0], g[1], s[0], 5, 2, 5, seed=4, pair_tag=3)
    assert (S2 == oracle.shat(s[0], F1, 5)).all()
    assert (F2 != F1).any()


def test_balanced_blend_of_constant_styles_is_constant():
    g, _ = synth.shift_clip(5, 20, 22, seed=2)
    s = np.full(g.shape, 140, np.uint8)
    out = oracle.blend_window_balanced(g, s, 3, 5, 2, 6, seed=1)
    assert np.abs(out - 140 / 255).max() <= 1e-6


def test_balanced_rejects_a_pyramid_and_large_alpha():
    g = np.zeros((2, 8, 8, 3), np.uint8)
    with pytest.raises(ValueError):
        oracle.nnf_balanced(g[0], g[1], g[0], 3, 1, 256)
