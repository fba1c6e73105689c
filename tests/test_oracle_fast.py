"""Pins of the oracle's fast mode (Sec. 3.4, Algs. 3-5 and the split identity)."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("N,window", [(9, 1), (9, 3), (9, 5), (13, 7), (16, 15), (23, 31)])
def test_constant_style_gives_the_constant_for_every_window_and_frame(N, window):
    # Every remap of a constant frame is that constant, so the result is exact only if the
    # query pieces cover each window [lo, hi] exactly once, every term carries the right
    # k^2 / k^4 weight, and the doubly counted S_i is removed.
    g, _ = synth.shift_clip(N, 14, 15, seed=N + window)
    s = np.full(g.shape, 201, np.uint8)
    out = oracle.blend_window_fast(g, s, window, 3, 1, seed=2)
    assert np.abs(out - np.float32(201 / 255)).max() <= 1e-6


def test_window_one_returns_the_frame():
    g, s = synth.small_clip(4, 12, 13, seed=3, motion="affine")
    out = oracle.blend_window_fast(g, s, 1, 5, 1, seed=1)
    assert (out == s.astype(np.float32) / np.float32(255)).all()


def test_linear_in_the_style_frames():
    g, s1 = synth.small_clip(6, 16, 17, seed=4, motion="affine")
    s2 = synth.lut_styles(g, seed=9)
    half1, half2 = s1 // 2, s2 // 2
    a = oracle.blend_window_fast(g, half1, 5, 3, 2, seed=3)
    b = oracle.blend_window_fast(g, half2, 5, 3, 2, seed=3)
    c = oracle.blend_window_fast(g, (half1 + half2).astype(np.uint8), 5, 3, 2, seed=3)
    assert np.abs(a + b - c).max() <= 2e-6


def test_known_shift_closed_form_on_interior():
    # With exact NNFs every table entry is a sum of shifted styles and its remap shifts
    # it again: (S_a -> S_j) -> S_i = S_a shifted by s_i - s_a, the same closed form as
    # the direct window sum.  Away from the borders (two remaps deep) the result is the
    # mean of the shifted styles.
    N, H, W, k, p, window = 8, 48, 48, 5, 2, 5
    g, sh = synth.shift_clip(N, H, W, seed=43)
    s = synth.colour_matrix_styles(g, seed=43)
    out = oracle.blend_window_fast(g, s, window, k, 10, seed=5)
    M, m = (window - 1) // 2, 2 * p + 2
    good = total = 0
    for i in range(N):
        js = range(max(0, i - M), min(N - 1, i + M) + 1)
        span = max(np.abs(sh[j] - sh[i]).max() for j in js) + max(np.abs(sh[j] - sh[a]).max()
                                                                   for j in js for a in js)
        for r in range(m + span, H - m - span):
            for c in range(m + span, W - m - span):
                num = np.zeros(3, np.int64)
                for j in js:
                    num += s[j, r + sh[i][0] - sh[j][0], c + sh[i][1] - sh[j][1]].astype(np.int64)
                total += 1
                want = (num * k ** 4).astype(np.float64) / (255.0 * k ** 4 * len(js))
                good += int((out[i, r, c] == want.astype(np.float32)).all())
    assert total > 800
    assert good / total >= 0.95
