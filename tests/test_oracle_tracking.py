"""Pins of the oracle's tracking (Sec. 3.5.1): the NNFs from one keyframe to consecutive
target frames exchange their matches as extra candidates."""
import numpy as np

import oracle
import synth


def _true_field(H, W, d):
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return np.stack([np.clip(rr + d[0], 0, H - 1), np.clip(cc + d[1], 0, W - 1)], -1).astype(np.int32)


def test_runs_of_one_frame_reduce_to_the_plain_interpolation():
    # Keys on every other frame: every chain has one pair, so there is nothing to track.
    g, _ = synth.small_clip(7, 20, 23, seed=3, motion="affine")
    keys = [0, 2, 4, 6]
    ks = synth.lut_styles(g, seed=5)[keys]
    a = oracle.interpolate_tracking(g, keys, ks, 5, 3, seed=4)
    b = oracle.interpolate(g, keys, ks, 5, 3, seed=4)
    assert (a == b).all()


def test_a_neighbour_target_hands_over_its_match():
    # Two identical target frames: the first starts at the true field, the second 12 rows
    # away everywhere.  With the random search limited to radius 1 and every propagation
    # neighbour equally wrong, only the tracking candidate -- the first target's match at
    # the same pixel -- repairs the second target in one iteration.
    H = W = 40
    g, sh = synth.shift_clip(2, H, W, seed=12)
    d = sh[1] - sh[0]
    Fstar = _true_field(H, W, d)
    far = Fstar.copy()
    far[..., 0] = np.clip(far[..., 0] + 12, 0, H - 1)
    tgts = np.stack([g[1], g[1]])
    F, E = oracle.nnf_chain(g[0], tgts, 5, 1, [7, 8], r0=1, seed=2, init=np.stack([Fstar, far]))
    inner = (slice(4, H - 4 - 12), slice(4, W - 4))
    inner_true = np.zeros((H, W), bool)
    inner_true[inner] = True
    for r in range(H):
        for c in range(W):
            ur, uc = r + d[0], c + d[1]
            if not (2 <= ur < H - 2 and 2 <= uc < W - 2):
                inner_true[r, c] = False
    assert inner_true.sum() > 300
    assert (E[1][inner_true] == 0).all() and (F[1][inner_true] == Fstar[inner_true]).all()


def test_tracking_never_raises_a_pixel_error_within_an_iteration():
    # The incumbent stays unless a candidate is strictly better: one more iteration from the
    # same start cannot raise any pixel's error (same streams for iteration 0).
    g, _ = synth.small_clip(5, 18, 21, seed=8, motion="affine")
    tags = [oracle.pair_tag(0, i) for i in range(1, 5)]
    F0, E0 = oracle.nnf_chain(g[0], g[1:], 5, 0, tags, seed=3)
    F1, E1 = oracle.nnf_chain(g[0], g[1:], 5, 1, tags, seed=3)
    assert (E1 <= E0).all() and (E1 < E0).any()


def test_eq9_weights_between_constant_keys_with_tracking():
    # A constant key style remaps to itself, so frame i between keys l and r is exactly
    # ((r - i) c_l + (i - l) c_r) / (r - l); frames outside the key range copy their key.
    N, keys = 11, [2, 9]
    g, _ = synth.small_clip(N, 16, 18, seed=2, motion="affine")
    ks = np.stack([np.full(g.shape[1:], 40, np.uint8), np.full(g.shape[1:], 180, np.uint8)])
    out = oracle.interpolate_tracking(g, keys, ks, 3, 2, seed=1)
    for i in range(N):
        if 2 < i < 9:
            num, den = 9 * ((9 - i) * 40 + (i - 2) * 180), 255 * 9 * 7
        else:
            num, den = 9 * (40 if i <= 2 else 180), 255 * 9
        assert (out[i] == np.float32(num) / np.float32(den)).all(), i


# ----------------------------------------------------------------------------------
# Tracking in the Eq. 2 blend (the optional setting of Sec. 3.5.1)
# ----------------------------------------------------------------------------------
def test_blend_tracking_at_window_3_is_the_plain_blend():
    # Window 3: every source's chains hold one target each, so nothing is tracked.
    g, s = synth.small_clip(6, 19, 22, seed=4, motion="affine")
    a = oracle.blend_window_tracking(g, s, 3, 5, 2, seed=6)
    b = oracle.blend_window(g, s, 3, 5, 2, seed=6)
    assert (a == b).all()


def test_blend_tracking_without_iterations_is_the_plain_blend():
    # Tracking only adds candidates to the iterations: with none, every NNF is its random
    # initialisation and the blend is the plain Eq. 2 mean of the same window.
    g, s = synth.small_clip(8, 17, 20, seed=9, motion="shift")
    for window in (5, 7, 15):
        a = oracle.blend_window_tracking(g, s, window, 3, 0, seed=2)
        b = oracle.blend_window(g, s, window, 3, 0, seed=2)
        assert (a == b).all(), window


def test_blend_tracking_constant_frame_styles_give_the_window_mean():
    # Frame j styled with the constant c_j remaps to c_j under any field, so output frame i
    # is exactly k^2 sum_j c_j / (255 k^2 n_i) over its truncated window.
    N, window, k = 7, 5, 5
    g, _ = synth.small_clip(N, 15, 16, seed=1, motion="affine")
    c = np.array([10, 70, 200, 35, 140, 255, 0])
    s = np.stack([np.full(g.shape[1:], v, np.uint8) for v in c])
    out = oracle.blend_window_tracking(g, s, window, k, 2, seed=5)
    for i in range(N):
        lo, hi = max(0, i - 2), min(N - 1, i + 2)
        num, den = k * k * int(c[lo:hi + 1].sum()), 255 * k * k * (hi - lo + 1)
        assert (out[i] == np.float32(num) / np.float32(den)).all(), i


def test_blend_tracking_chains_are_the_targets_on_each_side_of_the_source():
    # Composition check: output frame i is the Eq. 2 mean of S_i and, for every source j of
    # its window, the remap of S_j by the tracked chain of j's targets on i's side of j.
    N, window, k, iters, seed = 7, 5, 5, 2, 11
    g, s = synth.small_clip(N, 16, 19, seed=3, motion="affine")
    out = oracle.blend_window_tracking(g, s, window, k, iters, seed=seed)
    M = window // 2
    fields = {}
    for j in range(N):
        for lo, hi in ((max(0, j - M), j - 1), (j + 1, min(N - 1, j + M))):
            if lo > hi:
                continue
            tags = [oracle.pair_tag(j, t) for t in range(lo, hi + 1)]
            F, _ = oracle.nnf_chain(g[j], g[lo:hi + 1], k, iters, tags, seed=seed)
            for q, t in enumerate(range(lo, hi + 1)):
                fields[(j, t)] = F[q]
    for i in range(N):
        lo, hi = max(0, i - M), min(N - 1, i + M)
        acc = k * k * s[i].astype(np.uint64)
        for j in range(lo, hi + 1):
            if j != i:
                acc += oracle.remap_sum(s[j], fields[(j, i)], k).astype(np.uint64)
        ref = acc.astype(np.float32) / np.float32(255 * k * k * (hi - lo + 1))
        assert (out[i] == ref).all(), i
    # and the chains do track: the result differs from the independent NNFs
    assert not (out == oracle.blend_window(g, s, window, k, iters, seed=seed)).all()
