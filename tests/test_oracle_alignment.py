"""Pins of the oracle's alignment loss of Sec. 3.5.2 (Eq. 10): the NNFs from the two keys
l < r to each frame between them are coupled through a patch difference of the two
keyframes' styles at their current matches."""
import numpy as np
import pytest

import oracle
import synth


def _ssd(a, b, k, ar, ac, br, bc):
    """Eq. 1 by brute force: the k x k RGB patches of a at (ar, ac) and b at (br, bc), each
    clamped to its own image."""
    H, W = a.shape[:2]
    P = k // 2
    tot = 0
    for dy in range(-P, P + 1):
        for dx in range(-P, P + 1):
            pa = a[min(max(ar + dy, 0), H - 1), min(max(ac + dx, 0), W - 1)].astype(np.int64)
            pb = b[min(max(br + dy, 0), H - 1), min(max(bc + dx, 0), W - 1)].astype(np.int64)
            tot += int(((pa - pb) ** 2).sum())
    return tot


def _segment(N=6, H=18, W=21, seed=4, motion="affine"):
    g, s = synth.small_clip(N, H, W, seed=seed, motion=motion)
    l, r = 0, N - 1
    tl = [oracle.pair_tag(l, i) for i in range(l + 1, r)]
    tr = [oracle.pair_tag(r, i) for i in range(l + 1, r)]
    return g, s, l, r, tl, tr


@pytest.mark.parametrize("alpha", [1, 7, 255])
@pytest.mark.parametrize("tracking", [False, True])
def test_constant_key_styles_reduce_to_the_plain_search(alpha, tracking):
    # Constant keyframe styles make the pairwise term the same constant 3 k^2 (c_l - c_r)^2
    # for every candidate, so with alpha >= 1 the comparisons are those of Eq. 1 scaled by
    # alpha: the fields are the independent plain fields (tracked chains with tracking).
    g, _, l, r, tl, tr = _segment()
    k, iters = 5, 3
    sl = np.full(g.shape[1:], 30, np.uint8)
    sr = np.full(g.shape[1:], 200, np.uint8)
    F, E = oracle.nnf_segment(g[l], g[r], sl, sr, g[l + 1:r], k, iters, alpha, tl, tr,
                              tracking=tracking, seed=9)
    const = 3 * k * k * (200 - 30) ** 2
    for side, (src, tags) in enumerate(((g[l], tl), (g[r], tr))):
        if tracking:
            Fp, Ep = oracle.nnf_chain(src, g[l + 1:r], k, iters, tags, seed=9)
        else:
            pairs = [oracle.nnf(src, g[l + 1 + q], k, iters, seed=9, pair_tag=tags[q])
                     for q in range(len(tags))]
            Fp, Ep = np.stack([a for a, _ in pairs]), np.stack([b for _, b in pairs])
        assert (F[side] == Fp).all()
        assert (E[side].astype(np.int64) == alpha * Ep.astype(np.int64) + const).all()


def test_zero_alpha_and_constant_styles_keep_the_initial_fields():
    # alpha = 0 with constant styles: every candidate ties the incumbent, none is accepted.
    g, _, l, r, tl, tr = _segment(N=5)
    init = np.stack([np.stack([oracle.nnf(g[src], g[i], 3, 0, seed=2, pair_tag=oracle.pair_tag(src, i))[0]
                               for i in range(l + 1, r)]) for src in (l, r)])
    c = np.full(g.shape[1:], 77, np.uint8)
    F, E = oracle.nnf_segment(g[l], g[r], c, c, g[l + 1:r], 3, 4, 0, tl, tr, seed=2, init=init)
    assert (F == init).all() and (E == 0).all()


def test_identical_fields_and_styles_have_zero_pairwise_error():
    # Both keys styled alike and both fields equal: with alpha = 0 each pair's incumbent
    # already has loss 0, which no candidate beats.
    g, s, l, r, tl, tr = _segment(N=5)
    rng = np.random.default_rng(5)
    n, H, W = r - l - 1, g.shape[1], g.shape[2]
    A = np.stack([rng.integers(0, H, (n, H, W)), rng.integers(0, W, (n, H, W))], -1).astype(np.int32)
    F, E = oracle.nnf_segment(g[l], g[r], s[2], s[2], g[l + 1:r], 5, 3, 0, tl, tr, seed=1,
                              init=np.stack([A, A]))
    assert (F == np.stack([A, A])).all() and (E == 0).all()


@pytest.mark.parametrize("alpha", [0, 3])
def test_initial_loss_is_guide_term_plus_keyframe_patch_difference(alpha):
    # iters = 0: E of F_l at x = alpha Eq.1(G_l at F_l(x), G_i at x)
    #                          + Eq.1(S_l at F_l(x), S_r at F_r(x)), and symmetrically.
    g, s, l, r, tl, tr = _segment(N=4, H=11, W=13)
    k, n, H, W = 3, r - l - 1, g.shape[1], g.shape[2]
    rng = np.random.default_rng(alpha + 2)
    init = np.stack([np.stack([rng.integers(0, H, (n, H, W)), rng.integers(0, W, (n, H, W))], -1)
                     for _ in range(2)]).astype(np.int32)
    sl, sr = s[l], s[r]
    _, E = oracle.nnf_segment(g[l], g[r], sl, sr, g[l + 1:r], k, 0, alpha, tl, tr, init=init)
    for q in range(n):
        T = g[l + 1 + q]
        for y in range(H):
            for x in range(W):
                fl, fr = init[0, q, y, x], init[1, q, y, x]
                pair = _ssd(sl, sr, k, fl[0], fl[1], fr[0], fr[1])
                assert E[0, q, y, x] == alpha * _ssd(g[l], T, k, fl[0], fl[1], y, x) + pair
                assert E[1, q, y, x] == alpha * _ssd(g[r], T, k, fr[0], fr[1], y, x) + pair


@pytest.mark.parametrize("tracking", [False, True])
def test_the_two_sides_are_symmetric(tracking):
    # Exchanging the keys (guides, styles and streams) exchanges the fields: each side's
    # update uses its own inputs and the other side's snapshot only.
    g, s, l, r, tl, tr = _segment(N=6, seed=8)
    a = oracle.nnf_segment(g[l], g[r], s[l], s[r], g[l + 1:r], 5, 2, 4, tl, tr, tracking=tracking, seed=3)
    b = oracle.nnf_segment(g[r], g[l], s[r], s[l], g[l + 1:r], 5, 2, 4, tr, tl, tracking=tracking, seed=3)
    assert (a[0][0] == b[0][1]).all() and (a[0][1] == b[0][0]).all()
    assert (a[1][0] == b[1][1]).all() and (a[1][1] == b[1][0]).all()


@pytest.mark.parametrize("tracking", [False, True])
def test_an_iteration_never_raises_the_coupled_loss(tracking):
    # The incumbent is re-evaluated against the partner's snapshot and replaced only by a
    # strictly better candidate: after iteration t + 1 every pixel's loss is at most the
    # loss of the iteration-t fields (iters = 0 with them as the initial fields).
    g, s, l, r, tl, tr = _segment(N=5, H=16, W=17, seed=11)
    for t in range(3):
        Ft, _ = oracle.nnf_segment(g[l], g[r], s[l], s[r], g[l + 1:r], 5, t, 6, tl, tr,
                                   tracking=tracking, seed=7)
        _, Lt = oracle.nnf_segment(g[l], g[r], s[l], s[r], g[l + 1:r], 5, 0, 6, tl, tr, init=Ft)
        _, E1 = oracle.nnf_segment(g[l], g[r], s[l], s[r], g[l + 1:r], 5, t + 1, 6, tl, tr,
                                   tracking=tracking, seed=7)
        assert (E1 <= Lt).all() and (E1 < Lt).any()


def test_eq9_weights_between_constant_keys_with_alignment():
    N, keys = 11, [2, 9]
    g, _ = synth.small_clip(N, 16, 18, seed=2, motion="affine")
    ks = np.stack([np.full(g.shape[1:], 40, np.uint8), np.full(g.shape[1:], 180, np.uint8)])
    for tracking in (False, True):
        out = oracle.interpolate_aligned(g, keys, ks, 3, 2, 5, tracking=tracking, seed=1)
        for i in range(N):
            if 2 < i < 9:
                num, den = 9 * ((9 - i) * 40 + (i - 2) * 180), 255 * 9 * 7
            else:
                num, den = 9 * (40 if i <= 2 else 180), 255 * 9
            assert (out[i] == np.float32(num) / np.float32(den)).all(), (tracking, i)


def test_frames_with_one_key_take_the_plain_loss():
    # Frames before the first key and after the last have no partner: they equal the plain
    # (or tracked) interpolation; frames between keys differ.
    g, s = synth.small_clip(10, 20, 23, seed=6, motion="affine")
    keys = [3, 6]
    ks = np.ascontiguousarray(s[keys])
    for tracking, ref in ((False, oracle.interpolate(g, keys, ks, 5, 2, seed=4)),
                          (True, oracle.interpolate_tracking(g, keys, ks, 5, 2, seed=4))):
        out = oracle.interpolate_aligned(g, keys, ks, 5, 2, 10, tracking=tracking, seed=4)
        for i in (0, 1, 2, 3, 6, 7, 8, 9):
            assert (out[i] == ref[i]).all(), (tracking, i)
        assert not (out[4:6] == ref[4:6]).all()


@pytest.mark.parametrize("tracking", [False, True])
def test_segment_frames_are_the_eq9_mix_of_the_coupled_fields(tracking):
    # Composition check: frame i between keys l and r is ((r - i) V_l + (i - l) V_r) /
    # (255 k^2 (r - l)), V the remap sums of the keyframe styles through the coupled fields
    # whose random streams are those of the pairs (l -> i) and (r -> i).
    g, s = synth.small_clip(7, 17, 19, seed=12, motion="affine")
    keys, k, iters, alpha, seed = [1, 5], 5, 2, 8, 6
    ks = np.ascontiguousarray(s[keys])
    out = oracle.interpolate_aligned(g, keys, ks, k, iters, alpha, tracking=tracking, seed=seed)
    l, r = keys
    tl = [oracle.pair_tag(l, i) for i in range(l + 1, r)]
    tr = [oracle.pair_tag(r, i) for i in range(l + 1, r)]
    F, _ = oracle.nnf_segment(g[l], g[r], ks[0], ks[1], g[l + 1:r], k, iters, alpha, tl, tr,
                              tracking=tracking, seed=seed)
    for q, i in enumerate(range(l + 1, r)):
        acc = ((r - i) * oracle.remap_sum(ks[0], F[0, q], k).astype(np.uint64)
               + (i - l) * oracle.remap_sum(ks[1], F[1, q], k).astype(np.uint64))
        ref = acc.astype(np.float32) / np.float32(255 * k * k * (r - l))
        assert (out[i] == ref).all(), i
