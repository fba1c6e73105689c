"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: published
known-answer vectors, hand-derived values, closed forms, exhaustive search, or an
invariant of the algorithm.  The cases are chosen so that a plausible slip in the
oracle (a dropped term, a sign, a transposed operand, a wrong divisor) fails one.
"""
import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden

# ----------------------------------------------------------------------------------
# Philox-4x32-10 (counter-based stream behind init and random search, Sec. 3.2)
# ----------------------------------------------------------------------------------


def test_philox_known_answer_vectors():
    rows = read_golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        vals = [int(v, 16) for v in r]
        ctr, key, want = vals[0:4], vals[4:6], vals[6:10]
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


# ----------------------------------------------------------------------------------
# Eq. 1 patch distance
# ----------------------------------------------------------------------------------
def _img(rows):
    a = np.array(rows, np.uint8)
    return np.ascontiguousarray(np.repeat(a[..., None], 3, axis=2))


def test_ssd_hand_derived_cases():
    imgs = {"S": _img([[0, 10, 20], [30, 40, 50]]), "T": _img([[1, 2, 3], [4, 5, 6]]),
            "C": np.full((2, 3, 3), 5, np.uint8)}
    rows = read_golden("ssd_handcase.txt")
    assert len(rows) >= 4
    for s, t, k, ur, uc, xr, xc, want in rows:
        got = oracle.ssd(imgs[s], imgs[t], int(k), (int(ur), int(uc)), (int(xr), int(xc)))
        assert got == int(want), (s, t, ur, uc, xr, xc)


@pytest.mark.parametrize("k", [3, 5, 7, 9])
def test_ssd_constant_images_closed_form(k):
    a = np.full((11, 13, 3), 200, np.uint8)
    b = np.full((11, 13, 3), 37, np.uint8)
    for u, x in [((0, 0), (10, 12)), ((5, 6), (5, 6)), ((10, 0), (0, 12))]:
        assert oracle.ssd(a, b, k, u, x) == 3 * k * k * (200 - 37) ** 2


def test_ssd_single_channel_difference_counts_every_covering_patch():
    # One pixel of one channel differs by 9; an interior patch covering it counts
    # 81 once; a patch whose clamped footprint reads that edge pixel several times
    # counts it with that multiplicity.
    a = np.zeros((9, 9, 3), np.uint8)
    b = a.copy()
    b[4, 4, 1] = 9
    assert oracle.ssd(a, b, 5, (4, 4), (4, 4)) == 81
    assert oracle.ssd(a, b, 5, (4, 4), (0, 0)) == 0      # footprint rows/cols 0..2
    c = a.copy()
    c[0, 0, 2] = 9                                        # corner pixel, read 3x3 = 9 times
    assert oracle.ssd(a, c, 5, (4, 4), (0, 0)) == 9 * 81
    assert oracle.ssd(c, a, 5, (0, 0), (4, 4)) == 9 * 81  # same on the source side


# ----------------------------------------------------------------------------------
# Pyramid step of Alg. 1
# ----------------------------------------------------------------------------------
def test_downsample_box_mean_round_half_up_and_odd_edges():
    img = np.zeros((3, 3, 3), np.uint8)
    img[0, 0], img[0, 1], img[1, 0], img[1, 1] = 1, 2, 3, 4      # (1+2+3+4+2)>>2 = 3
    img[0, 2], img[1, 2] = 5, 6                                  # odd column: (5+5+6+6+2)>>2 = 6
    img[2, 0], img[2, 1] = 7, 8                                  # odd row: (7+8+7+8+2)>>2 = 8
    img[2, 2] = 9                                                # corner: 9
    d = oracle.downsample(img)
    assert d.shape == (2, 2, 3)
    assert d[0, 0, 0] == 3 and d[0, 1, 0] == 6 and d[1, 0, 0] == 8 and d[1, 1, 0] == 9
    assert (oracle.downsample(np.full((7, 5, 3), 77, np.uint8)) == 77).all()


# ----------------------------------------------------------------------------------
# Random draws
# ----------------------------------------------------------------------------------
def test_random_search_offsets_uniform_on_closed_interval():
    r = 3
    draws = np.array([oracle.rs_offset(12345, pix, 7, 0, 2, t, r)
                      for pix in range(3000) for t in (0, 1)])
    assert draws.min() == -r and draws.max() == r
    for axis in (0, 1):
        counts = np.bincount(draws[:, axis] + r, minlength=2 * r + 1)
        expected = len(draws) / (2 * r + 1)
        chi2 = ((counts - expected) ** 2 / expected).sum()
        assert chi2 < 30.0, counts                     # 6 dof; p ~ 4e-5
    # the two candidates sharing a Philox block are not the same draw
    assert (draws[0::2] != draws[1::2]).any(axis=1).mean() > 0.8


def test_random_init_covers_source_uniformly():
    g = np.zeros((40, 50, 3), np.uint8)
    F, E = oracle.nnf(g, g, 3, 0, seed=99)
    assert F[..., 0].min() == 0 and F[..., 0].max() == 39
    assert F[..., 1].min() == 0 and F[..., 1].max() == 49
    assert abs(F[..., 0].mean() - 19.5) < 1.0 and abs(F[..., 1].mean() - 24.5) < 1.5
    assert (E == 0).all()


# ----------------------------------------------------------------------------------
# Alg. 1 patch matching
# ----------------------------------------------------------------------------------
def _noise_pair(H, W, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 256, (H, W, 3), dtype=np.uint8),
            rng.integers(0, 256, (H, W, 3), dtype=np.uint8))


@pytest.mark.parametrize("k,levels", [(3, 1), (5, 1), (5, 2), (7, 1)])
def test_nnf_never_beats_exhaustive_search(k, levels):
    s, t = _noise_pair(14, 17, 5 + k)
    F, E = oracle.nnf(s, t, k, 3, levels=levels, seed=3)
    Fb, Eb = oracle.nnf_bruteforce(s, t, k)
    assert (E >= Eb).all()
    assert ((F[..., 0] >= 0) & (F[..., 0] < 14) & (F[..., 1] >= 0) & (F[..., 1] < 17)).all()
    for r in range(14):
        for c in range(17):
            assert E[r, c] == oracle.ssd(s, t, k, F[r, c], (r, c))


def test_nnf_reaches_exhaustive_optimum_with_many_iterations():
    g, _ = synth.shift_clip(2, 16, 16, seed=11)
    F, E = oracle.nnf(g[0], g[1], 5, 20, seed=1)
    Fb, Eb = oracle.nnf_bruteforce(g[0], g[1], 5)
    assert (E == Eb).mean() >= 0.99


def test_exhaustive_search_matches_known_shift_on_interior():
    g, sh = synth.shift_clip(2, 20, 22, seed=4)
    Fb, Eb = oracle.nnf_bruteforce(g[0], g[1], 5)
    d = sh[1] - sh[0]
    for r in range(2, 18):
        for c in range(2, 20):
            u = (r + d[0], c + d[1])
            if 2 <= u[0] < 18 and 2 <= u[1] < 20:
                assert Eb[r, c] == 0 and tuple(Fb[r, c]) == u


def _true_field(H, W, d):
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    return np.stack([np.clip(rr + d[0], 0, H - 1), np.clip(cc + d[1], 0, W - 1)], -1).astype(np.int32)


def test_known_shift_field_is_a_fixed_point():
    g, sh = synth.shift_clip(3, 30, 34, seed=8)
    j, i, k, p = 0, 2, 5, 2
    d = sh[i] - sh[j]
    Fstar = _true_field(30, 34, d)
    F, E = oracle.nnf(g[j], g[i], k, 3, seed=5, init=Fstar)
    inner = np.zeros((30, 34), bool)
    for r in range(p, 30 - p):
        for c in range(p, 34 - p):
            ur, uc = r + d[0], c + d[1]
            inner[r, c] = p <= ur < 30 - p and p <= uc < 34 - p
    assert inner.sum() > 300
    assert (E[inner] == 0).all()
    assert (F[inner] == Fstar[inner]).all()


def test_propagation_repairs_one_wrong_match_with_the_correct_sign():
    # Every match is the true shift except one pixel, placed 15 px away.  With the
    # random search limited to radius 1, only propagation F(x+d) - d can repair it
    # in one iteration; F(x+d) + d would land 2 px off and keep a positive error.
    g, sh = synth.shift_clip(2, 40, 40, seed=21)
    d = sh[1] - sh[0]
    Fstar = _true_field(40, 40, d)
    init = Fstar.copy()
    x0 = (20, 19)
    init[x0] = (min(39, Fstar[x0][0] + 15), Fstar[x0][1])
    F, E = oracle.nnf(g[0], g[1], 5, 1, r0=1, seed=2, init=init)
    assert tuple(F[x0]) == tuple(Fstar[x0])
    assert E[x0] == 0


def test_propagation_repairs_runs_along_both_axes_with_the_correct_signs():
    # A horizontal run of wrong matches can only be repaired from the rows above and
    # below (d = (-1,0), (1,0)), a vertical run only from the columns beside it: each
    # checks the sign of F(x+d) - d on its own axis (random search limited to radius 1).
    g, sh = synth.shift_clip(2, 40, 40, seed=21)
    d = sh[1] - sh[0]
    Fstar = _true_field(40, 40, d)
    init = Fstar.copy()
    run_h = [(20, c) for c in range(10, 30)]
    run_v = [(r, 8) for r in range(10, 30)]
    for x in run_h:
        init[x] = (min(39, Fstar[x][0] + 15), Fstar[x][1])
    for x in run_v:
        init[x] = (Fstar[x][0], min(39, Fstar[x][1] + 15))
    F, E = oracle.nnf(g[0], g[1], 5, 1, r0=1, seed=2, init=init)
    for x in run_h + run_v:
        assert tuple(F[x]) == tuple(Fstar[x]) and E[x] == 0, x


def test_ties_keep_the_incumbent():
    # Alg. 1 updates only where the new error is strictly smaller.  On identical
    # constant frames every candidate ties, so the random initial field never changes.
    g = np.full((24, 28, 3), 77, np.uint8)
    F0, _ = oracle.nnf(g, g, 5, 0, seed=12)
    F3, E3 = oracle.nnf(g, g, 5, 3, seed=12)
    assert (F3 == F0).all() and (E3 == 0).all()


def test_random_init_rows_and_columns_are_independent():
    # A match drawn uniformly over the source has independent row and column: the
    # 8 x 8 grid of (row, column) cells is uniformly populated.
    g = np.zeros((64, 64, 3), np.uint8)
    F, _ = oracle.nnf(g, g, 3, 0, seed=31)
    cells = (F[..., 0] // 8) * 8 + F[..., 1] // 8
    counts = np.bincount(cells.ravel(), minlength=64)
    expected = F.shape[0] * F.shape[1] / 64
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 120.0, chi2                       # 63 dof; p ~ 2e-5
    assert abs(np.corrcoef(F[..., 0].ravel(), F[..., 1].ravel())[0, 1]) < 0.05


def test_random_search_starts_at_radius_r0():
    # Target = source moved one column left (match x + (0, 1)), identity start: the
    # propagation candidates F(x+d) - d all equal the incumbent, so only the random
    # search can move a pixel, and with r0 = 1 its single candidate (radius r0 >> 0 = 1)
    # hits the match with probability 1/9 per pixel.
    a, b = synth.noise_pair(48, 48, seed=5, shift=(0, -1))
    ident = _true_field(48, 48, (0, 0))
    F, E = oracle.nnf(a, b, 5, 1, r0=1, seed=8, init=ident)
    inner = (slice(3, 45), slice(3, 44))
    hit = (E[inner] == 0).mean()
    assert 0.05 < hit < 0.2, hit


def test_upsampled_field_keeps_the_pixel_parity():
    # An even shift (2, 4) commutes with the 2x2 box mean, so the coarse level holds the
    # exact half shift after enough iterations, and the upsampled field 2 F(x/2) + parity
    # is the exact fine shift: zero error before the first fine iteration.
    a, b = synth.noise_pair(40, 40, seed=6, shift=(2, 4))
    F, T = oracle.nnf_trace(a, b, 5, 8, levels=2, seed=3)
    inner = (slice(6, 34), slice(8, 32))
    assert (T[0][inner] == 0).mean() > 0.9


def test_random_search_is_centred_on_the_running_best():
    # Smooth texture, known shift d.  Every pixel starts one column off (x + d + (0, 1))
    # except a checkerboard of pixels that start 12 rows further away.  In one iteration
    # those pixels take the off-by-one match from a neighbour by propagation, and the
    # radius-1 random candidate around that running best hits the true match with
    # probability 1/9; centred on the far start it could not.
    H = W = 48
    g, sh = synth.shift_clip(2, H, W, seed=21)
    d = sh[1] - sh[0]
    init = _true_field(H, W, (d[0], d[1] + 1))
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    far = (rr + cc) % 2 == 0
    init[far, 0] = np.clip(rr[far] + d[0] + 12, 0, H - 1)
    F, E = oracle.nnf(g[0], g[1], 5, 1, r0=1, seed=4, init=init)
    sel = far & (rr >= 6) & (rr < H - 18) & (cc >= 6) & (cc < W - 8)
    hit = (E[sel] == 0).mean()
    assert 0.05 < hit < 0.2, hit


def test_error_is_monotone_per_pixel_across_iterations():
    g, _ = synth.small_clip(2, 33, 29, seed=17, motion="affine")
    F, T = oracle.nnf_trace(g[0], g[1], 5, 6, seed=4)
    assert (np.diff(T.astype(np.int64), axis=0) <= 0).all()
    assert (T[-1] < T[0]).mean() > 0.5


def test_zero_error_identity_is_a_fixed_point():
    s, _ = _noise_pair(12, 15, 2)
    ident = _true_field(12, 15, (0, 0))
    F, E = oracle.nnf(s, s, 3, 4, seed=9, init=ident)
    assert (F == ident).all() and (E == 0).all()


def test_nnf_is_deterministic_and_seed_and_tag_dependent():
    s, t = _noise_pair(16, 16, 3)
    a = oracle.nnf(s, t, 3, 1, seed=1, pair_tag=5)[0]
    assert (a == oracle.nnf(s, t, 3, 1, seed=1, pair_tag=5)[0]).all()
    assert (a != oracle.nnf(s, t, 3, 1, seed=2, pair_tag=5)[0]).any()
    assert (a != oracle.nnf(s, t, 3, 1, seed=1, pair_tag=6)[0]).any()


def test_pyramid_levels_reduce_error_on_large_motion():
    g, _ = synth.shift_clip(2, 64, 64, seed=31, max_step=12)
    _, E1 = oracle.nnf(g[0], g[1], 5, 1, levels=1, seed=3)
    _, E3 = oracle.nnf(g[0], g[1], 5, 1, levels=3, seed=3)
    assert E3.mean() < E1.mean()


# ----------------------------------------------------------------------------------
# Alg. 2 remap
# ----------------------------------------------------------------------------------
def test_remap_hand_derived_case():
    S = _img([[0, 10, 20], [30, 40, 50]])
    F = _true_field(2, 3, (0, 0))
    F[0, 1] = (1, 1)
    V = oracle.remap_sum(S, F, 3)
    for xr, xc, want in read_golden("remap_handcase.txt"):
        assert (V[int(xr), int(xc)] == int(want)).all()


@pytest.mark.parametrize("k", [3, 5, 7, 9])
def test_remap_identity_is_exact(k):
    rng = np.random.default_rng(k)
    S = rng.integers(0, 256, (13, 11, 3), dtype=np.uint8)
    out = oracle.remap(S, _true_field(13, 11, (0, 0)), k)
    assert (out == S.astype(np.float32) / np.float32(255.0)).all()
    assert (oracle.remap_sum(S, _true_field(13, 11, (0, 0)), k) == k * k * S.astype(np.uint32)).all()


def test_remap_integer_shift_gives_the_shifted_image():
    rng = np.random.default_rng(1)
    S = rng.integers(0, 256, (20, 24, 3), dtype=np.uint8)
    d, k, p = (3, -2), 5, 2
    V = oracle.remap_sum(S, _true_field(20, 24, d), k)
    for r in range(p, 20 - p):
        for c in range(p, 24 - p):
            sr, sc = r + d[0], c + d[1]
            if p <= sr < 20 - p and p <= sc < 24 - p:
                assert (V[r, c] == k * k * S[sr, sc].astype(np.uint32)).all()


def test_remap_out_of_range_nnf_entries_are_clamped():
    S = np.random.default_rng(2).integers(0, 256, (9, 9, 3), dtype=np.uint8)
    F = _true_field(9, 9, (0, 0))
    big = F.copy()
    big[..., 0] += 1000
    clamped = F.copy()
    clamped[..., 0] = 8
    assert (oracle.remap_sum(S, big, 3) == oracle.remap_sum(S, clamped, 3)).all()


# ----------------------------------------------------------------------------------
# Eq. 2 window blend
# ----------------------------------------------------------------------------------
BL = dict(patch=5, iters=3, seed=77)


def test_blend_constant_style_is_constant_including_truncated_windows():
    g, _ = synth.small_clip(6, 24, 20, seed=3)
    s = np.full_like(g, 133)
    for window in (1, 3, 5, 11):
        out = oracle.blend_window(g, s, window, **BL)
        assert np.abs(out - np.float32(133 / 255)).max() <= 1e-7


def test_blend_self_term_weight_and_divisor():
    # Only frame 2 carries style: its own output is S_2 / (255 * frames in window),
    # exactly, whatever the NNFs are.
    g, _ = synth.small_clip(5, 20, 18, seed=9)
    s = np.zeros_like(g)
    s[2] = np.random.default_rng(0).integers(0, 256, s[2].shape, dtype=np.uint8)
    for window, count in ((1, 1), (3, 3), (5, 5), (9, 5)):
        out = oracle.blend_frame(g, s, window, 2, **BL)
        want = s[2].astype(np.float64) / (255.0 * count)
        assert np.abs(out - want).max() <= 1e-7 and (window == 1 or out.max() < 1.0)


def _numerators(out, den):
    return np.rint(out.astype(np.float64) * den).astype(np.int64)


def test_blend_is_linear_in_the_style_frames():
    g, _ = synth.small_clip(5, 22, 19, seed=12)
    rng = np.random.default_rng(3)
    a = rng.integers(0, 128, g.shape, dtype=np.uint8)
    b = rng.integers(0, 128, g.shape, dtype=np.uint8)
    oa = oracle.blend_window(g, a, 3, **BL)
    ob = oracle.blend_window(g, b, 3, **BL)
    oab = oracle.blend_window(g, (a + b).astype(np.uint8), 3, **BL)
    k = BL["patch"]
    for i in range(5):
        den = 255 * k * k * (min(4, i + 1) - max(0, i - 1) + 1)
        assert (_numerators(oa[i], den) + _numerators(ob[i], den) == _numerators(oab[i], den)).all()


def test_blend_known_shift_closed_form_on_interior():
    # With exact NNFs the blended frame i is the mean of the style frames shifted by
    # s_i - s_j.  Many iterations make the NNF exact on almost every interior pixel.
    N, H, W, k, p = 5, 36, 36, 5, 2
    g, sh = synth.shift_clip(N, H, W, seed=41)
    s = synth.colour_matrix_styles(g, seed=41)
    out = oracle.blend_window(g, s, 3, patch=k, iters=10, seed=5)
    good = total = 0
    for i in range(N):
        js = [j for j in range(max(0, i - 1), min(N - 1, i + 1) + 1)]
        for r in range(p + 3, H - p - 3):
            for c in range(p + 3, W - p - 3):
                num = np.zeros(3, np.int64)
                ok = True
                for j in js:
                    ur, uc = r + sh[i][0] - sh[j][0], c + sh[i][1] - sh[j][1]
                    if not (p + 2 <= ur < H - p - 2 and p + 2 <= uc < W - p - 2):
                        ok = False
                        break
                    num += k * k * s[j, ur, uc].astype(np.int64)
                if not ok:
                    continue
                total += 1
                want = num.astype(np.float32) / np.float32(255 * k * k * len(js))
                good += int((out[i, r, c] == want).all())
    assert total > 1500
    assert good / total >= 0.97


# ----------------------------------------------------------------------------------
# Sec. 3.5.2 keyframe combination
# ----------------------------------------------------------------------------------
IP = dict(patch=5, iters=3, seed=5)


def test_interpolation_copies_keyframes_exactly():
    g, st = synth.small_clip(7, 21, 23, seed=2)
    keys = [1, 5]
    out = oracle.interpolate(g, keys, st[keys], **IP)
    for m, kf in enumerate(keys):
        assert (out[kf] == st[kf].astype(np.float32) / np.float32(255.0)).all()


def test_interpolation_weights_between_constant_keys():
    g, _ = synth.small_clip(9, 18, 20, seed=6)
    keys = [1, 7]
    ks = np.stack([np.full((18, 20, 3), 30, np.uint8), np.full((18, 20, 3), 210, np.uint8)])
    out = oracle.interpolate(g, keys, ks, **IP)
    for i in range(9):
        if i <= 1:
            want = 30 / 255
        elif i >= 7:
            want = 210 / 255
        else:
            want = ((7 - i) * 30 + (i - 1) * 210) / (6 * 255)
        assert np.abs(out[i] - want).max() <= 2e-7, i


def test_single_keyframe_renders_whole_clip_from_it():
    g, st = synth.small_clip(4, 16, 16, seed=8)
    ks = np.full((1, 16, 16, 3), 99, np.uint8)
    out = oracle.interpolate(g, [2], ks, **IP)
    assert np.abs(out - np.float32(99 / 255)).max() <= 1e-7


def test_interpolation_known_shift_closed_form_on_interior():
    N, H, W, k, p = 6, 36, 36, 5, 2
    g, sh = synth.shift_clip(N, H, W, seed=44)
    st = synth.colour_matrix_styles(g, seed=44)
    keys = [0, 5]
    out = oracle.interpolate(g, keys, st[keys], patch=k, iters=10, seed=3)
    good = total = 0
    for i in range(1, 5):
        for r in range(p + 3, H - p - 3):
            for c in range(p + 3, W - p - 3):
                num = np.zeros(3, np.int64)
                ok = True
                for kf, wgt in ((0, 5 - i), (5, i)):
                    ur, uc = r + sh[i][0] - sh[kf][0], c + sh[i][1] - sh[kf][1]
                    if not (p + 2 <= ur < H - p - 2 and p + 2 <= uc < W - p - 2):
                        ok = False
                        break
                    num += wgt * k * k * st[kf, ur, uc].astype(np.int64)
                if not ok:
                    continue
                total += 1
                want = num.astype(np.float32) / np.float32(255 * k * k * 5)
                good += int((out[i, r, c] == want).all())
    assert total > 800
    assert good / total >= 0.97
