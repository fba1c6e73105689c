"""The oracle's pins catch plausible mistakes.

Each mutant below is a one-place edit of oracle/fbref.c of the kind a restatement of
the paper can get wrong (a dropped term, a wrong sign, an index of the wrong axis, a
non-strict acceptance, an off-by-one bound or constant).  It is compiled into a
temporary directory and the pin suites (tests/test_oracle_pins.py,
tests/test_oracle_balanced.py, tests/test_oracle_fast.py, tests/test_oracle_accurate.py,
tests/test_oracle_tracking.py, tests/test_oracle_alignment.py) are run against it:
every mutant must make at least one pin fail.  The oracle's own source is not touched.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fbref.c")

# name: (original text, replacement, which occurrence (0-based, in source order: the
# plain-mode site precedes the balanced-mode one, which precedes the alignment one) or
# None for a unique site)
MUTANTS = {
    "philox_nine_rounds": ("round < 10", "round < 9", None),
    "philox_weyl_constant": ("#define PHILOX_WEYL_B 0xBB67AE85u", "#define PHILOX_WEYL_B 0xBB67AE84u", None),
    "philox_words_swapped": ("uint32_t y1 = pb_lo;", "uint32_t y1 = pa_lo;", None),
    "ssd_drops_a_channel": ("for (int ch = 0; ch < 3; ++ch) {\n                int d",
                            "for (int ch = 0; ch < 2; ++ch) {\n                int d", None),
    "ssd_target_row_clamped_to_width": ("int tr = clampi(xr + a, 0, H - 1)", "int tr = clampi(xr + a, 0, W - 1)", None),
    "ssd_source_column_mirrored": ("sc = clampi(uc + b, 0, W - 1);", "sc = clampi(uc - b, 0, W - 1);", None),
    "downsample_rounds_half_down": ("(uint8_t)((s + 2) >> 2)", "(uint8_t)((s + 1) >> 2)", None),
    "uniform_offset_excludes_plus_r": ("uniform_below(u[w], (uint32_t)(2 * r + 1)) - r",
                                       "uniform_below(u[w], (uint32_t)(2 * r)) - r", None),
    "init_row_from_column_word": ("*r = uniform_below(u[0], (uint32_t)H);", "*r = uniform_below(u[1], (uint32_t)H);", None),
    "propagation_row_offset_sign": ("int cr = clampi(F[2 * n] - dirs[d][0], 0, h - 1);",
                                "int cr = clampi(F[2 * n] + dirs[d][0], 0, h - 1);", 0),
    "propagation_column_offset_sign": ("int cc = clampi(F[2 * n + 1] - dirs[d][1], 0, w - 1);",
                                       "int cc = clampi(F[2 * n + 1] + dirs[d][1], 0, w - 1);", 0),
    "propagation_accepts_ties": ("if (e < be) { be = e; br = cr; bc = cc; }",
                                 "if (e <= be) { be = e; br = cr; bc = cc; }", 0),
    "random_search_accepts_ties": ("if (e < be) { be = e; br = cr; bc = cc; }",
                                   "if (e <= be) { be = e; br = cr; bc = cc; }", 1),
    "random_search_skips_largest_radius": ("int rad = r0 >> t;", "int rad = r0 >> (t + 1);", 0),
    "random_search_centred_on_snapshot": ("int cr = clampi(br + dr, 0, h - 1);\n                        int cc = clampi(bc + dc, 0, w - 1);",
                                          "int cr = clampi(F[2 * x] + dr, 0, h - 1);\n                        int cc = clampi(F[2 * x + 1] + dc, 0, w - 1);", 0),
    "upsample_drops_parity": ("Fn[2 * x] = clampi(2 * F[2 * xc] + (r & 1), 0, h - 1);",
                              "Fn[2 * x] = clampi(2 * F[2 * xc], 0, h - 1);", None),
    "remap_offset_sign": ("int sr = clampi(fr - (qr - r), 0, H - 1);", "int sr = clampi(fr + (qr - r), 0, H - 1);", 0),
    "remap_unclamped_neighbour_offset": ("int sc = clampi(fc - (qc - c), 0, W - 1);", "int sc = clampi(fc - b, 0, W - 1);", 0),
    "remap_rows_and_columns_swapped": ("int fr = clampi(nnf[2 * q], 0, H - 1), fc = clampi(nnf[2 * q + 1], 0, W - 1);",
                                       "int fr = clampi(nnf[2 * q + 1], 0, H - 1), fc = clampi(nnf[2 * q], 0, W - 1);", 0),
    "remap_divisor_off_by_one": ("float den = (float)(255 * k * k);\n    for (size_t i = 0; i < n; ++i)",
                                 "float den = (float)(255 * k * k + 1);\n    for (size_t i = 0; i < n; ++i)", None),
    "downsample_drops_second_row": ("int r0 = 2 * r, r1 = clampi(2 * r + 1, 0, H - 1);",
                                    "int r0 = 2 * r, r1 = clampi(2 * r, 0, H - 1);", None),
    "interpolation_single_key_weight": ("fbref_pair_tag(l, i), 1u, acc);", "fbref_pair_tag(l, i), 2u, acc);", None),
    "shat_rounds_down": ("shat[t] = (uint8_t)((v[t] + kk / 2) / kk);", "shat[t] = (uint8_t)(v[t] / kk);", None),
    "balanced_alpha_on_style_term": ("return alpha * fbref_ssd(gs, gt, H, W, k, ur, uc, xr, xc) +\n           fbref_ssd(ss, shat, H, W, k, ur, uc, xr, xc);",
                                     "return fbref_ssd(gs, gt, H, W, k, ur, uc, xr, xc) +\n           alpha * fbref_ssd(ss, shat, H, W, k, ur, uc, xr, xc);", None),
    "balanced_guide_term_on_style_image": ("return alpha * fbref_ssd(gs, gt,", "return alpha * fbref_ssd(ss, gt,", 0),
    "align_guide_term_on_style_image": ("return alpha * fbref_ssd(gs, gt,", "return alpha * fbref_ssd(ss, gt,", 1),
    "balanced_style_term_against_target_guide": ("           fbref_ssd(ss, shat, H, W, k, ur, uc, xr, xc);", "           fbref_ssd(ss, gt, H, W, k, ur, uc, xr, xc);", None),
    "balanced_error_not_reevaluated": ("                E[x] = balanced_loss(", "                if (it == 0) E[x] = balanced_loss(", None),
    "balanced_shat_not_refreshed": ("        fbref_shat(src_style, F, h, w, k, shat);", "        if (it == 0) fbref_shat(src_style, F, h, w, k, shat);", None),
    "balanced_propagation_row_offset_sign": ("int cr = clampi(F[2 * n] - dirs[d][0], 0, h - 1);",
                                             "int cr = clampi(F[2 * n] + dirs[d][0], 0, h - 1);", 1),
    "balanced_random_search_skips_largest_radius": ("int rad = r0 >> t;", "int rad = r0 >> (t + 1);", 1),
    "tracking_wrong_neighbours": ("for (int nb = m - 1; nb <= m + 1; nb += 2) {", "for (int nb = m - 2; nb <= m + 2; nb += 4) {", None),
    "tracking_candidate_offset": ("uint32_t e = fbref_ssd(src, T, h, w, k, Fb[0], Fb[1], r, c);\n                        if (e < be) { be = e; br = Fb[0]; bc = Fb[1]; }",
                                  "uint32_t e = fbref_ssd(src, T, h, w, k, clampi(Fb[0] + 1, 0, h - 1), Fb[1], r, c);\n                        if (e < be) { be = e; br = clampi(Fb[0] + 1, 0, h - 1); bc = Fb[1]; }", None),
    "tracking_interpolation_weights_swapped": ("wgt = (uint32_t)(next - i); dd = (uint32_t)(next - a);", "wgt = (uint32_t)(i - a); dd = (uint32_t)(next - a);", None),
    "tracking_pair_stream_reversed": ("for (int q = 0; q < n; ++q) tags[q] = fbref_pair_tag(a, lo + q);", "for (int q = 0; q < n; ++q) tags[q] = fbref_pair_tag(lo + q, a);", 0),
    "align_one_key_run_stream_reversed": ("for (int q = 0; q < n; ++q) tags[q] = fbref_pair_tag(a, lo + q);", "for (int q = 0; q < n; ++q) tags[q] = fbref_pair_tag(lo + q, a);", 1),
    "tracking_run_includes_the_next_key": ("const int runs[2][2] = {{prev + 1, a - 1}, {a + 1, next - 1}};", "const int runs[2][2] = {{prev + 1, a - 1}, {a + 1, next < N ? next : N - 1}};", None),
    "blend_tracking_chain_includes_the_source": ("const int runs[2][2] = {{j - M < 0 ? 0 : j - M, j - 1}, {j + 1, j + M > N - 1 ? N - 1 : j + M}};",
                                                 "const int runs[2][2] = {{j - M < 0 ? 0 : j - M, j - 1}, {j, j + M > N - 1 ? N - 1 : j + M}};", None),
    "blend_tracking_one_chain_per_source": ("        for (int side = 0; side < 2 && rc == 0; ++side) {\n            const int lo = runs[side][0], hi = runs[side][1];\n            if (lo > hi) continue;\n            const int n = hi - lo + 1;\n            uint32_t *tags = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));\n            int32_t *F = (int32_t *)malloc((size_t)n * npx * 2 * sizeof(int32_t));\n            for (int q = 0; q < n; ++q) tags[q] = fbref_pair_tag(j, lo + q);",
                                            "        for (int side = 1; side < 2 && rc == 0; ++side) {\n            const int lo = runs[side][0], hi = runs[side][1];\n            if (lo > hi) continue;\n            const int n = hi - lo + 1;\n            uint32_t *tags = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));\n            int32_t *F = (int32_t *)malloc((size_t)n * npx * 2 * sizeof(int32_t));\n            for (int q = 0; q < n; ++q) tags[q] = fbref_pair_tag(j, lo + q);", None),
    "blend_tracking_pair_stream_reversed": ("for (int q = 0; q < n; ++q) tags[q] = fbref_pair_tag(j, lo + q);", "for (int q = 0; q < n; ++q) tags[q] = fbref_pair_tag(lo + q, j);", None),
    "blend_tracking_window_short_by_one": ("float den = (float)(255 * k * k * (hi - lo + 1));\n        for (size_t t = 0; t < fsz; ++t) out[(size_t)i * fsz + t]",
                                           "float den = (float)(255 * k * k * (hi - lo + 2));\n        for (size_t t = 0; t < fsz; ++t) out[(size_t)i * fsz + t]", None),
    "align_partner_is_own_field": ("const int32_t *Fo = F + ((size_t)(1 - sd) * n + m) * npx * 2;", "const int32_t *Fo = F + ((size_t)sd * n + m) * npx * 2;", None),
    "align_pairwise_term_own_style": ("*Ss = S[sd], *So = S[1 - sd];", "*Ss = S[sd], *So = S[sd];", None),
    "align_guide_weight_dropped": ("    return alpha * fbref_ssd(gs, gt, H, W, k, ur, uc, xr, xc) +\n           fbref_ssd(ss, so, H, W, k, ur, uc, pr, pc);",
                                   "    return fbref_ssd(gs, gt, H, W, k, ur, uc, xr, xc) +\n           fbref_ssd(ss, so, H, W, k, ur, uc, pr, pc);", None),
    "align_pairwise_term_at_the_target_pixel": ("fbref_ssd(ss, so, H, W, k, ur, uc, pr, pc);", "fbref_ssd(ss, so, H, W, k, ur, uc, xr, xc);", None),
    "align_tracking_neighbour_from_partner_side": ("const int32_t *Fb = F + (((size_t)sd * n + nb) * npx + x) * 2;", "const int32_t *Fb = F + (((size_t)(1 - sd) * n + nb) * npx + x) * 2;", None),
    "align_random_search_partner_stream": ("fbref_rs_offset(p->seed, (uint32_t)x, tags[sd][m], 0, it, t, rad, &dr, &dc);", "fbref_rs_offset(p->seed, (uint32_t)x, tags[1 - sd][m], 0, it, t, rad, &dr, &dc);", None),
    "align_segment_tags_swapped": ("tr[q] = fbref_pair_tag(r, l + 1 + q);", "tr[q] = fbref_pair_tag(l + 1 + q, r);", None),
    "align_eq9_weights_swapped": ("acc[(size_t)i * fsz + t] += (uint32_t)(r - i) * V[t];", "acc[(size_t)i * fsz + t] += (uint32_t)(i - l) * V[t];", None),
    "accurate_tbar_rounds_down": ("tbar[t] = (uint8_t)((acc[t] + den_t / 2) / den_t);", "tbar[t] = (uint8_t)(acc[t] / den_t);", None),
    "accurate_tbar_without_self_term": ("        for (size_t t = 0; t < fsz; ++t) acc[t] = kk * Si[t];\n        for (int m = 0; m < np; ++m) {\n            fbref_remap_sum",
                                        "        for (size_t t = 0; t < fsz; ++t) acc[t] = 0;\n        for (int m = 0; m < np; ++m) {\n            fbref_remap_sum", None),
    "accurate_propagation_row_offset_sign": ("int cr = clampi(Fm[2 * n] - dirs[d][0], 0, h - 1);", "int cr = clampi(Fm[2 * n] + dirs[d][0], 0, h - 1);", None),
    "accurate_random_search_skips_largest_radius": ("int rad = r0 >> t;", "int rad = r0 >> (t + 1);", 2),
    "accurate_pair_stream_reversed": ("const uint32_t tag = fbref_pair_tag(js[m], i);", "const uint32_t tag = fbref_pair_tag(i, js[m]);", None),
    "fast_table_remap_offset_sign": ("int sr = clampi(fr - (qr - r), 0, H - 1);", "int sr = clampi(fr + (qr - r), 0, H - 1);", 1),
    "fast_walk_steps_twice_the_piece": ("        i -= 1 << L;", "        i -= 2 << L;", None),
    "fast_identity_piece_unweighted": ("acc[t] += (uint32_t)(k * k) * B[t];  /* identity remap */",
                                       "acc[t] += B[t];  /* identity remap */", None),
    "fast_self_term_not_removed": ("uint32_t num = acc[t] - k4 * styles[(size_t)i * fsz + t];", "uint32_t num = acc[t];", None),
    "fast_query_nnf_reversed": ("rc = fbref_nnf(guides + (size_t)fi * fsz, guides + (size_t)fr * fsz, H, W, p,\n                           fbref_pair_tag(fi, fr)",
                                "rc = fbref_nnf(guides + (size_t)fr * fsz, guides + (size_t)fi * fsz, H, W, p,\n                           fbref_pair_tag(fr, fi)", None),
    "fast_entry_nnf_reversed": ("rc = fbref_nnf(guides + (size_t)fa * fsz, guides + (size_t)fj * fsz, H, W, p,\n                       fbref_pair_tag(fa, fj)",
                                "rc = fbref_nnf(guides + (size_t)fj * fsz, guides + (size_t)fa * fsz, H, W, p,\n                       fbref_pair_tag(fj, fa)", None),
    "fast_right_side_not_reversed": ("rc = query(guides, styles, N, H, W, p, 1, N - 1 - hi, N - 1 - i, acc);",
                                     "rc = query(guides, styles, N, H, W, p, 0, i, hi, acc);", None),
    "fast_piece_may_leave_the_interval": ("while (((i >> L) & 1) && i - (1 << (L + 1)) + 1 >= l) ++L;",
                                          "while (((i >> L) & 1) && i - (1 << (L + 1)) + 1 >= l - 1) ++L;", None),
    "fast_entry_misses_a_source": ("for (int a = j - (1 << L) + 1; a < j && rc == 0; ++a) {",
                                   "for (int a = j - (1 << L) + 2; a < j && rc == 0; ++a) {", None),
    "fast_divisor_count": ("double den = 255.0 * k4 * (double)(hi - lo + 1);", "double den = 255.0 * k4 * (double)(hi - lo);", None),
    "blend_divisor_drops_self_term": ("float den = (float)(255 * k * k * (hi - lo + 1));",
                                      "float den = (float)(255 * k * k * (hi - lo));", 0),
    "blend_self_term_unweighted": ("for (size_t t = 0; t < fsz; ++t) acc[t] = (uint32_t)(k * k) * styles[(size_t)i * fsz + t];",
                                   "for (size_t t = 0; t < fsz; ++t) acc[t] = styles[(size_t)i * fsz + t];", 0),
    "blend_window_upper_end_short": ("hi = i + M > N - 1 ? N - 1 : i + M;", "hi = i + M > N - 1 ? N - 2 : i + M;", 0),
    "interpolation_weights_swapped": ("fbref_pair_tag(l, i), (uint32_t)(r - i), acc);", "fbref_pair_tag(l, i), (uint32_t)(i - l), acc);", None),
    "interpolation_key_not_copied": ("den_int = (uint32_t)(255 * k * k);\n    } else if", "den_int = (uint32_t)(255 * k * k + 1);\n    } else if", None),
}


def mutate(src: str, old: str, new: str, which):
    n = src.count(old)
    assert n >= 1, f"mutation site not found: {old!r}"
    if which is None:
        assert n == 1, f"{n} sites for {old!r}"
        return src.replace(old, new)
    pos = -1
    for _ in range(which + 1):
        pos = src.index(old, pos + 1)
    return src[:pos] + new + src[pos + len(old):]


def run_mutant(name: str, workdir: str):
    """Compile mutant `name` into workdir and run the pin suites against it; returns
    (pytest exit code, tail of its output)."""
    old, new, which = MUTANTS[name]
    with open(SRC) as f:
        src = f.read()
    try:
        text = mutate(src, old, new, which)
    except AssertionError as e:          # a mutation site that is missing or ambiguous
        return -1, str(e)
    mutant_c = os.path.join(workdir, f"{name}.c")
    with open(mutant_c, "w") as f:
        f.write(text)
    lib = os.path.join(workdir, f"lib{name}.so")
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                    "-I", os.path.join(ROOT, "oracle"), "-o", lib, mutant_c], check=True)
    env = dict(os.environ, FBREF_TEST_LIBRARY=lib, OMP_NUM_THREADS="2")
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                          os.path.join(ROOT, "tests", "test_oracle_balanced.py"),
                          os.path.join(ROOT, "tests", "test_oracle_fast.py"),
                          os.path.join(ROOT, "tests", "test_oracle_accurate.py"),
                          os.path.join(ROOT, "tests", "test_oracle_tracking.py"),
                          os.path.join(ROOT, "tests", "test_oracle_alignment.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return res.returncode, res.stdout[-1500:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """All mutants, compiled and tested concurrently (each in its own processes)."""
    from concurrent.futures import ThreadPoolExecutor
    workdir = str(tmp_path_factory.mktemp("oracle_mutants"))
    workers = max(2, min(8, (os.cpu_count() or 2)))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {name: ex.submit(run_mutant, name, workdir) for name in MUTANTS}
        return {name: f.result() for name, f in futs.items()}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, outcomes):
    code, out = outcomes[name]
    assert code == 1, f"no pin failed for mutant {name}:\n{out}"
