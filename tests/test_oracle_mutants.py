"""The oracle's pins catch plausible mistakes.

Each mutant below is a one-place edit of oracle/fbref.c of the kind a restatement of
the paper can get wrong (a dropped term, a wrong sign, an index of the wrong axis, a
non-strict acceptance, an off-by-one bound or constant).  It is compiled into a
temporary directory and the pin suites (tests/test_oracle_pins.py,
tests/test_oracle_balanced.py) are run against it:
every mutant must make at least one pin fail.  The oracle's own source is not touched.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fbref.c")

# name: (original text, replacement, which occurrence (0-based; the plain-mode site
# precedes the balanced-mode one) or None for a unique site)
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
                                          "int cr = clampi(F[2 * x] + dr, 0, h - 1);\n                        int cc = clampi(F[2 * x + 1] + dc, 0, w - 1);", None),
    "upsample_drops_parity": ("Fn[2 * x] = clampi(2 * F[2 * xc] + (r & 1), 0, h - 1);",
                              "Fn[2 * x] = clampi(2 * F[2 * xc], 0, h - 1);", None),
    "remap_offset_sign": ("int sr = clampi(fr - (qr - r), 0, H - 1);", "int sr = clampi(fr + (qr - r), 0, H - 1);", None),
    "remap_unclamped_neighbour_offset": ("int sc = clampi(fc - (qc - c), 0, W - 1);", "int sc = clampi(fc - b, 0, W - 1);", None),
    "remap_rows_and_columns_swapped": ("int fr = clampi(nnf[2 * q], 0, H - 1), fc = clampi(nnf[2 * q + 1], 0, W - 1);",
                                       "int fr = clampi(nnf[2 * q + 1], 0, H - 1), fc = clampi(nnf[2 * q], 0, W - 1);", None),
    "remap_divisor_off_by_one": ("float den = (float)(255 * k * k);\n    for (size_t i = 0; i < n; ++i)",
                                 "float den = (float)(255 * k * k + 1);\n    for (size_t i = 0; i < n; ++i)", None),
    "downsample_drops_second_row": ("int r0 = 2 * r, r1 = clampi(2 * r + 1, 0, H - 1);",
                                    "int r0 = 2 * r, r1 = clampi(2 * r, 0, H - 1);", None),
    "interpolation_single_key_weight": ("fbref_pair_tag(l, i), 1u, acc);", "fbref_pair_tag(l, i), 2u, acc);", None),
    "shat_rounds_down": ("shat[t] = (uint8_t)((v[t] + kk / 2) / kk);", "shat[t] = (uint8_t)(v[t] / kk);", None),
    "balanced_alpha_on_style_term": ("return alpha * fbref_ssd(gs, gt, H, W, k, ur, uc, xr, xc) +\n           fbref_ssd(ss, shat, H, W, k, ur, uc, xr, xc);",
                                     "return fbref_ssd(gs, gt, H, W, k, ur, uc, xr, xc) +\n           alpha * fbref_ssd(ss, shat, H, W, k, ur, uc, xr, xc);", None),
    "balanced_guide_term_on_style_image": ("return alpha * fbref_ssd(gs, gt,", "return alpha * fbref_ssd(ss, gt,", None),
    "balanced_style_term_against_target_guide": ("           fbref_ssd(ss, shat, H, W, k, ur, uc, xr, xc);", "           fbref_ssd(ss, gt, H, W, k, ur, uc, xr, xc);", None),
    "balanced_error_not_reevaluated": ("                E[x] = balanced_loss(", "                if (it == 0) E[x] = balanced_loss(", None),
    "balanced_shat_not_refreshed": ("        fbref_shat(src_style, F, h, w, k, shat);", "        if (it == 0) fbref_shat(src_style, F, h, w, k, shat);", None),
    "balanced_propagation_row_offset_sign": ("int cr = clampi(F[2 * n] - dirs[d][0], 0, h - 1);",
                                             "int cr = clampi(F[2 * n] + dirs[d][0], 0, h - 1);", 1),
    "balanced_random_search_skips_largest_radius": ("int rad = r0 >> t;", "int rad = r0 >> (t + 1);", 1),
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


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new, which = MUTANTS[name]
    with open(SRC) as f:
        src = f.read()
    mutant_c = tmp_path / "fbref_mutant.c"
    mutant_c.write_text(mutate(src, old, new, which))
    lib = tmp_path / "libfbref_mutant.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                    "-I", os.path.join(ROOT, "oracle"), "-o", str(lib), str(mutant_c)], check=True)
    env = dict(os.environ, FBREF_TEST_LIBRARY=str(lib), OMP_NUM_THREADS="4")
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                          os.path.join(ROOT, "tests", "test_oracle_balanced.py")],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 1, f"no pin failed for mutant {name}:\n{res.stdout[-1500:]}"
