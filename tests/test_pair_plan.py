"""Pair enumeration (a1) as the blend and interpolation calls perform it, checked on the
host against the definitions: Eq. 2's window (Sec. 3.4), the key pairs and Eq. 9 weights
of Sec. 3.5.2, and the chain neighbours (Sec. 3.5.1) and partners (Eq. 10) the tracking
and alignment kernels read.  No GPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402


@pytest.fixture(scope="module")
def fbp():
    import paper_2311_09265_b300 as m
    m.build()
    return m


def _brute_blend(N, window):
    M = (window - 1) // 2
    return [(j, i, 1) for i in range(N) for j in range(N) if j != i and abs(i - j) <= M]


def _brute_interp(N, keys):
    out = []
    for i in range(N):
        if i in keys:
            continue
        left = [k for k in keys if k < i]
        right = [k for k in keys if k > i]
        if left and right:
            l, r = max(left), min(right)
            out += [(l, i, r - i), (r, i, i - l)]
        else:
            out.append(((max(left) if left else min(right)), i, 1))
    return out


def _check_links(plan, tracking, align):
    index = {(p["src"], p["tgt"]): q for q, p in enumerate(plan)}
    for q, p in enumerate(plan):
        want_prev = index.get((p["src"], p["tgt"] - 1), -1) if tracking else -1
        want_next = index.get((p["src"], p["tgt"] + 1), -1) if tracking else -1
        assert (p["prev"], p["next"]) == (want_prev, want_next), p
        others = [r for r, o in enumerate(plan) if o["tgt"] == p["tgt"] and r != q]
        assert p["partner"] == (others[0] if align and others else -1), p
        if p["partner"] >= 0:
            assert plan[p["partner"]]["partner"] == q


@pytest.mark.parametrize("N,window", [(1, 1), (1, 15), (2, 3), (5, 1), (8, 3), (9, 5), (16, 15),
                                      (60, 15), (7, 31)])
@pytest.mark.parametrize("tracking", [False, True])
def test_blend_pairs(fbp, N, window, tracking):
    plan = fbp.fb_pair_plan(N, window, flags=fbp.FB_FLAG_TRACKING if tracking else 0)
    got = [(p["src"], p["tgt"], p["weight"]) for p in plan]
    assert got == _brute_blend(N, window)
    assert all(p["tag"] == oracle.pair_tag(p["src"], p["tgt"]) and p["out_frame"] == p["tgt"] for p in plan)
    _check_links(plan, tracking, False)


@pytest.mark.parametrize("N,keys", [(48, (0, 47)), (10, (2, 5, 7)), (6, (3,)), (5, (0, 1, 2, 3, 4)),
                                    (9, (0, 4, 8)), (7, (6,)), (1, (0,)), (12, (1, 2, 10))])
@pytest.mark.parametrize("flags", ["", "T", "A", "TA"])
def test_interpolation_pairs(fbp, N, keys, flags):
    f = (fbp.FB_FLAG_TRACKING if "T" in flags else 0) | (fbp.FB_FLAG_ALIGN if "A" in flags else 0)
    plan = fbp.fb_pair_plan(N, 0, list(keys), flags=f)
    got = [(p["src"], p["tgt"], p["weight"]) for p in plan]
    assert got == _brute_interp(N, keys)
    assert all(p["tag"] == oracle.pair_tag(p["src"], p["tgt"]) for p in plan)
    _check_links(plan, "T" in flags, "A" in flags)


def test_pair_plan_argument_errors(fbp):
    bad = [lambda: fbp.fb_pair_plan(0, 3), lambda: fbp.fb_pair_plan(5, 4),
           lambda: fbp.fb_pair_plan(5, 3, [0]), lambda: fbp.fb_pair_plan(5, 0, []),
           lambda: fbp.fb_pair_plan(5, 0, [3, 1]), lambda: fbp.fb_pair_plan(5, 0, [0, 5]),
           lambda: fbp.fb_pair_plan(5, 3, flags=fbp.FB_FLAG_ALIGN),
           lambda: fbp.fb_pair_plan(5, 3, flags=fbp.FB_FLAG_BALANCED)]
    for f in bad:
        with pytest.raises(fbp.FastBlendError) as ei:
            f()
        assert ei.value.status == fbp.FB_ERR_ARG
