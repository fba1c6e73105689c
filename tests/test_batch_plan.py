"""Host-side planning of batched submissions (no GPU): pair counts, work items and
chunking of fb_batch_plan, and its argument checks."""
import pytest

import paper_2311_09265_b300 as fbp
import synth
from paper_2311_09265_b300 import _build


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def expected_pairs(N, window):
    M = (window - 1) // 2
    return sum(min(N - 1, i + M) - max(0, i - M) for i in range(N))


def expected_items(H, W):
    return ((W + 31) // 32) * ((H + 7) // 8)


def test_plan_counts_every_pair_and_tile():
    shapes = [(5, 40, 52, 3, 5), (6, 33, 64, 5, 7), (4, 64, 48, 7, 3), (3, 48, 48, 1, 5)]
    p = fbp.Params.make(5, 2)
    n_pairs, n_items, n_chunks = fbp.fb_batch_plan(shapes, p)
    assert n_pairs == sum(expected_pairs(N, w) for N, H, W, w, k in shapes)
    assert n_items == sum(expected_pairs(N, w) * expected_items(H, W) for N, H, W, w, k in shapes)
    assert n_chunks == 3                       # one per patch size present


def test_plan_splits_into_chunks_under_a_small_budget():
    shapes = [(10, 64, 64, 5, 5)]
    p = fbp.Params.make(5, 2)
    per_pair = 64 * 64 * 16
    pairs = expected_pairs(10, 5)
    _, _, one = fbp.fb_batch_plan(shapes, p)
    assert one == 1
    _, _, many = fbp.fb_batch_plan(shapes, p, budget_bytes=4 * per_pair)
    # a chunk holds whole output frames (at most 4 NNFs each) within 4 NNFs of scratch
    assert many >= (pairs + 3) // 4 and many <= 10
    with pytest.raises(fbp.FastBlendError) as e:
        fbp.fb_batch_plan(shapes, p, budget_bytes=3 * per_pair)   # a full window needs 4
    assert e.value.status == fbp.FB_ERR_OOM


def test_plan_of_the_32_clip_manifest():
    m = synth.batch_manifest()
    assert len(m) == 32
    for N, H, W, w, k in m:
        assert 256 <= H <= 1024 and 256 <= W <= 1024 and H % 64 == 0 and W % 64 == 0
        assert 16 <= N <= 120 and w % 2 == 1 and 5 <= w <= 31 and k in (5, 7)
    n_pairs, _, n_chunks = fbp.fb_batch_plan(m, fbp.Params.make(5, 6))
    assert n_pairs == sum(expected_pairs(N, w) for N, H, W, w, k in m)
    assert n_chunks > 2


def test_plan_argument_checks():
    p = fbp.Params.make(5, 2)
    bad = [
        ([(5, 40, 52, 4, 5)], p),                 # even window
        ([(5, 40, 52, 3, 4)], p),                 # even patch
        ([(0, 40, 52, 3, 5)], p),                 # no frames
        ([(5, 4, 52, 3, 5)], p),                  # smaller than the patch
    ]
    for shapes, params in bad:
        with pytest.raises(fbp.FastBlendError) as e:
            fbp.fb_batch_plan(shapes, params)
        assert e.value.status == fbp.FB_ERR_ARG
    with pytest.raises(fbp.FastBlendError) as e:
        fbp.fb_batch_plan([(5, 40, 52, 3, 5)], fbp.Params.make(5, 2, levels=2))
    assert e.value.status == fbp.FB_ERR_UNSUPPORTED
