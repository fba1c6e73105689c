"""Host-side planning of the fast mode (fb_fast_plan, no GPU)."""
import pytest

import paper_2311_09265_b300 as fbp


def direct_nnfs(N, window):
    M = (window - 1) // 2
    return sum(min(N - 1, i + M) - max(0, i - M) for i in range(N))


def test_hand_worked_four_frames_window_three():
    # left pieces give (0->1), (1->2), (2->3); the reversed clip gives (1->0), (2->1), (3->2)
    n, e, pc = fbp.fb_fast_plan(4, 3)
    assert n == 6


def test_window_one_needs_no_nnf():
    n, e, pc = fbp.fb_fast_plan(16, 1)
    assert n == 0 and e == 32 and pc == 32     # one identity piece per side and frame


@pytest.mark.parametrize("N,window", [(60, 15), (60, 31), (120, 31), (100, 63)])
def test_fewer_nnfs_than_the_direct_sum_for_wide_windows(N, window):
    n, _, _ = fbp.fb_fast_plan(N, window)
    assert n < direct_nnfs(N, window)


def test_nnfs_grow_as_n_log_n_not_n_times_window():
    # Doubling the window from 31 to 63 adds about two NNFs per frame (one more level per
    # side), while the direct sum doubles.
    a, _, _ = fbp.fb_fast_plan(200, 31)
    b, _, _ = fbp.fb_fast_plan(200, 63)
    assert b - a < 4 * 200
    assert direct_nnfs(200, 63) - direct_nnfs(200, 31) > 25 * 200


def test_plan_argument_errors():
    for N, w in ((0, 3), (70000, 3), (10, 0), (10, 4)):
        with pytest.raises(fbp.FastBlendError):
            fbp.fb_fast_plan(N, w)
