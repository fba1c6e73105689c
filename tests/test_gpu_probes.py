"""The roofline probes bench.py divides by: each runs, reports a rate within what one B300
can do, and rejects arguments it does not measure.  (The rates themselves are reported by
bench.py, not asserted: they depend on the clock the GPU runs at.)"""
import pytest

pytestmark = pytest.mark.gpu

SMS, MAX_CLK = 148, 2.1e9   # an upper bound on any rate per SM-clock below


@pytest.fixture(scope="module")
def ctx():
    import paper_2311_09265_b300 as fbp
    fbp.build()
    c = fbp.Context(0)
    yield fbp, c
    c.close()


def test_dp4a_probe_is_below_its_issue_limit(ctx):
    fbp, c = ctx
    rate, ms = c.probe_dp4a()
    assert ms > 0 and 0 < rate <= 64 * SMS * MAX_CLK


@pytest.mark.parametrize("patch", [5, 7])
def test_ssd_mix_probe_is_below_the_dp4a_bound(ctx, patch):
    fbp, c = ctx
    rate, ms = c.probe_ssd_mix(patch)
    assert ms > 0 and 0 < rate <= 64 * 4 * SMS * MAX_CLK


def test_gather_probe_rates(ctx):
    """Scattered 32-byte loads: at most a few sectors per SM-clock from an L1-resident buffer,
    and no faster from one that spills to L2."""
    fbp, c = ctx
    l1, ms1 = c.probe_gather(64 * 1024)
    l2, ms2 = c.probe_gather(4 * 1024 * 1024)
    assert ms1 > 0 and ms2 > 0
    assert 0 < l1 <= 4 * SMS * MAX_CLK and 0 < l2 <= 4 * SMS * MAX_CLK
    assert l2 <= 2 * l1


@pytest.mark.parametrize("nbytes", [0, 1000, 3 * 1024, 2 << 30])
def test_gather_probe_rejects_sizes_that_are_not_powers_of_two_in_range(ctx, nbytes):
    fbp, c = ctx
    with pytest.raises(fbp.FastBlendError) as e:
        c.probe_gather(nbytes)
    assert e.value.status == fbp.FB_ERR_ARG


def test_ssd_mix_probe_rejects_other_patches(ctx):
    fbp, c = ctx
    with pytest.raises(fbp.FastBlendError):
        c.probe_ssd_mix(3)
