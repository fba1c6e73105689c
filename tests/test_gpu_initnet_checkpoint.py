"""Checkpoint / resume of the learned initialiser's training: parameters, Adam state, the
schedule step and the batch sampler survive a save and a load into a fresh network."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2311_09265_b300 as fbp
    from paper_2311_09265_b300 import initnet_train as it
    fbp.build()
    ctx = fbp.Context(0)
    ts = it.make_training_set(ctx, n_clips=1, frames=6, H=128, W=128, pairs_per_clip=16,
                              target_iters=12, seed=4321)
    assert float(ts.weight.sum()) > 0     # some blocks have coherent targets: a gradient
    yield fbp, it, ctx, ts
    ctx.close()


def fresh(fbp, it, ctx):
    net = fbp.InitNet(ctx, 8, 128, 128, downscale=8)
    net.set_params(it.initial_params(net.n_params, 7))
    return net


def test_optimizer_state_round_trips(setup):
    fbp, it, ctx, ts = setup
    a = fresh(fbp, it, ctx)
    it.train(a, ts, steps=6, batch_size=4, warmup=2, seed=1, log_every=3)
    m, v, n = a.get_optimizer()
    assert n == 6 and np.abs(m).sum() > 0 and (v >= 0).all() and v.sum() > 0
    b = fresh(fbp, it, ctx)
    b.set_optimizer(m, v, n)
    m2, v2, n2 = b.get_optimizer()
    assert np.array_equal(m, m2) and np.array_equal(v, v2) and n2 == n
    b.set_params(a.get_params())     # setting parameters resets the Adam state
    assert b.get_optimizer()[2] == 0 and not b.get_optimizer()[0].any()
    with pytest.raises(ValueError):
        b.set_optimizer(m[:-1], v, n)
    a.close()
    b.close()


def test_resumed_training_follows_the_uninterrupted_run(setup, tmp_path):
    fbp, it, ctx, ts = setup
    kw = dict(steps=20, batch_size=4, lr=1e-3, warmup=4, log_every=5)
    whole = fresh(fbp, it, ctx)
    it.train(whole, ts, seed=3, **kw)
    first = fresh(fbp, it, ctx)
    rng = np.random.default_rng(3)
    it.train(first, ts, stop=10, rng=rng, **kw)
    path = str(tmp_path / "ckpt.npz")
    it.save_checkpoint(first, path, 10, rng)
    resumed = fresh(fbp, it, ctx)
    step, rng2 = it.load_checkpoint(resumed, path)
    assert step == 10 and resumed.get_optimizer()[2] == 10
    assert np.array_equal(resumed.get_params(), first.get_params())
    it.train(resumed, ts, start=step, rng=rng2, **kw)
    p_whole, p_res = whole.get_params(), resumed.get_params()
    # Every gradient is a sum in a fixed order (the weight gradient's per-split slices and
    # the bias gradient's per-block partials are added in index order, no atomics), so a
    # training run is reproducible bit for bit -- and a resumed one equals the uninterrupted
    # run exactly, Adam state included.
    again = fresh(fbp, it, ctx)
    it.train(again, ts, seed=3, **kw)
    assert np.array_equal(again.get_params(), p_whole)
    assert np.array_equal(p_res, p_whole)
    for x, y in zip(resumed.get_optimizer(), whole.get_optimizer()):
        assert np.array_equal(x, y)
    # Restarting from the parameters alone (fresh Adam state, schedule from step 0) does not.
    rel = lambda a: float(np.linalg.norm(a - p_whole) / np.linalg.norm(p_whole))  # noqa: E731
    cold = fresh(fbp, it, ctx)
    cold.set_params(first.get_params())
    it.train(cold, ts, stop=10, rng=np.random.default_rng(3), **kw)
    cold_drift = rel(cold.get_params())
    print(f"cold-restart drift {cold_drift:.3g}")
    assert cold_drift > 1e-2
    for n in (whole, first, resumed, again, cold):
        n.close()
