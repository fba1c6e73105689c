"""Pins of the learned-initialiser oracle (oracle/initnet.py) on the CPU: gradients
against central finite differences, closed forms of the convolution."""
import numpy as np

from oracle import initnet as ref


def test_bf16_rounding_is_round_to_nearest_even():
    vals = np.array([1.0, 1.00390625, 1.005859375, 1.0078125, -3.0, 1e-3], np.float64)
    r = ref.bf16(vals)
    assert r[0] == 1.0 and r[4] == -3.0
    assert r[1] == 1.0                      # halfway 1 + 2^-8 -> even mantissa (1.0)
    assert r[2] == 1.0078125                # above halfway rounds up
    assert abs(r[5] - 1e-3) / 1e-3 < 2 ** -8


def test_identity_kernel_copies_the_input():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 5, 7, 8))
    w = np.zeros((8, 3, 3, 8))
    w[:, 1, 1, :] = np.eye(8)
    assert np.allclose(ref.conv3x3(x, w, np.zeros(8), 1), x)
    y2 = ref.conv3x3(x, w, np.zeros(8), 2)
    assert y2.shape == (2, 3, 4, 8) and np.allclose(y2, x[:, ::2, ::2])


def test_shift_kernel_and_zero_padding():
    x = np.arange(1 * 4 * 4 * 8, dtype=np.float64).reshape(1, 4, 4, 8)
    w = np.zeros((8, 3, 3, 8))
    w[:, 0, 0, :] = np.eye(8)               # tap (-1, -1): y[r, c] = x[r-1, c-1]
    y = ref.conv3x3(x, w, np.zeros(8), 1)
    assert np.all(y[:, 0, :] == 0) and np.all(y[:, :, 0] == 0)
    assert np.allclose(y[:, 1:, 1:], x[:, :-1, :-1])


def test_conv_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    for stride in (1, 2):
        x = rng.normal(size=(2, 5, 6, 8))
        w = rng.normal(size=(8, 3, 3, 8)) * 0.3
        b = rng.normal(size=8)
        dz = rng.normal(size=ref.conv3x3(x, w, b, stride).shape)
        dx, dw, db = ref.conv3x3_backward(x, w, dz, stride)
        f = lambda xx, ww, bb: float((ref.conv3x3(xx, ww, bb, stride) * dz).sum())
        eps = 1e-6
        for _ in range(12):
            i = tuple(rng.integers(0, s) for s in x.shape)
            xp, xm = x.copy(), x.copy()
            xp[i] += eps
            xm[i] -= eps
            assert abs((f(xp, w, b) - f(xm, w, b)) / (2 * eps) - dx[i]) < 1e-5
            j = tuple(rng.integers(0, s) for s in w.shape)
            wp, wm = w.copy(), w.copy()
            wp[j] += eps
            wm[j] -= eps
            assert abs((f(x, wp, b) - f(x, wm, b)) / (2 * eps) - dw[j]) < 1e-5
        bp = b.copy()
        bp[3] += eps
        bm = b.copy()
        bm[3] -= eps
        assert abs((f(x, w, bp) - f(x, w, bm)) / (2 * eps) - db[3]) < 1e-5


def test_network_gradient_matches_finite_differences_of_its_loss():
    # Without bf16 rounding in the loop, the network's backward is the exact gradient.
    rng = np.random.default_rng(2)
    saved = ref.bf16
    ref.bf16 = lambda a: np.asarray(a, dtype=np.float64)
    try:
        src = rng.integers(0, 256, size=(1, 32, 32, 3)).astype(np.uint8)
        tgt = rng.integers(0, 256, size=(1, 32, 32, 3)).astype(np.uint8)
        params = ref.init_params(3)
        params[-8 * 9 * 32 - 8:] = rng.normal(0, 0.05, size=8 * 9 * 32 + 8)   # make the head live
        target = rng.normal(0, 3, size=(1, 8, 8, 2))
        head, cache = ref.forward(params, src, tgt)
        loss, dhead = ref.loss_and_grad_head(head, target, None, 64.0)
        g = ref.backward(cache, dhead)
        def L(p):
            h, _ = ref.forward(p, src, tgt)
            return ref.loss_and_grad_head(h, target, None, 64.0)[0]
        eps = 1e-6
        idx = rng.choice(np.nonzero(np.abs(g) > 1e-4)[0], size=10, replace=False)
        for i in idx:
            p1, p2 = params.copy(), params.copy()
            p1[i] += eps
            p2[i] -= eps
            num = (L(p1) - L(p2)) / (2 * eps)
            assert abs(num - g[i]) <= 1e-4 * max(1.0, abs(g[i])), (i, num, g[i])
    finally:
        ref.bf16 = saved
    assert ref.n_params() == 779592
