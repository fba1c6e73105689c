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


def test_conv_and_its_gradients_equal_the_library_convolution():
    """The special case that reduces to a library routine: oracle conv3x3 (NHWC, weights
    [Cout][3][3][Cin]) equals torch's 2-D cross-correlation with zero padding 1 in float64,
    and conv3x3_backward equals autograd's input, weight and bias gradients -- for an
    asymmetric kernel (a transposed tap order or a mirrored offset would differ) at
    strides 1 and 2 on odd sizes."""
    import torch
    import torch.nn.functional as TF
    rng = np.random.default_rng(3)
    for stride, (H, W) in ((1, (7, 9)), (2, (7, 9)), (2, (8, 6))):
        x = rng.normal(size=(2, H, W, 8))
        w = rng.normal(size=(16, 3, 3, 8))
        b = rng.normal(size=16)
        y = ref.conv3x3(x, w, b, stride)
        xt = torch.tensor(x.transpose(0, 3, 1, 2), requires_grad=True)
        wt = torch.tensor(w.transpose(0, 3, 1, 2), requires_grad=True)
        bt = torch.tensor(b, requires_grad=True)
        yt = TF.conv2d(xt, wt, bt, stride=stride, padding=1)
        assert y.shape == tuple(yt.permute(0, 2, 3, 1).shape)
        assert np.allclose(y, yt.detach().numpy().transpose(0, 2, 3, 1), atol=1e-10)
        dz = rng.normal(size=y.shape)
        yt.backward(torch.tensor(dz.transpose(0, 3, 1, 2)))
        dx, dw, db = ref.conv3x3_backward(x, w, dz, stride)
        assert np.allclose(dx, xt.grad.numpy().transpose(0, 2, 3, 1), atol=1e-10)
        assert np.allclose(dw, wt.grad.numpy().transpose(0, 2, 3, 1), atol=1e-10)
        assert np.allclose(db, bt.grad.numpy(), atol=1e-10)


def test_network_input_closed_forms():
    """Box means of constant images map 0 -> -0.5 and 255 -> +0.5; a 2x2 checkerboard of
    0/255 averages to 127.5 -> 0 at downscale 4; the two spare channels are zero."""
    n, H, W = 1, 16, 16
    src = np.zeros((n, H, W, 3), np.uint8)
    tgt = np.full((n, H, W, 3), 255, np.uint8)
    x = ref.net_input(src, tgt, ds=4)
    assert x.shape == (1, 4, 4, 8)
    assert (x[..., 0:3] == -0.5).all() and (x[..., 3:6] == 0.5).all() and (x[..., 6:] == 0).all()
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    chk = np.repeat((((rr + cc) % 2) * 255).astype(np.uint8)[None, :, :, None], 3, axis=3)
    x = ref.net_input(chk, chk, ds=4)
    assert (x[..., :6] == 0).all()


def test_offset_loss_closed_forms():
    """Smooth-L1 (delta one pixel) of 16 * head against the target: zero at the target,
    0.5 d^2 inside one pixel, |d| - 0.5 outside, weights and their sum applied."""
    head = np.zeros((1, 2, 2, 8))
    target = np.zeros((1, 2, 2, 2))
    target[0, 0, 0] = (16.0, -32.0)          # head = target / 16 gives zero there
    head[0, 0, 0, :2] = (1.0, -2.0)
    target[0, 0, 1] = (0.5, 0.0)             # d = -0.5  -> 0.125
    target[0, 1, 0] = (3.0, 0.0)             # d = -3    -> 2.5
    weight = np.array([[[1.0, 1.0], [1.0, 0.0]]])
    loss, g = ref.loss_and_grad_head(head, target, weight, 2.0)
    assert np.isclose(loss, (0.0 + 0.125 + 2.5) / 2.0)
    assert np.isclose(g[0, 0, 1, 0], -0.5 * 16 / 2.0) and np.isclose(g[0, 1, 0, 0], -1.0 * 16 / 2.0)
    assert (g[0, 0, 0] == 0).all() and (g[..., 2:] == 0).all()
