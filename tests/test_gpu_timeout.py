"""Failure detection on the GPU without a fault: the tensor-core kernels' bounded waits.

Every wait of the learned initialiser's kernels on an mbarrier is bounded.  When a
progress wait (operands landed, a stage free, the accumulator complete) gives up, the CTA
lets the MMAs it committed and the copies it issued finish (those drain waits keep the
full limit), skips its epilogue, releases its tensor memory and raises the timeout flag.
Here the progress limit is set to zero polls, so every such wait gives up at once:
each kernel family (the TMA-fed forward and gradients, the cp.async-gathered forward and
input gradient, the synchronous weight gradient, and a whole forward pass of the network)
must report the timeout, the device must stay usable, and once the limit is restored
the same calls must give the results they gave before.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbp():
    import paper_2311_09265_b300 as m
    m.build()
    return m


@pytest.fixture
def expire(fbp):
    """Every progress wait gives up at once inside the block; the default afterwards."""
    import contextlib

    @contextlib.contextmanager
    def ctx():
        fbp.fb_debug_set_wait_limit(0)
        try:
            yield
        finally:
            fbp.fb_debug_set_wait_limit(-1)
    return ctx


def _layer(seed, n, H, W, Cin, Cout):
    import torch
    g = torch.Generator().manual_seed(seed)
    x = torch.randn((n, H, W, Cin), generator=g).to(torch.bfloat16).cuda()
    w = (torch.randn((Cout, 3, 3, Cin), generator=g) / (3 * Cin ** 0.5)).to(torch.bfloat16).cuda()
    b = torch.randn(Cout, generator=g).cuda()
    return x, w, b


@pytest.mark.parametrize("path", [0, 1, 2])   # 0: TMA, row reuse; 1: cp.async gathers; 2: TMA per tap
def test_forward_layer_times_out_then_recovers(fbp, expire, path):
    import torch
    x, w, b = _layer(11 + path, 2, 32, 32, 64, 64)
    old = fbp.fb_conv_gemm_path(path)
    try:
        ref, st = fbp.conv3x3_forward(x, w, b, 1, True, out_f32=True)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        tma0 = fbp.fb_conv_gemm_path(-1)
        with expire():
            _, st = fbp.conv3x3_forward(x, w, b, 1, True, out_f32=True)
            torch.cuda.synchronize()
        assert int(st.item()) == 1
        if path != 1:
            assert fbp.fb_conv_gemm_path(-1) > tma0      # the TMA-fed kernel is the one that ran
        again, st = fbp.conv3x3_forward(x, w, b, 1, True, out_f32=True)
        torch.cuda.synchronize()
        assert int(st.item()) == 0 and torch.equal(again, ref)
    finally:
        fbp.fb_conv_gemm_path(0)


@pytest.mark.parametrize("path", [0, 1, 2])   # 0, 2: TMA-fed gradients, 1: gathered
def test_backward_layer_times_out_then_recovers(fbp, expire, path):
    """The input gradient and the weight gradient: the weight gradient alone, then both."""
    import torch
    x, w, _ = _layer(21, 2, 16, 16, 32, 64)
    wt = w.permute(3, 1, 2, 0).contiguous()
    g = torch.Generator().manual_seed(5)
    dz = torch.randn((2, 16, 16, 64), generator=g).to(torch.bfloat16).cuda()
    old = fbp.fb_conv_gemm_path(path)
    try:
        dx0, dw0, st = fbp.conv3x3_backward(x, wt, dz, 1)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        for input_grad in (False, True):
            tma0 = fbp.fb_conv_gemm_path(-1)
            with expire():
                _, _, st = fbp.conv3x3_backward(x, wt, dz, 1, input_grad=input_grad)
                torch.cuda.synchronize()
            assert int(st.item()) == 1
            if path != 1:
                assert fbp.fb_conv_gemm_path(-1) > tma0   # the TMA-fed kernels are the ones that ran
        dx1, dw1, st = fbp.conv3x3_backward(x, wt, dz, 1)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert torch.equal(dx1, dx0)
        assert torch.equal(dw1, dw0)   # the splits are added in a fixed order
    finally:
        fbp.fb_conv_gemm_path(0)


def test_stride2_input_gradient_times_out_then_recovers(fbp, expire):
    """The parity-class input gradient of a stride-2 layer (TMA-fed)."""
    import torch
    x, w, _ = _layer(31, 2, 32, 32, 32, 64)
    wt = w.permute(3, 1, 2, 0).contiguous()
    g = torch.Generator().manual_seed(7)
    dz = torch.randn((2, 16, 16, 64), generator=g).to(torch.bfloat16).cuda()
    dx0, _, st = fbp.conv3x3_backward(x, wt, dz, 2, weight_grad=False)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    tma0 = fbp.fb_conv_gemm_path(-1)
    with expire():
        _, _, st = fbp.conv3x3_backward(x, wt, dz, 2, weight_grad=False)
        torch.cuda.synchronize()
    assert int(st.item()) == 1 and fbp.fb_conv_gemm_path(-1) > tma0
    dx1, _, st = fbp.conv3x3_backward(x, wt, dz, 2, weight_grad=False)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and torch.equal(dx1, dx0)


def test_network_forward_reports_timeout_then_recovers(fbp, expire):
    import torch

    import synth
    from paper_2311_09265_b300 import initnet_train as it
    ctx = fbp.Context(0)
    net = fbp.InitNet(ctx, 2, 128, 128, downscale=8)
    net.set_params(it.initial_params(net.n_params, 3))
    g, _ = synth.small_clip(3, 128, 128, seed=77, motion="affine")
    src = torch.from_numpy(np.ascontiguousarray(g[[0, 1]])).cuda()
    tgt = torch.from_numpy(np.ascontiguousarray(g[[1, 2]])).cuda()
    ref = net.forward(src, tgt).clone()
    torch.cuda.synchronize()
    assert net.status() == fbp.FB_OK
    with expire():
        net.forward(src, tgt)
        torch.cuda.synchronize()
    assert net.status() == fbp.FB_ERR_TIMEOUT
    assert net.status() == fbp.FB_OK              # reported once, then cleared
    again = net.forward(src, tgt)
    torch.cuda.synchronize()
    assert net.status() == fbp.FB_OK and torch.equal(again, ref)
    net.close()
    ctx.close()
