"""The TMA-staged convolutions against the gathered kernels of the same GEMMs and the
FP64 CPU oracle.  Forward (tiled TMA loads of the activation box displaced per tap and
strided by the layer's stride, and of the weight box, tcgen05 MMAs) and stride-1 input
gradient: the same products in the same order as the gather path, so bit-identical.
Weight gradient (both operands MN-major): the same products in another order, so equal to
fp32 rounding.  Layers whose boxes do not tile run the gathered kernels."""
import numpy as np
import pytest

from oracle import initnet as ref

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbp():
    import paper_2311_09265_b300 as m
    m.build()
    yield m
    m.fb_conv_gemm_path(0)


def to_bf16_tensor(a):
    import torch
    return torch.from_numpy(ref.bf16_bits(a).view(np.int16).copy()).view(torch.bfloat16).cuda()


def run(fbp, x, w, b, stride, relu, out_f32, mode):
    import torch
    fbp.fb_conv_gemm_path(mode)
    n0 = fbp.fb_conv_gemm_path(-1)
    y, st = fbp.conv3x3_forward(to_bf16_tensor(x), to_bf16_tensor(w),
                                torch.tensor(b, dtype=torch.float32, device="cuda"), stride, relu,
                                out_f32=out_f32)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return (y.float() if not out_f32 else y).cpu().numpy(), fbp.fb_conv_gemm_path(-1) - n0


TMA_CASES = [  # n, H, W, Cin, Cout, stride: the initialiser's layers at 512x512 / 8 and more
    (2, 64, 64, 32, 32, 1), (1, 64, 64, 8, 32, 1), (2, 32, 32, 64, 64, 1), (3, 16, 16, 96, 96, 1),
    (4, 8, 8, 128, 128, 1), (3, 8, 8, 128, 128, 1), (2, 16, 16, 224, 96, 1), (2, 32, 32, 160, 64, 1),
    (2, 64, 64, 96, 32, 1), (2, 64, 64, 32, 8, 1), (1, 4, 32, 40, 24, 1), (5, 4, 4, 16, 16, 1),
    (2, 64, 64, 32, 64, 2), (2, 32, 32, 64, 96, 2), (3, 16, 16, 96, 128, 2), (1, 16, 15, 32, 32, 2),
    (3, 8, 8, 64, 32, 2), (2, 32, 32, 16, 32, 1), (2, 16, 16, 56, 64, 2), (1, 8, 16, 48, 16, 1),
    (2, 16, 16, 24, 32, 1), (2, 8, 8, 192, 64, 1),
]


def rows_reuse(H, W, Cin, stride):
    """Whether the default path may run the row-reuse kernel: stride 1, tiles of whole rows
    of one image (128 output pixels per tile), a width divisible by 8 (and three stages
    fitting in shared memory, which these cases do unless the tile is 128 wide with
    64-channel blocks)."""
    return stride == 1 and (H * W) % 128 == 0 and 128 % W == 0 and W % 8 == 0 and Cin % 32 == 0


@pytest.mark.parametrize("n,H,W,Cin,Cout,stride", TMA_CASES)
def test_tma_conv_is_bit_identical_to_the_gather_path(fbp, n, H, W, Cin, Cout, stride):
    """One box per tap (mode 2) against the gathers (mode 1): bit-identical for Cin % 16 == 0.
    The default (mode 0; row reuse where it applies) against both: fp32 rounding."""
    rng = np.random.default_rng(n * 1000 + H * W + Cin + Cout)
    x = ref.bf16(rng.normal(size=(n, H, W, Cin)))
    w = ref.bf16(rng.normal(size=(Cout, 3, 3, Cin)) / np.sqrt(9 * Cin))
    b = rng.normal(size=Cout).astype(np.float32).astype(np.float64)
    # Columns of 16 or more channels give the gather path's K = 16 steps (16 channels of
    # one tap); 8-channel columns (Cin an odd multiple of 8) pair two taps in a step,
    # where the gather path pads each tap to 16: same products, other grouping.
    same_steps = Cin % 16 == 0
    for relu, out_f32 in ((False, True), (True, False)):
        yg, used_g = run(fbp, x, w, b, stride, relu, out_f32, mode=1)
        yt, used_t = run(fbp, x, w, b, stride, relu, out_f32, mode=2)
        yr, used_r = run(fbp, x, w, b, stride, relu, out_f32, mode=0)
        assert used_g == 0 and used_t == 1 and used_r == 1
        if same_steps:
            assert np.array_equal(yt.view(np.uint32) if out_f32 else yt, yg.view(np.uint32) if out_f32 else yg)
        elif out_f32:
            assert float(np.linalg.norm(yt - yg) / np.linalg.norm(yg)) < 1e-6
        if out_f32:
            assert float(np.linalg.norm(yr - yg) / np.linalg.norm(yg)) < 1e-6
            if not rows_reuse(H, W, Cin, stride):
                assert np.array_equal(yr.view(np.uint32), yt.view(np.uint32))
        else:   # bf16 outputs: at most one rounding step apart
            assert float(np.abs(yr - yg).max()) <= 2.0 ** -6 * max(1.0, float(np.abs(yg).max()))
    want = ref.conv3x3(x, w, b, stride)
    y32, _ = run(fbp, x, w, b, stride, False, True, mode=0)
    assert float(np.linalg.norm(y32 - want) / np.linalg.norm(want)) < 1e-5


@pytest.mark.parametrize("n,H,W,Cin,Cout,stride", [(2, 17, 23, 32, 64, 1), (2, 24, 24, 32, 32, 1),
                                                  (2, 48, 48, 32, 64, 2)])
def test_layers_the_tma_boxes_cannot_tile_use_the_gathers(fbp, n, H, W, Cin, Cout, stride):
    rng = np.random.default_rng(7)
    x = ref.bf16(rng.normal(size=(n, H, W, Cin)))
    w = ref.bf16(rng.normal(size=(Cout, 3, 3, Cin)) / np.sqrt(9 * Cin))
    b = rng.normal(size=Cout).astype(np.float32).astype(np.float64)
    y, used = run(fbp, x, w, b, stride, False, True, mode=0)
    assert used == 0
    want = ref.conv3x3(x, w, b, stride)
    assert float(np.linalg.norm(y - want) / np.linalg.norm(want)) < 1e-5


def test_gemm_path_argument_errors(fbp):
    for mode in (3, -2):
        with pytest.raises(fbp.FastBlendError):
            fbp.fb_conv_gemm_path(mode)


DGRAD_CASES = [  # n, H, W, Cin, Cout of stride-1 layers: the input gradient's boxes tile
    (2, 64, 64, 8, 32), (2, 64, 64, 32, 32), (2, 32, 32, 64, 64), (3, 16, 16, 96, 96),
    (4, 8, 8, 128, 128), (2, 64, 64, 96, 32), (2, 64, 64, 32, 8), (2, 32, 32, 40, 24),
    (2, 32, 32, 160, 64), (2, 16, 16, 224, 96),   # concatenated decoder inputs: two N tiles
]


@pytest.mark.parametrize("n,H,W,Cin,Cout", DGRAD_CASES)
def test_tma_input_gradient_is_bit_identical_to_the_gather_path(fbp, n, H, W, Cin, Cout):
    """Stride 1: the input gradient is the convolution of dZ with the tap-mirrored
    transposed weights, staged by TMA (boxes displaced by the mirrored taps); it must
    equal the cp.async gather path (same products, same order when Cout is a multiple of
    16) and the FP64 oracle."""
    import torch
    rng = np.random.default_rng(n * 7 + H + Cin * 3 + Cout)
    x = ref.bf16(rng.normal(size=(n, H, W, Cin)))
    w = ref.bf16(rng.normal(size=(Cout, 3, 3, Cin)) / np.sqrt(9 * Cin))
    dz = ref.bf16(rng.normal(size=(n, H, W, Cout)))
    wt = np.ascontiguousarray(np.transpose(w, (3, 1, 2, 0)))
    out = {}
    for mode in (1, 2, 0):
        fbp.fb_conv_gemm_path(mode)
        n0 = fbp.fb_conv_gemm_path(-1)
        dx, _, st = fbp.conv3x3_backward(to_bf16_tensor(x), to_bf16_tensor(wt), to_bf16_tensor(dz), 1,
                                         weight_grad=False)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        out[mode] = (dx.cpu().numpy(), fbp.fb_conv_gemm_path(-1) - n0)
    fbp.fb_conv_gemm_path(0)
    (dxg, used_g), (dxt, used_t), (dxr, used_r) = out[1], out[2], out[0]
    assert used_g == 0 and used_t == 1 and used_r == 1
    if Cout % 16 == 0:
        assert np.array_equal(dxt.view(np.uint32), dxg.view(np.uint32))
    else:
        assert float(np.linalg.norm(dxt - dxg) / np.linalg.norm(dxg)) < 1e-6
    # the default: the row-reuse kernel where the input gradient's geometry allows it
    assert float(np.linalg.norm(dxr - dxg) / np.linalg.norm(dxg)) < 1e-6
    if not rows_reuse(H, W, Cout, 1):
        assert np.array_equal(dxr.view(np.uint32), dxt.view(np.uint32))
    dx_ref, _, _ = ref.conv3x3_backward(x, w, dz, 1)
    assert float(np.linalg.norm(dxt - dx_ref) / np.linalg.norm(dx_ref)) < 1e-5
    assert float(np.linalg.norm(dxr - dx_ref) / np.linalg.norm(dx_ref)) < 1e-5


WGRAD_CASES = [  # n, H, W, Cin, Cout, stride: whole-row pixel chunks; channels padded to 32
    (2, 64, 64, 32, 32, 1), (2, 64, 64, 96, 32, 1), (2, 32, 32, 64, 64, 1), (3, 16, 16, 96, 96, 1),
    (4, 8, 8, 128, 128, 1), (2, 16, 16, 224, 96, 1), (2, 32, 32, 160, 64, 1), (2, 64, 64, 32, 64, 2),
    (2, 32, 32, 64, 96, 2), (3, 16, 16, 96, 128, 2), (2, 64, 64, 8, 32, 1), (2, 64, 64, 32, 8, 1),
    (2, 32, 32, 40, 24, 1), (1, 4, 32, 48, 16, 1), (3, 16, 16, 24, 8, 2),
]


@pytest.mark.parametrize("n,H,W,Cin,Cout,stride", WGRAD_CASES)
def test_tma_weight_gradient_matches_the_gather_path_and_the_oracle(fbp, n, H, W, Cin, Cout, stride):
    """The weight gradient with both operands MN-major, staged by TMA: the same products
    as the gathered kernel, summed in another order (tensor-core K steps, another split of
    the pixels), so equal to it up to fp32 rounding, and to the FP64 oracle.  Each path adds
    its splits in a fixed order, so a repeated call is bit-identical."""
    import torch
    rng = np.random.default_rng(n * 5 + H + Cin + 7 * Cout + stride)
    x = ref.bf16(rng.normal(size=(n, H, W, Cin)))
    w = ref.bf16(rng.normal(size=(Cout, 3, 3, Cin)) / np.sqrt(9 * Cin))
    Ho, Wo = ref.out_size(H, stride), ref.out_size(W, stride)
    dz = ref.bf16(rng.normal(size=(n, Ho, Wo, Cout)))
    out = {}
    for mode in (1, 0):
        fbp.fb_conv_gemm_path(mode)
        n0 = fbp.fb_conv_gemm_path(-1)
        _, dw, st = fbp.conv3x3_backward(to_bf16_tensor(x), None, to_bf16_tensor(dz), stride, input_grad=False)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        out[mode] = (dw.cpu().numpy(), fbp.fb_conv_gemm_path(-1) - n0)
        _, dw2, _ = fbp.conv3x3_backward(to_bf16_tensor(x), None, to_bf16_tensor(dz), stride, input_grad=False)
        assert np.array_equal(dw2.cpu().numpy(), out[mode][0])
    fbp.fb_conv_gemm_path(0)
    (dwg, used_g), (dwt, used_t) = out[1], out[0]
    assert used_g == 0 and used_t == 1
    assert float(np.linalg.norm(dwt - dwg) / np.linalg.norm(dwg)) < 2e-6
    _, dw_ref, _ = ref.conv3x3_backward(x, w, dz, stride)
    assert float(np.linalg.norm(dwt - dw_ref) / np.linalg.norm(dw_ref)) < 1e-5


@pytest.mark.parametrize("n,H,W,Cin,Cout,stride", [(3, 9, 11, 32, 8, 1), (2, 17, 23, 32, 64, 2)])
def test_weight_gradients_the_tma_boxes_cannot_tile_use_the_gathers(fbp, n, H, W, Cin, Cout, stride):
    import torch
    rng = np.random.default_rng(3)
    x = ref.bf16(rng.normal(size=(n, H, W, Cin)))
    Ho, Wo = ref.out_size(H, stride), ref.out_size(W, stride)
    dz = ref.bf16(rng.normal(size=(n, Ho, Wo, Cout)))
    n0 = fbp.fb_conv_gemm_path(-1)
    _, dw, st = fbp.conv3x3_backward(to_bf16_tensor(x), None, to_bf16_tensor(dz), stride, input_grad=False)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and fbp.fb_conv_gemm_path(-1) == n0
    w = np.zeros((Cout, 3, 3, Cin))
    _, dw_ref, _ = ref.conv3x3_backward(x, w, dz, stride)
    assert float(np.linalg.norm(dw.cpu().numpy() - dw_ref) / np.linalg.norm(dw_ref)) < 1e-5


S2_DGRAD_CASES = [  # n, H, W, Cin, Cout of stride-2 layers with even inputs: output-parity classes
    (2, 64, 64, 32, 64), (2, 32, 32, 64, 96), (3, 16, 16, 96, 128), (2, 64, 64, 32, 32), (2, 32, 64, 16, 64),
]


@pytest.mark.parametrize("n,H,W,Cin,Cout", S2_DGRAD_CASES)
def test_stride2_input_gradient_by_output_parity(fbp, n, H, W, Cin, Cout):
    """Stride 2: every parity class of dX is a stride-1 convolution of dZ with its one, two or
    four taps at displacements 0 or +1, staged by TMA (mode 0); the gathered path (mode 1)
    walks all nine taps: the same products in another order, so equal to fp32 rounding, and
    both equal the FP64 oracle."""
    import torch
    rng = np.random.default_rng(n * 11 + H + W + Cin + Cout)
    x = ref.bf16(rng.normal(size=(n, H, W, Cin)))
    w = ref.bf16(rng.normal(size=(Cout, 3, 3, Cin)) / np.sqrt(9 * Cin))
    dz = ref.bf16(rng.normal(size=(n, H // 2, W // 2, Cout)))
    wt = np.ascontiguousarray(np.transpose(w, (3, 1, 2, 0)))
    out = {}
    for mode in (1, 0):
        fbp.fb_conv_gemm_path(mode)
        n0 = fbp.fb_conv_gemm_path(-1)
        dx, _, st = fbp.conv3x3_backward(to_bf16_tensor(x), to_bf16_tensor(wt), to_bf16_tensor(dz), 2,
                                         weight_grad=False)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        out[mode] = (dx.cpu().numpy(), fbp.fb_conv_gemm_path(-1) - n0)
    fbp.fb_conv_gemm_path(0)
    (dxg, used_g), (dxt, used_t) = out[1], out[0]
    assert used_g == 0 and used_t == 1
    assert float(np.linalg.norm(dxt - dxg) / np.linalg.norm(dxg)) < 1e-6
    dx_ref, _, _ = ref.conv3x3_backward(x, w, dz, 2)
    assert float(np.linalg.norm(dxt - dx_ref) / np.linalg.norm(dx_ref)) < 1e-5


@pytest.mark.parametrize("n,H,W,Cin,Cout", [(2, 32, 32, 32, 24), (2, 34, 34, 32, 64), (2, 33, 32, 32, 64)])
def test_stride2_input_gradients_the_parity_kernel_cannot_take_use_the_gathers(fbp, n, H, W, Cin, Cout):
    """Cout not a multiple of 32, a row width that does not tile, or an odd input size."""
    import torch
    rng = np.random.default_rng(5)
    x = ref.bf16(rng.normal(size=(n, H, W, Cin)))
    w = ref.bf16(rng.normal(size=(Cout, 3, 3, Cin)) / np.sqrt(9 * Cin))
    Ho, Wo = ref.out_size(H, 2), ref.out_size(W, 2)
    dz = ref.bf16(rng.normal(size=(n, Ho, Wo, Cout)))
    wt = np.ascontiguousarray(np.transpose(w, (3, 1, 2, 0)))
    n0 = fbp.fb_conv_gemm_path(-1)
    dx, _, st = fbp.conv3x3_backward(to_bf16_tensor(x), to_bf16_tensor(wt), to_bf16_tensor(dz), 2,
                                     weight_grad=False)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and fbp.fb_conv_gemm_path(-1) == n0
    dx_ref, _, _ = ref.conv3x3_backward(x, w, dz, 2)
    assert float(np.linalg.norm(dx.cpu().numpy() - dx_ref) / np.linalg.norm(dx_ref)) < 1e-5
