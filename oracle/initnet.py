"""CPU oracle for the learned NNF initialiser -- TEST INFRASTRUCTURE ONLY.

Plain numpy in float64.  Tensors are NHWC; conv weights are [Cout][3][3][Cin]; every
convolution is 3x3 with zero padding 1 and stride 1 or 2, written tap by tap from the
definition y[p] = b + sum_tap W[tap] . x[p*s + tap - 1].  Values are rounded to bf16 at
the points where the device stores bf16 (input, weights, layer outputs, the gradient at
each pre-activation), so the comparison isolates accumulation order.
Pins (tests/test_initnet_oracle.py): central finite differences of the conv gradients
and of the whole network's loss, the identity-kernel closed form, stride-2 sizes.
This network is not part of the paper's method (Sec. 3.1: model-free); it is trained on
NNFs that the method computes.
"""
from __future__ import annotations

import numpy as np

# (Cin, Cout, stride, relu) of e0a e0b e1a e1b e2a e2b e3a e3b d2 d1 d0 head
LAYERS = [(8, 32, 1, 1), (32, 32, 1, 1), (32, 64, 2, 1), (64, 64, 1, 1), (64, 96, 2, 1),
          (96, 96, 1, 1), (96, 128, 2, 1), (128, 128, 1, 1), (224, 96, 1, 1), (160, 64, 1, 1),
          (96, 32, 1, 1), (32, 8, 1, 0)]
OFFSET_SCALE = 16.0


def bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_bits(a) -> np.ndarray:
    """bfloat16 bit patterns (uint16) of the rounded values."""
    f = bf16(a).astype(np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def out_size(n: int, stride: int) -> int:
    return (n + stride - 1) // stride


def _taps(xpad, Ho, Wo, stride, ty, tx):
    return xpad[:, ty:ty + stride * (Ho - 1) + 1:stride, tx:tx + stride * (Wo - 1) + 1:stride, :]


def conv3x3(x, w, b, stride):
    """y = b + sum over the 9 taps of w[:, ty, tx, :] applied to the shifted input."""
    n, H, W, Cin = x.shape
    Cout = w.shape[0]
    Ho, Wo = out_size(H, stride), out_size(W, stride)
    xpad = np.zeros((n, H + 2, W + 2, Cin))
    xpad[:, 1:H + 1, 1:W + 1] = x
    y = np.zeros((n, Ho, Wo, Cout)) + b
    for ty in range(3):
        for tx in range(3):
            y += np.einsum("nhwc,oc->nhwo", _taps(xpad, Ho, Wo, stride, ty, tx), w[:, ty, tx, :])
    return y


def conv3x3_backward(x, w, dz, stride):
    """(dx, dw, db) of conv3x3 given the gradient dz at its output."""
    n, H, W, Cin = x.shape
    Ho, Wo = dz.shape[1], dz.shape[2]
    xpad = np.zeros((n, H + 2, W + 2, Cin))
    xpad[:, 1:H + 1, 1:W + 1] = x
    dxpad = np.zeros_like(xpad)
    dw = np.zeros_like(w)
    for ty in range(3):
        for tx in range(3):
            dw[:, ty, tx, :] = np.einsum("nhwo,nhwc->oc", dz, _taps(xpad, Ho, Wo, stride, ty, tx))
            dxpad[:, ty:ty + stride * (Ho - 1) + 1:stride, tx:tx + stride * (Wo - 1) + 1:stride, :] += \
                np.einsum("nhwo,oc->nhwc", dz, w[:, ty, tx, :])
    return dxpad[:, 1:H + 1, 1:W + 1], dw, dz.sum(axis=(0, 1, 2))


def split_params(flat):
    """Per layer (w [Cout,3,3,Cin], b [Cout]) views of the flat parameter vector."""
    out, off = [], 0
    for cin, cout, _, _ in LAYERS:
        nw = cout * 9 * cin
        out.append((flat[off:off + nw].reshape(cout, 3, 3, cin), flat[off + nw:off + nw + cout]))
        off += nw + cout
    return out


def n_params() -> int:
    return sum(cout * 9 * cin + cout for cin, cout, _, _ in LAYERS)


def net_input(src, tgt, ds=4):
    """ds x ds box means of both guide stacks, /255 - 0.5, 8 channels (last two zero)."""
    n, H, W, _ = src.shape
    def q(a):
        return a.astype(np.float64).reshape(n, H // ds, ds, W // ds, ds, 3).mean(axis=(2, 4))
    x = np.zeros((n, H // ds, W // ds, 8))
    x[..., 0:3] = q(src) / 255.0 - 0.5
    x[..., 3:6] = q(tgt) / 255.0 - 0.5
    return bf16(x)


def _up(a):
    return np.repeat(np.repeat(a, 2, axis=1), 2, axis=2)


def forward(params, src, tgt, ds=4):
    """Returns (head [n, H/ds, W/ds, 8] float64, cache for backward)."""
    P = [(bf16(w), b) for w, b in split_params(params)]
    acts = {"in": net_input(src, tgt, ds)}
    order = ["e0a", "e0b", "e1a", "e1b", "e2a", "e2b", "e3a", "e3b", "d2", "d1", "d0", "head"]
    inputs = {"e0a": "in", "e0b": "e0a", "e1a": "e0b", "e1b": "e1a", "e2a": "e1b", "e2b": "e2a",
              "e3a": "e2b", "e3b": "e3a", "d2": "cat2", "d1": "cat1", "d0": "cat0", "head": "d0"}
    cats = {"d2": ("e3b", "e2b"), "d1": ("d2", "e1b"), "d0": ("d1", "e0b")}
    for l, name in enumerate(order):
        if name in cats:
            lo, skip = cats[name]
            acts[inputs[name]] = np.concatenate([_up(acts[lo]), acts[skip]], axis=-1)
        cin, cout, stride, relu = LAYERS[l]
        z = conv3x3(acts[inputs[name]], P[l][0], P[l][1], stride)
        if name == "head":
            acts[name] = z                       # float32 on the device, not rounded
        else:
            acts[name] = bf16(np.maximum(z, 0.0) if relu else z)
    return acts["head"], (P, acts, order, inputs, cats)


def loss_and_grad_head(head, target, weight, weight_sum):
    """Smooth-L1 (delta 1 pixel) between 16 * head[..., :2] and target, weighted."""
    d = OFFSET_SCALE * head[..., :2] - target
    ad = np.abs(d)
    w = np.ones(head.shape[:-1]) if weight is None else weight
    per = np.where(ad < 1.0, 0.5 * d * d, ad - 0.5)
    loss = float((per * w[..., None]).sum() / weight_sum)
    g = np.where(ad < 1.0, d, np.sign(d)) * w[..., None] * OFFSET_SCALE / weight_sum
    dhead = np.zeros_like(head)
    dhead[..., :2] = g
    return loss, dhead


def backward(cache, dhead):
    """Flat gradient of the parameters given the gradient at the head output."""
    P, acts, order, inputs, cats = cache
    grads = [None] * len(order)
    dact = {k: np.zeros_like(v) for k, v in acts.items()}
    dact["head"] = dhead
    for l in range(len(order) - 1, -1, -1):
        name = order[l]
        cin, cout, stride, relu = LAYERS[l]
        dz = dact[name] * (acts[name] > 0) if relu else dact[name]
        dz = bf16(dz)
        dx, dw, db = conv3x3_backward(acts[inputs[name]], P[l][0], dz, stride)
        grads[l] = (dw, db)
        if l > 0:
            dact[inputs[name]] += dx
        if name in cats:
            lo, skip = cats[name]
            c1 = acts[lo].shape[-1]
            dcat = dact[inputs[name]]
            n, H2, W2, _ = dcat.shape
            dact[lo] += dcat[..., :c1].reshape(n, H2 // 2, 2, W2 // 2, 2, c1).sum(axis=(2, 4))
            dact[skip] += dcat[..., c1:]
    return np.concatenate([np.concatenate([dw.ravel(), db]) for dw, db in grads])


def init_params(seed: int) -> np.ndarray:
    """He-normal weights, zero biases, head weights scaled by 0.1."""
    rng = np.random.default_rng(seed)
    out = []
    for l, (cin, cout, _, _) in enumerate(LAYERS):
        std = np.sqrt(2.0 / (9 * cin)) * (0.1 if l == len(LAYERS) - 1 else 1.0)
        w = rng.normal(0.0, std, size=(cout, 3, 3, cin))
        if l == len(LAYERS) - 1:
            w[2:] = 0.0                        # only channels 0, 1 of the head are used
        out.append(np.concatenate([w.ravel(), np.zeros(cout)]))
    return np.concatenate(out)
