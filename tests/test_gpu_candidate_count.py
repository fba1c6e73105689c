"""The number of candidates the NNF kernels consider equals its closed form (debug
build libfb_debug.so, which counts them on the device)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUNNER = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import synth
import paper_2311_09265_b300 as fbp
from paper_2311_09265_b300 import _build
fbp.LIB_PATH = _build.build_debug()
ctx = fbp.Context(0)
out = {}
for name, (H, W, k, iters, levels, r0) in json.loads(sys.argv[2]).items():
    g = synth.noise_pair(H, W, seed=3)
    fbp.fb_debug_candidates_considered(reset=True)
    p = fbp.Params.make(k, iters, levels, r0, 9, 0)
    fbp.fb_nnf(ctx, torch.tensor(g[0], device="cuda"), torch.tensor(g[1], device="cuda"), p)
    torch.cuda.synchronize()
    out[name] = fbp.fb_debug_candidates_considered()
w = synth.WORKLOADS["blend_tiny"]
gg, ss = synth.make_clip("blend_tiny")
fbp.fb_debug_candidates_considered(reset=True)
fbp.fb_blend_window(ctx, torch.tensor(gg, device="cuda"), torch.tensor(ss, device="cuda"), w.window,
                    fbp.Params.make(w.patch, w.iters, 1, 0, w.seed))
torch.cuda.synchronize()
out["blend_tiny"] = fbp.fb_debug_candidates_considered()
print(json.dumps(out))
"""

CASES = {"square": (64, 64, 5, 3, 1, 0), "ragged": (37, 53, 7, 2, 1, 0), "r0": (40, 44, 5, 3, 1, 4),
         "pyramid": (61, 77, 5, 2, 3, 0)}


def per_pair(H, W, iters, levels, r0):
    """Alg. 1: at each level one initial candidate per pixel, then per iteration one per
    propagation neighbour inside the image and one per radius r0 >> t >= 1."""
    total, h, w = 0, H, W
    sizes = []
    for _ in range(levels):
        sizes.append((h, w))
        h, w = (h + 1) // 2, (w + 1) // 2
    for h, w in sizes:
        r = r0 if r0 > 0 else max(h, w)
        radii = r.bit_length()
        neighbours = 4 * h * w - 2 * h - 2 * w
        total += h * w + iters * (neighbours + h * w * radii)
    return total


def test_candidates_considered_equal_the_closed_form():
    res = subprocess.run([sys.executable, "-c", RUNNER, ROOT, json.dumps(CASES)], cwd=ROOT,
                         capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    got = json.loads(res.stdout.strip().splitlines()[-1])
    for name, (H, W, k, iters, levels, r0) in CASES.items():
        assert got[name] == per_pair(H, W, iters, levels, r0), (name, got[name])
    import synth
    w = synth.WORKLOADS["blend_tiny"]
    assert got["blend_tiny"] == w.pairs() * per_pair(w.H, w.W, w.iters, 1, 0)


def test_product_library_does_not_count():
    import paper_2311_09265_b300 as fbp
    with pytest.raises(fbp.FastBlendError) as ei:
        fbp.fb_debug_candidates_considered()
    assert ei.value.status == fbp.FB_ERR_UNSUPPORTED
