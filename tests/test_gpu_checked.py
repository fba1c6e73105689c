"""The checked build (libfb_checked.so, FB_CHECKED): device-side invariant checks that
record failures in a status word instead of faulting.

Every case of checked_cases.py runs through the checked library in a child process: no
check may fail, the checks must have visited the pixels (exactly the closed-form count
where there is one), and the outputs must be bit-identical to the product library's and,
for the plain NNF, blend and interpolation, to the CPU oracle's.  Then fb_nnf_step plants
an inconsistent snapshot -- errors that are not the loss of their matches, a state a race
in the Jacobi ping-pong would leave behind -- and the energy check must report exactly
the planted pixels, with no access outside any buffer (the step reads only in-image
matches).
"""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import checked_cases
import oracle
import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.dirname(os.path.abspath(__file__))

RUNNER = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[2])
import synth, checked_cases
import paper_2311_09265_b300 as fbp
from paper_2311_09265_b300 import _build
fbp.LIB_PATH = _build.build_checked()
out_dir = sys.argv[3]
ctx = fbp.Context(0)
fbp.fb_check_status(reset=True)
status = {}
for name in checked_cases.CASES:
    arrays = checked_cases.run(fbp, ctx, name)
    torch.cuda.synchronize()
    status[name] = fbp.fb_check_status(reset=True)
    np.savez(f"{out_dir}/{name}.npz", *arrays)

# Jacobi step from a consistent snapshot, then from one with planted errors.
H, W, k = 45, 62, 5
g, _ = synth.small_clip(2, H, W, seed=99, motion="affine")
src, tgt = torch.from_numpy(g[1]).cuda(), torch.from_numpy(g[0]).cuda()
p = fbp.Params.make(k, 1, 1, 0, 5, 3)
F, E = fbp.fb_nnf(ctx, src, tgt, p)
torch.cuda.synchronize()
fbp.fb_check_status(reset=True)  # count the step's visits only
F1, E1 = fbp.fb_nnf_step(ctx, src, tgt, p, 1, F, E)
torch.cuda.synchronize()
status["step_clean"] = fbp.fb_check_status(reset=True)
np.savez(f"{out_dir}/step_clean.npz", F1.cpu().numpy(), E1.cpu().numpy())
planted = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (7, 31), (22, 40), (31, 5)]
E_bad = E.clone()
for r, c in planted:
    E_bad[r, c] += 1 + r
fbp.fb_nnf_step(ctx, src, tgt, p, 1, F, E_bad)
torch.cuda.synchronize()
status["step_planted"] = fbp.fb_check_status(reset=True)
E_host = E.cpu().numpy().view(np.uint32)
status["planted_words"] = [[3, int(E_host[r, c]) + 1 + r, int(E_host[r, c])] for r, c in planted]
ctx.close()
print("CHECKED_STATUS " + json.dumps(status))
"""


@pytest.fixture(scope="module")
def checked_run():
    with tempfile.TemporaryDirectory() as d:
        res = subprocess.run([sys.executable, "-c", RUNNER, ROOT, TESTS, d], capture_output=True,
                             text=True, timeout=900)
        assert res.returncode == 0, res.stderr[-4000:]
        line = [ln for ln in res.stdout.splitlines() if ln.startswith("CHECKED_STATUS ")][-1]
        status = json.loads(line[len("CHECKED_STATUS "):])
        outs = {}
        for f in os.listdir(d):
            with np.load(os.path.join(d, f)) as z:
                outs[f[:-4]] = [z[f"arr_{i}"] for i in range(len(z.files))]
        yield status, outs


@pytest.fixture(scope="module")
def product():
    import torch
    import paper_2311_09265_b300 as fbp
    fbp.build()
    ctx = fbp.Context(0)
    yield fbp, ctx
    torch.cuda.synchronize()
    ctx.close()


def decode(word: int):
    return word >> 56, (word >> 28) & 0xFFFFFFF, word & 0xFFFFFFF


def test_product_library_has_no_checks(product):
    fbp, _ = product
    with pytest.raises(fbp.FastBlendError):
        fbp.fb_check_status()


@pytest.mark.parametrize("name", sorted(checked_cases.CASES))
def test_case_passes_every_check_and_matches_the_product_library(checked_run, product, name):
    status, outs = checked_run
    first, failed, visits = status[name]
    assert failed == 0 and first == 0, (name, decode(first), failed)
    want_visits = checked_cases.expected_visits(name)
    if want_visits is not None:
        assert visits == want_visits
    else:
        assert visits > 0
    fbp, ctx = product
    ref = checked_cases.run(fbp, ctx, name)
    assert len(ref) == len(outs[name])
    for got, want in zip(outs[name], ref):
        assert got.shape == want.shape and (got == want).all(), name


@pytest.mark.parametrize("name", ["nnf_k3", "nnf_k5_pyramid", "nnf_k7", "nnf_k9_r0"])
def test_checked_nnf_matches_the_oracle(checked_run, name):
    _, outs = checked_run
    H, W, k, iters, levels, r0 = checked_cases.CASES[name][1]
    g, _ = synth.small_clip(2, H, W, seed=H * 1000 + W + k, motion="affine")
    Fo, Eo = oracle.nnf(g[1], g[0], k, iters, levels=levels, r0=r0, seed=checked_cases.SEED,
                        pair_tag=oracle.pair_tag(1, 0))
    F, E = outs[name]
    assert (F == Fo).all() and (E.view(np.uint32) == Eo).all()


def test_checked_blend_and_interpolation_match_the_oracle(checked_run):
    _, outs = checked_run
    N, H, W, k, window, iters, levels, _ = checked_cases.CASES["blend_plain"][1]
    g, s = synth.small_clip(N, H, W, seed=N * 100 + H + W, motion="affine")
    ref = oracle.blend_window(g, s, window, k, iters, levels=levels, seed=checked_cases.SEED)
    assert (outs["blend_plain"][0] == ref).all()
    N, H, W, k, iters, keys, _ = checked_cases.CASES["interp_plain"][1]
    g, s = synth.small_clip(N, H, W, seed=N * 10 + H + W, motion="affine")
    ref = oracle.interpolate(g, list(keys), s[list(keys)], k, iters, seed=checked_cases.SEED)
    assert (outs["interp_plain"][0] == ref).all()


def test_step_from_a_consistent_snapshot_passes_and_equals_the_oracle(checked_run):
    status, outs = checked_run
    first, failed, visits = status["step_clean"]
    assert failed == 0 and first == 0 and visits == 45 * 62
    g, _ = synth.small_clip(2, 45, 62, seed=99, motion="affine")
    Fo, Eo = oracle.nnf(g[1], g[0], 5, 2, seed=5, pair_tag=3)
    F, E = outs["step_clean"]
    assert (F == Fo).all() and (E.view(np.uint32) == Eo).all()


def test_planted_snapshot_errors_are_reported_exactly(checked_run):
    status, _ = checked_run
    first, failed, visits = status["step_planted"]
    planted = [tuple(w) for w in status["planted_words"]]
    assert failed == len(planted)
    assert visits == 45 * 62
    assert decode(first) in planted
