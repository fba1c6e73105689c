"""The learned-initialiser oracle's pins catch plausible mistakes: each mutant is a
one-place edit of oracle/initnet.py, executed into the imported module in a subprocess,
and the pin suite tests/test_initnet_oracle.py must fail on it."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "initnet.py")

MUTANTS = {
    "conv_taps_transposed": ('w[:, ty, tx, :])\n    return y', 'w[:, tx, ty, :])\n    return y'),
    "conv_padding_offset": ("    xpad[:, 1:H + 1, 1:W + 1] = x\n    y = ", "    xpad[:, 0:H, 0:W] = x\n    y = "),
    "wgrad_taps_transposed": ("dw[:, ty, tx, :] = np.einsum", "dw[:, tx, ty, :] = np.einsum"),
    "bias_gradient_halved": ("dz.sum(axis=(0, 1, 2))", "0.5 * dz.sum(axis=(0, 1, 2))"),
    "loss_gradient_sign": ("g = np.where(ad < 1.0, d, np.sign(d))", "g = np.where(ad < 1.0, -d, np.sign(d))"),
    "loss_huber_threshold": ("per = np.where(ad < 1.0, 0.5 * d * d, ad - 0.5)", "per = np.where(ad < 2.0, 0.5 * d * d, ad - 0.5)"),
    "relu_mask_not_applied": ("dz = dact[name] * (acts[name] > 0) if relu else dact[name]",
                              "dz = dact[name] * (acts[name] >= 0) if relu else dact[name]"),
    "concat_gradient_swapped": ("dact[skip] += dcat[..., c1:]", "dact[skip] += dcat[..., :dact[skip].shape[-1]]"),
    "bf16_rounds_half_up": ("r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16", "r = ((u + 0x8000) >> 16) << 16"),
    "input_scale_256": ("x[..., 0:3] = q(src) / 255.0 - 0.5", "x[..., 0:3] = q(src) / 256.0 - 0.5"),
    "offset_scale_8": ("OFFSET_SCALE = 16.0", "OFFSET_SCALE = 8.0"),
    "skip_and_upsampled_swapped": ("np.concatenate([_up(acts[lo]), acts[skip]], axis=-1)",
                                   "np.concatenate([acts[skip], _up(acts[lo])], axis=-1)"),
}

RUNNER = """
import sys
import pytest
import oracle.initnet as m
exec(compile(open(sys.argv[1]).read(), "initnet_mutant", "exec"), m.__dict__)
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", sys.argv[2]]))
"""


def run_mutant(name: str, workdir: str):
    old, new = MUTANTS[name]
    with open(SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation site of {name} not unique: {old!r}"
    mutant = os.path.join(workdir, f"{name}.py")
    with open(mutant, "w") as f:
        f.write(src.replace(old, new))
    res = subprocess.run([sys.executable, "-c", RUNNER, mutant,
                          os.path.join(ROOT, "tests", "test_initnet_oracle.py")],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    return res.returncode, res.stdout[-1500:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """All mutants, tested concurrently (each in its own process)."""
    from concurrent.futures import ThreadPoolExecutor
    workdir = str(tmp_path_factory.mktemp("initnet_mutants"))
    with ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        futs = {name: ex.submit(run_mutant, name, workdir) for name in MUTANTS}
        return {name: f.result() for name, f in futs.items()}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, outcomes):
    code, out = outcomes[name]
    assert code == 1, f"no pin failed for mutant {name}:\n{out}"
