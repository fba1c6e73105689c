"""Training of the learned NNF initialiser on fields computed by Alg. 1.

Every compute step runs in libfb.so: the targets come from fb_nnf (Alg. 1 with more
iterations than the blend uses) and fb_initnet_targets, the loss, backward pass and
Adam update from fb_initnet_train_step.  PyTorch only holds device memory and gathers
the pair stacks of a batch.  The guide clips are the seeded synthetic clips of the
`synth` module (smooth random affine motion), drawn with seeds other than the ones the
benchmarks evaluate on.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np
import torch

import synth

from . import (FB_FLAG_LEARNED_INIT, Context, InitNet, Params, fb_initnet_targets, fb_nnf)


@dataclass
class TrainingSet:
    frames: list          # per clip: (N, H, W, 3) uint8 CUDA tensor
    pairs: np.ndarray     # (P, 3): clip, source frame, target frame
    target: torch.Tensor  # (P, H/D, W/D, 2) float32
    weight: torch.Tensor  # (P, H/D, W/D) float32


def make_training_set(ctx: Context, n_clips: int = 6, frames: int = 24, H: int = 512, W: int = 512,
                      max_gap: int = 7, pairs_per_clip: int = 160, target_iters: int = 12,
                      downscale: int = 8, seed: int = synth.clip_seed(4)) -> TrainingSet:
    """Seeded clips, random ordered pairs with 1 <= |i - j| <= max_gap, and the method's
    own NNFs (target_iters iterations of Alg. 1) turned into block-mean targets."""
    rng = np.random.default_rng(seed)
    clips, pairs, targets, weights = [], [], [], []
    for c in range(n_clips):
        g, _ = synth.affine_clip(frames, H, W, seed + 101 * c)
        gd = torch.tensor(g, device="cuda")
        clips.append(gd)
        for _ in range(pairs_per_clip):
            i = int(rng.integers(0, frames))
            d = int(rng.integers(1, max_gap + 1)) * (1 if rng.random() < 0.5 else -1)
            j = min(max(i + d, 0), frames - 1)
            if j == i:
                j = i + 1 if i + 1 < frames else i - 1
            p = Params.make(5, target_iters, 1, 0, seed + 7 * len(pairs), 0)
            F, _ = fb_nnf(ctx, gd[j], gd[i], p)
            t, w = fb_initnet_targets(F.unsqueeze(0), downscale)
            pairs.append((c, j, i))
            targets.append(t[0])
            weights.append(w[0])
    return TrainingSet(clips, np.array(pairs, np.int64), torch.stack(targets), torch.stack(weights))


def batch(ts: TrainingSet, idx):
    src = torch.stack([ts.frames[c][j] for c, j, _ in ts.pairs[idx]])
    tgt = torch.stack([ts.frames[c][i] for c, _, i in ts.pairs[idx]])
    return src, tgt, ts.target[idx].contiguous(), ts.weight[idx].contiguous()


def initial_params(n_params: int, seed: int) -> np.ndarray:
    """He-normal weights, zero biases; the head starts small and uses channels 0, 1."""
    from .initnet_layout import LAYERS
    rng = np.random.default_rng(seed)
    out = []
    for l, (cin, cout) in enumerate(LAYERS):
        std = math.sqrt(2.0 / (9 * cin)) * (0.1 if l == len(LAYERS) - 1 else 1.0)
        w = rng.normal(0.0, std, size=(cout, 3, 3, cin)).astype(np.float32)
        if l == len(LAYERS) - 1:
            w[2:] = 0.0
        out.append(np.concatenate([w.ravel(), np.zeros(cout, np.float32)]))
    p = np.concatenate(out)
    assert p.size == n_params
    return p


def train(net: InitNet, ts: TrainingSet, steps: int = 1500, batch_size: int = 8, lr: float = 1e-3,
          warmup: int = 200, seed: int = 0, log_every: int = 100, start: int = 0, stop: int = None,
          rng: np.random.Generator = None):
    """Adam with a linear warm-up over `warmup` steps, then a cosine-decayed step size;
    returns the loss history (every log_every).  Without the warm-up the first few
    hundred steps swing widely and a run can stall on a plateau.  Steps [start, stop) of
    the `steps`-step schedule run (a resumed run passes the checkpoint's step and batch
    sampler `rng`)."""
    rng = np.random.default_rng(seed) if rng is None else rng
    hist = []
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    for s in range(start, steps if stop is None else stop):
        idx = rng.choice(len(ts.pairs), size=batch_size, replace=False)
        src, tgt, target, weight = batch(ts, idx)
        wsum = max(float(weight.sum()), 1.0)
        cur = lr * (0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * s / steps)))
        if warmup > 0:
            cur *= min(1.0, (s + 1) / warmup)
        net.train_step(src, tgt, target, weight, wsum, cur, loss_out=loss)
        if s % log_every == 0 or s == steps - 1:
            hist.append((s, float(loss.item()), time.perf_counter() - t0))
    return hist


def save(net: InitNet, path: str) -> None:
    """The FP32 parameters only (what an evaluation needs)."""
    np.save(path, net.get_params())


def load(net: InitNet, path: str) -> None:
    net.set_params(np.load(path))


def save_checkpoint(net: InitNet, path: str, step: int, rng: np.random.Generator) -> None:
    """Everything a resumed run needs: parameters, Adam moments and update count, the
    schedule step and the batch sampler's state (a host .npz file)."""
    import json
    m, v, updates = net.get_optimizer()
    np.savez(path, params=net.get_params(), adam_m=m, adam_v=v, updates=np.uint64(updates),
             step=np.int64(step), rng=np.array(json.dumps(rng.bit_generator.state)))


def load_checkpoint(net: InitNet, path: str):
    """Restores a save_checkpoint file into `net`; returns (schedule step, batch sampler)."""
    import json
    z = np.load(path)
    net.set_params(z["params"])
    net.set_optimizer(z["adam_m"], z["adam_v"], int(z["updates"]))
    rng = np.random.default_rng()
    rng.bit_generator.state = json.loads(str(z["rng"]))
    return int(z["step"]), rng


def train_default(ctx: Context, H: int, W: int, max_pairs: int = 256, steps: int = 2500,
                  n_clips: int = 6, frames: int = 24, pairs_per_clip: int = 200,
                  downscale: int = 8, seed: int = synth.clip_seed(4)):
    """The recipe used for the benchmarks: a fresh net trained on the method's own NNFs
    of seeded clips (different seeds from the evaluation clips).  Returns
    (net, loss history, seconds for the training set, seconds for training)."""
    t0 = time.perf_counter()
    ts = make_training_set(ctx, n_clips=n_clips, frames=frames, H=H, W=W,
                           pairs_per_clip=pairs_per_clip, downscale=downscale, seed=seed)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = InitNet(ctx, max_pairs, H, W, downscale=downscale)
    net.set_params(initial_params(net.n_params, seed & 0xFFFF))
    t0 = time.perf_counter()
    hist = train(net, ts, steps=steps, batch_size=8, lr=1e-3, warmup=200, seed=seed & 0xFFFF,
                 log_every=max(steps // 10, 1))
    torch.cuda.synchronize()
    return net, hist, t_data, time.perf_counter() - t0
