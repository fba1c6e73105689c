"""Seeded synthetic clips shaped like the workloads of FastBlend (arXiv 2311.09265).

The paper measures on real videos whose style frames come from a diffusion model
(Sec. 4.1, Sec. 4.5); neither is available, so these generators stand in for them.
This module holds none of the method's arithmetic (no patch distance, no NNF, no
remap, no blend): it only draws guide and style frames, and the ground-truth motion
that produced them.  Both the CUDA path and the CPU oracle consume its output as
plain data.

Recipes
  shift clip    gradient-noise texture (Perlin's lattice-gradient construction with
                quintic fade, gradients drawn from a seeded generator; a few octaves)
                plus i.i.d. integer jitter baked into the texture so every patch is
                unique; frame t is the texture cropped at an integer offset s_t that
                follows a random walk with steps in [-3, 3]^2.  The true match of
                target pixel x of frame i in frame j is x + s_i - s_j.
  colour-matrix style  a fixed 3x3 colour matrix applied to the guide plus per-frame
                uniform integer noise in [-8, 8] (flicker), clamped to [0, 255].
  affine clip   multi-octave gradient noise sampled bilinearly at coordinates moved
                by a smooth random affine motion: rotation steps of at most 2 degrees
                and translation steps of at most 6 px per frame (a smoothed random
                walk, kept within a bounded excursion), then rounded to uint8.
  LUT style     a random monotone tone curve per channel and frame plus Gaussian
                noise of sigma 6, rounded and clamped.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 0x2311_0926_0000


def clip_seed(cfg: int, clip: int = 0) -> int:
    return SEED_BASE + cfg * 1000 + clip


# ----------------------------------------------------------------------------------
# Gradient noise
# ----------------------------------------------------------------------------------
def _fade(t: np.ndarray) -> np.ndarray:
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def gradient_noise(H: int, W: int, period: float, rng: np.random.Generator) -> np.ndarray:
    """One octave of 2-D lattice gradient noise on an H x W grid, values ~[-1, 1]."""
    gh = int(math.ceil(H / period)) + 2
    gw = int(math.ceil(W / period)) + 2
    ang = rng.uniform(0.0, 2.0 * math.pi, size=(gh, gw)).astype(np.float32)
    gy, gx = np.sin(ang), np.cos(ang)
    y = (np.arange(H, dtype=np.float32) + 0.5) / np.float32(period)
    x = (np.arange(W, dtype=np.float32) + 0.5) / np.float32(period)
    y0 = np.floor(y).astype(np.int64)
    x0 = np.floor(x).astype(np.int64)
    fy = (y - y0)[:, None]
    fx = (x - x0)[None, :]
    Y0, X0 = y0[:, None], x0[None, :]

    def corner(dy: int, dx: int) -> np.ndarray:
        return gy[Y0 + dy, X0 + dx] * (fy - dy) + gx[Y0 + dy, X0 + dx] * (fx - dx)

    uy, ux = _fade(fy), _fade(fx)
    top = corner(0, 0) * (1 - ux) + corner(0, 1) * ux
    bot = corner(1, 0) * (1 - ux) + corner(1, 1) * ux
    return (top * (1 - uy) + bot * uy).astype(np.float32) * np.float32(1.4142)


def noise_texture(H: int, W: int, rng: np.random.Generator, periods=(32.0, 12.0),
                  jitter: int = 6) -> np.ndarray:
    """H x W x 3 float texture in [0, 255] (not yet rounded), per-channel octaves."""
    out = np.empty((H, W, 3), np.float32)
    for ch in range(3):
        acc = np.zeros((H, W), np.float32)
        amp, norm = 1.0, 0.0
        for per in periods:
            acc += np.float32(amp) * gradient_noise(H, W, per, rng)
            norm += amp
            amp *= 0.6
        out[..., ch] = 127.5 + 110.0 * np.clip(acc / np.float32(norm), -1.0, 1.0)
    if jitter:
        out += rng.integers(-jitter, jitter + 1, size=out.shape).astype(np.float32)
    return np.clip(out, 0.0, 255.0)


# ----------------------------------------------------------------------------------
# Guide clips
# ----------------------------------------------------------------------------------
def shift_clip(N: int, H: int, W: int, seed: int, max_step: int = 3):
    """Guides (N,H,W,3) uint8 and integer shifts (N,2) int64 with s_0 = (0, 0)."""
    rng = np.random.default_rng(seed)
    steps = rng.integers(-max_step, max_step + 1, size=(N, 2))
    steps[0] = 0
    shifts = np.cumsum(steps, axis=0)
    m = max_step * max(N, 1)
    tex = np.rint(noise_texture(H + 2 * m, W + 2 * m, rng)).astype(np.uint8)
    g = np.empty((N, H, W, 3), np.uint8)
    for t in range(N):
        r0, c0 = m + shifts[t, 0], m + shifts[t, 1]
        g[t] = tex[r0:r0 + H, c0:c0 + W]
    return g, shifts


@dataclass
class AffineMotion:
    theta_deg: np.ndarray          # (N,) rotation of frame t
    shift: np.ndarray              # (N, 2) translation (rows, cols) of frame t
    margin: int = 0


def affine_motion(N: int, rng: np.random.Generator, max_rot_step: float = 2.0,
                  max_shift_step: float = 6.0, max_rot: float = 12.0,
                  max_shift: float = 48.0) -> AffineMotion:
    """Smoothed random walk: velocity = 0.8 velocity + 0.2 noise, clipped per frame."""
    th = np.zeros(N)
    sh = np.zeros((N, 2))
    vth, vsh = 0.0, np.zeros(2)
    for t in range(1, N):
        vth = float(np.clip(0.8 * vth + 0.2 * rng.normal(0.0, 2.5), -max_rot_step, max_rot_step))
        vsh = np.clip(0.8 * vsh + 0.2 * rng.normal(0.0, 8.0, size=2), -max_shift_step, max_shift_step)
        th[t] = np.clip(th[t - 1] + vth, -max_rot, max_rot)
        sh[t] = np.clip(sh[t - 1] + vsh, -max_shift, max_shift)
    return AffineMotion(th, sh)


def affine_clip(N: int, H: int, W: int, seed: int, frames=None):
    """Guides (N,H,W,3) uint8 under smooth random affine motion, and the motion.
    frames=(a, b): only clip frames [a, b) of the same N-frame clip, bit-identical to
    those frames of the whole clip (the motion and texture are drawn for the whole clip
    first), returned as (b - a,H,W,3)."""
    a, b = (0, N) if frames is None else frames
    if not 0 <= a < b <= N:
        raise ValueError(f"frames {frames} outside [0, {N})")
    rng = np.random.default_rng(seed)
    mot = affine_motion(N, rng)
    half_diag = 0.5 * math.hypot(H, W)
    m = int(math.ceil(half_diag * math.sin(math.radians(12.0)) + 48 + 8))
    TH, TW = H + 2 * m, W + 2 * m
    tex = noise_texture(TH, TW, rng, periods=(48.0, 20.0, 9.0, 4.0), jitter=5)
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64) - (H - 1) / 2.0,
                         np.arange(W, dtype=np.float64) - (W - 1) / 2.0, indexing="ij")
    g = np.empty((b - a, H, W, 3), np.uint8)
    for t in range(a, b):
        ang = math.radians(mot.theta_deg[t])
        ca, sa = math.cos(ang), math.sin(ang)
        sy = ca * yy - sa * xx + mot.shift[t, 0] + (TH - 1) / 2.0
        sx = sa * yy + ca * xx + mot.shift[t, 1] + (TW - 1) / 2.0
        y0 = np.clip(np.floor(sy).astype(np.int64), 0, TH - 2)
        x0 = np.clip(np.floor(sx).astype(np.int64), 0, TW - 2)
        fy = np.clip(sy - y0, 0.0, 1.0)[..., None].astype(np.float32)
        fx = np.clip(sx - x0, 0.0, 1.0)[..., None].astype(np.float32)
        v = (tex[y0, x0] * (1 - fy) * (1 - fx) + tex[y0, x0 + 1] * (1 - fy) * fx
             + tex[y0 + 1, x0] * fy * (1 - fx) + tex[y0 + 1, x0 + 1] * fy * fx)
        g[t - a] = np.clip(np.rint(v), 0, 255).astype(np.uint8)
    mot.margin = m
    return g, mot


# ----------------------------------------------------------------------------------
# Style frames
# ----------------------------------------------------------------------------------
def colour_matrix_styles(guides: np.ndarray, seed: int, noise: int = 8) -> np.ndarray:
    """Fixed 3x3 colour matrix of the guide plus per-frame uniform flicker noise."""
    rng = np.random.default_rng(seed ^ 0x5717E)
    Mx = rng.uniform(0.0, 1.0, size=(3, 3))
    Mx /= Mx.sum(axis=1, keepdims=True)
    out = np.empty_like(guides)
    for t in range(guides.shape[0]):
        v = guides[t].astype(np.float32) @ Mx.T.astype(np.float32)
        v += rng.integers(-noise, noise + 1, size=v.shape).astype(np.float32)
        out[t] = np.clip(np.rint(v), 0, 255).astype(np.uint8)
    return out


def random_lut(rng: np.random.Generator) -> np.ndarray:
    inc = rng.gamma(2.0, 1.0, size=256)
    curve = np.cumsum(inc)
    curve = (curve - curve[0]) / (curve[-1] - curve[0])
    lo, hi = rng.uniform(0, 40), rng.uniform(215, 255)
    return lo + (hi - lo) * curve


def lut_styles(guides: np.ndarray, seed: int, sigma: float = 6.0) -> np.ndarray:
    """Per-frame random monotone tone curve per channel plus Gaussian noise."""
    rng = np.random.default_rng(seed ^ 0x1C7)
    out = np.empty_like(guides)
    for t in range(guides.shape[0]):
        v = np.empty(guides.shape[1:], np.float32)
        for ch in range(3):
            v[..., ch] = random_lut(rng)[guides[t, ..., ch]]
        v += rng.normal(0.0, sigma, size=v.shape).astype(np.float32)
        out[t] = np.clip(np.rint(v), 0, 255).astype(np.uint8)
    return out


def lut_styles_indexed(guides: np.ndarray, seed: int, first: int = 0, sigma: float = 6.0) -> np.ndarray:
    """The LUT style recipe with one generator per clip frame index (first + t): any range
    of frames of a long clip is styled on its own, identically wherever it is cut (a clip
    split over several processes)."""
    out = np.empty_like(guides)
    for t in range(guides.shape[0]):
        rng = np.random.default_rng([seed ^ 0x1C7, first + t])
        v = np.empty(guides.shape[1:], np.float32)
        for ch in range(3):
            v[..., ch] = random_lut(rng)[guides[t, ..., ch]]
        v += rng.normal(0.0, sigma, size=v.shape).astype(np.float32)
        out[t] = np.clip(np.rint(v), 0, 255).astype(np.uint8)
    return out


# ----------------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    mode: str                      # "blend" or "interpolate"
    N: int
    H: int
    W: int
    patch: int
    iters: int
    window: int = 1
    keys: tuple = ()
    levels: int = 1
    seed: int = 0
    motion: str = "affine"
    extra: dict = field(default_factory=dict)

    def pairs(self) -> int:
        if self.mode == "blend":
            M = (self.window - 1) // 2
            return sum(min(self.N - 1, i + M) - max(0, i - M) for i in range(self.N))
        keys = list(self.keys)
        n = 0
        for i in range(self.N):
            if i in keys:
                continue
            left = any(k < i for k in keys)
            right = any(k > i for k in keys)
            n += int(left) + int(right)
        return n

    def random_search_radii(self) -> int:
        r0 = max(self.H, self.W)
        return int(math.floor(math.log2(r0))) + 1

    def candidate_evals(self) -> int:
        """Analytic count per call: one init evaluation plus, per iteration, four
        propagation and R random-search candidates per pixel (levels = 1)."""
        return self.pairs() * self.H * self.W * (1 + self.iters * (4 + self.random_search_radii()))


WORKLOADS = {
    "blend_tiny": Workload("plain blend 8x96x96 k5 w3 n4 (shift motion)", "blend", 8, 96, 96,
                           patch=5, iters=4, window=3, seed=clip_seed(0), motion="shift"),
    "blend_512": Workload("plain blend all-pairs 60x512x512 k5 w15 n6 (affine motion)", "blend",
                          60, 512, 512, patch=5, iters=6, window=15, seed=clip_seed(1)),
    "blend_512_16f": Workload("plain blend all-pairs 16x512x512 k5 w15 n6 (affine motion)", "blend",
                              16, 512, 512, patch=5, iters=6, window=15, seed=clip_seed(1, 16)),
    "interp_1024x576": Workload("plain interpolation 48x576x1024 k7 n8 keys 0,47 (affine motion)",
                                "interpolate", 48, 576, 1024, patch=7, iters=8, keys=(0, 47),
                                seed=clip_seed(2)),
}


@functools.lru_cache(maxsize=4)
def make_clip(key: str):
    """(guides, styles) for a named workload.  For interpolation `styles` holds the
    stylised keyframes only (len(keys) frames)."""
    w = WORKLOADS[key]
    if w.motion == "shift":
        g, _ = shift_clip(w.N, w.H, w.W, w.seed)
        s = colour_matrix_styles(g, w.seed)
    else:
        g, _ = affine_clip(w.N, w.H, w.W, w.seed)
        s = lut_styles(g, w.seed)
    if w.mode == "interpolate":
        s = np.ascontiguousarray(s[list(w.keys)])
    g.setflags(write=False)
    s.setflags(write=False)
    return g, s


def noise_pair(H: int, W: int, seed: int, shift=(1, 3)):
    """Two (H, W, 3) uint8 frames for edge-case shapes (e.g. one side at the largest
    supported size) where the smooth textures above are slow to synthesise: i.i.d.
    uniform bytes, and the same texture translated by `shift` (row, col) with
    edge-replicated borders."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    dr, dc = shift
    rows = np.clip(np.arange(H) - dr, 0, H - 1)
    cols = np.clip(np.arange(W) - dc, 0, W - 1)
    b = a[rows][:, cols]
    return np.stack([a, b])


def small_clip(N: int, H: int, W: int, seed: int, motion: str = "shift"):
    """A small clip for parity tests: guides and styles (N,H,W,3) uint8."""
    if motion == "shift":
        g, _ = shift_clip(N, H, W, seed)
        return g, colour_matrix_styles(g, seed)
    g, _ = affine_clip(N, H, W, seed)
    return g, lut_styles(g, seed)


# ----------------------------------------------------------------------------------
# Batched submission manifest: clips of uneven size, length, window and patch
# ----------------------------------------------------------------------------------
def batch_manifest(n_clips: int = 32, seed: int = clip_seed(3), sizes=(256, 1024),
                   frames=(16, 120), windows=(5, 31), patches=(5, 7)):
    """Seeded list of (N, H, W, window, patch): H, W multiples of 64 in [sizes],
    N uniform in [frames], odd windows uniform in [windows], patch from `patches`."""
    rng = np.random.default_rng(seed)
    out = []
    lo, hi = sizes[0] // 64, sizes[1] // 64
    for _ in range(n_clips):
        H = int(rng.integers(lo, hi + 1)) * 64
        W = int(rng.integers(lo, hi + 1)) * 64
        N = int(rng.integers(frames[0], frames[1] + 1))
        window = int(rng.integers(windows[0] // 2, windows[1] // 2 + 1)) * 2 + 1
        patch = int(rng.choice(patches))
        out.append((N, H, W, window, patch))
    return out


def batch_clip(N: int, H: int, W: int, seed: int):
    """Guides and styles of one manifest clip: the shift-clip recipe (cheap to draw at
    any size) with the colour-matrix flicker style."""
    g, _ = shift_clip(N, H, W, seed, max_step=2)
    return g, colour_matrix_styles(g, seed)
