"""CPU oracle for the FastBlend hot path (arXiv 2311.09265) -- ctypes front end.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code with it; ``fbref.c`` restates the paper's
algorithms (Alg. 1, Eq. 1, Alg. 2, Eq. 2, Sec. 3.5.2) with plain loops.

All arrays are numpy: images ``(H, W, 3) uint8``, stacks ``(N, H, W, 3) uint8``,
NNFs ``(H, W, 2) int32`` holding (row, col), errors ``(H, W) uint32``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_DIR, "fbref.c")
_HDR = os.path.join(_DIR, "fbref.h")
LIB_PATH = os.path.join(_DIR, "libfbref.so")
# tests/test_oracle_mutants.py runs the pins against deliberately broken builds of
# fbref.c; this variable points the front end at such a build instead of LIB_PATH.
_LIB_OVERRIDE = os.environ.get("FBREF_TEST_LIBRARY")

_lib = None


def build(force: bool = False) -> str:
    """Compile fbref.c into libfbref.so (gcc, -O2, OpenMP, IEEE float: no fast-math)."""
    stale = (not os.path.exists(LIB_PATH)
             or os.path.getmtime(LIB_PATH) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                        "-fno-fast-math", "-o", tmp, _SRC], check=True)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("patch", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("r0", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_f32p = ctypes.POINTER(ctypes.c_float)
_P = ctypes.POINTER(Params)


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if _LIB_OVERRIDE:
            L = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            L = ctypes.CDLL(LIB_PATH)
        L.fbref_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.fbref_ssd.argtypes = [_u8p, _u8p] + [ctypes.c_int] * 7
        L.fbref_ssd.restype = ctypes.c_uint32
        L.fbref_downsample.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, _u8p]
        L.fbref_rs_offset.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      _i32p, _i32p]
        L.fbref_nnf.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int, _P, ctypes.c_uint32,
                                _i32p, _i32p, _u32p]
        L.fbref_nnf_trace.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int, _P,
                                      ctypes.c_uint32, _i32p, _i32p, _u32p]
        L.fbref_nnf_bruteforce.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           _i32p, _u32p]
        L.fbref_remap_sum.argtypes = [_u8p, _i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u32p]
        L.fbref_remap.argtypes = [_u8p, _i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _f32p]
        L.fbref_blend_window.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _P, _f32p]
        L.fbref_blend_frame.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, _P, ctypes.c_int, _f32p]
        L.fbref_interpolate.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p,
                                        _u8p, ctypes.c_int, _P, _f32p]
        L.fbref_interpolate_frame.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              _i32p, _u8p, ctypes.c_int, _P, ctypes.c_int, _f32p]
        L.fbref_shat.argtypes = [_u8p, _i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8p]
        L.fbref_nnf_balanced.argtypes = [_u8p, _u8p, _u8p, ctypes.c_int, ctypes.c_int, _P,
                                         ctypes.c_uint32, ctypes.c_uint32, _i32p, _i32p, _u32p, _u8p]
        L.fbref_nnf_balanced.restype = ctypes.c_int
        L.fbref_blend_frame_balanced.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, _P, ctypes.c_uint32,
                                                 ctypes.c_int, _f32p]
        L.fbref_blend_frame_balanced.restype = ctypes.c_int
        L.fbref_blend_window_balanced.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_int, _P, ctypes.c_uint32,
                                                  _f32p]
        L.fbref_blend_window_balanced.restype = ctypes.c_int
        L.fbref_nnf_chain.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P,
                                      _u32p, _i32p, _i32p, _u32p]
        L.fbref_nnf_chain.restype = ctypes.c_int
        L.fbref_interpolate_tracking.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 _i32p, _u8p, ctypes.c_int, _P, _f32p]
        L.fbref_interpolate_tracking.restype = ctypes.c_int
        L.fbref_blend_window_tracking.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_int, _P, _f32p]
        L.fbref_blend_window_tracking.restype = ctypes.c_int
        L.fbref_nnf_segment.argtypes = [_u8p, _u8p, _u8p, _u8p, _u8p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, _P, ctypes.c_uint32, ctypes.c_int, _u32p,
                                        _u32p, _i32p, _i32p, _u32p]
        L.fbref_nnf_segment.restype = ctypes.c_int
        L.fbref_interpolate_aligned.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                _i32p, _u8p, ctypes.c_int, _P, ctypes.c_uint32,
                                                ctypes.c_int, _f32p]
        L.fbref_interpolate_aligned.restype = ctypes.c_int
        L.fbref_blend_frame_accurate.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, _P, ctypes.c_uint32,
                                                 ctypes.c_int, _f32p, _u8p, _i32p]
        L.fbref_blend_frame_accurate.restype = ctypes.c_int
        L.fbref_blend_window_accurate.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_int, _P, ctypes.c_uint32,
                                                  _f32p]
        L.fbref_blend_window_accurate.restype = ctypes.c_int
        L.fbref_blend_frame_fast.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, _P, ctypes.c_int, _f32p]
        L.fbref_blend_frame_fast.restype = ctypes.c_int
        L.fbref_blend_window_fast.argtypes = [_u8p, _u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, _P, _f32p]
        L.fbref_blend_window_fast.restype = ctypes.c_int
        L.fbref_pair_tag.argtypes = [ctypes.c_int, ctypes.c_int]
        L.fbref_pair_tag.restype = ctypes.c_uint32
        L.fbref_num_threads.restype = ctypes.c_int
        L.fbref_set_num_threads.argtypes = [ctypes.c_int]
        for name in ("fbref_nnf", "fbref_nnf_trace", "fbref_blend_window", "fbref_blend_frame",
                     "fbref_interpolate", "fbref_interpolate_frame"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    assert a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous"
    return a.ctypes.data_as(ctype)


def _u8(a) -> np.ndarray:
    a = np.ascontiguousarray(a)
    assert a.dtype == np.uint8, a.dtype
    return a


def params(patch: int, iters: int, levels: int = 1, r0: int = 0, seed: int = 0) -> Params:
    return Params(patch, iters, levels, r0, seed & 0xFFFFFFFFFFFFFFFF)


def num_threads() -> int:
    return lib().fbref_num_threads()


def set_num_threads(n: int) -> None:
    lib().fbref_set_num_threads(int(n))


def pair_tag(j: int, i: int) -> int:
    return lib().fbref_pair_tag(j, i)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().fbref_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
    return out


def ssd(src, tgt, k: int, u, x) -> int:
    src, tgt = _u8(src), _u8(tgt)
    H, W = src.shape[:2]
    return int(lib().fbref_ssd(_ptr(src, _u8p), _ptr(tgt, _u8p), H, W, k,
                               int(u[0]), int(u[1]), int(x[0]), int(x[1])))


def downsample(img) -> np.ndarray:
    img = _u8(img)
    H, W = img.shape[:2]
    out = np.zeros(((H + 1) // 2, (W + 1) // 2, 3), np.uint8)
    lib().fbref_downsample(_ptr(img, _u8p), H, W, _ptr(out, _u8p))
    return out


def rs_offset(seed: int, pix: int, tag: int, level: int, it: int, t: int, r: int):
    dr, dc = ctypes.c_int32(), ctypes.c_int32()
    lib().fbref_rs_offset(seed, pix, tag, level, it, t, r, ctypes.byref(dr), ctypes.byref(dc))
    return dr.value, dc.value


def nnf(src, tgt, patch: int, iters: int, levels: int = 1, r0: int = 0, seed: int = 0,
        pair_tag: int = 0, init=None):
    """Alg. 1 for one pair; returns (F (H,W,2) int32, E (H,W) uint32)."""
    src, tgt = _u8(src), _u8(tgt)
    H, W = src.shape[:2]
    F = np.zeros((H, W, 2), np.int32)
    E = np.zeros((H, W), np.uint32)
    p = params(patch, iters, levels, r0, seed)
    ip = None
    if init is not None:
        init = np.ascontiguousarray(init, dtype=np.int32)
        ip = _ptr(init, _i32p)
    rc = lib().fbref_nnf(_ptr(src, _u8p), _ptr(tgt, _u8p), H, W, ctypes.byref(p), pair_tag, ip,
                         _ptr(F, _i32p), _ptr(E, _u32p))
    if rc != 0:
        raise ValueError("fbref_nnf: bad arguments")
    return F, E


def nnf_trace(src, tgt, patch: int, iters: int, r0: int = 0, seed: int = 0, pair_tag: int = 0,
              init=None, levels: int = 1):
    """Alg. 1 returning the full-resolution E before the first and after each iteration
    of level 0: (iters+1, H, W).  With levels > 1, T[0] is the error of the field
    upsampled from the coarser level."""
    src, tgt = _u8(src), _u8(tgt)
    H, W = src.shape[:2]
    F = np.zeros((H, W, 2), np.int32)
    T = np.zeros((iters + 1, H, W), np.uint32)
    p = params(patch, iters, levels, r0, seed)
    ip = None
    if init is not None:
        init = np.ascontiguousarray(init, dtype=np.int32)
        ip = _ptr(init, _i32p)
    rc = lib().fbref_nnf_trace(_ptr(src, _u8p), _ptr(tgt, _u8p), H, W, ctypes.byref(p), pair_tag,
                               ip, _ptr(F, _i32p), _ptr(T, _u32p))
    if rc != 0:
        raise ValueError("fbref_nnf_trace: bad arguments")
    return F, T


def nnf_bruteforce(src, tgt, patch: int):
    src, tgt = _u8(src), _u8(tgt)
    H, W = src.shape[:2]
    F = np.zeros((H, W, 2), np.int32)
    E = np.zeros((H, W), np.uint32)
    lib().fbref_nnf_bruteforce(_ptr(src, _u8p), _ptr(tgt, _u8p), H, W, patch,
                               _ptr(F, _i32p), _ptr(E, _u32p))
    return F, E


def remap_sum(style, F, patch: int) -> np.ndarray:
    style = _u8(style)
    F = np.ascontiguousarray(F, dtype=np.int32)
    H, W = style.shape[:2]
    V = np.zeros((H, W, 3), np.uint32)
    lib().fbref_remap_sum(_ptr(style, _u8p), _ptr(F, _i32p), H, W, patch, _ptr(V, _u32p))
    return V


def remap(style, F, patch: int) -> np.ndarray:
    style = _u8(style)
    F = np.ascontiguousarray(F, dtype=np.int32)
    H, W = style.shape[:2]
    out = np.zeros((H, W, 3), np.float32)
    lib().fbref_remap(_ptr(style, _u8p), _ptr(F, _i32p), H, W, patch, _ptr(out, _f32p))
    return out


def blend_window(guides, styles, window: int, patch: int, iters: int, levels: int = 1,
                 r0: int = 0, seed: int = 0) -> np.ndarray:
    guides, styles = _u8(guides), _u8(styles)
    N, H, W = guides.shape[:3]
    out = np.zeros((N, H, W, 3), np.float32)
    p = params(patch, iters, levels, r0, seed)
    rc = lib().fbref_blend_window(_ptr(guides, _u8p), _ptr(styles, _u8p), N, H, W, window,
                                  ctypes.byref(p), _ptr(out, _f32p))
    if rc != 0:
        raise ValueError("fbref_blend_window: bad arguments")
    return out


def blend_frame(guides, styles, window: int, i: int, patch: int, iters: int, levels: int = 1,
                r0: int = 0, seed: int = 0) -> np.ndarray:
    guides, styles = _u8(guides), _u8(styles)
    N, H, W = guides.shape[:3]
    out = np.zeros((H, W, 3), np.float32)
    p = params(patch, iters, levels, r0, seed)
    rc = lib().fbref_blend_frame(_ptr(guides, _u8p), _ptr(styles, _u8p), N, H, W, window,
                                 ctypes.byref(p), i, _ptr(out, _f32p))
    if rc != 0:
        raise ValueError("fbref_blend_frame: bad arguments")
    return out


def interpolate(guides, key_idx, key_styles, patch: int, iters: int, levels: int = 1,
                r0: int = 0, seed: int = 0) -> np.ndarray:
    guides, key_styles = _u8(guides), _u8(key_styles)
    keys = np.ascontiguousarray(key_idx, dtype=np.int32)
    N, H, W = guides.shape[:3]
    out = np.zeros((N, H, W, 3), np.float32)
    p = params(patch, iters, levels, r0, seed)
    rc = lib().fbref_interpolate(_ptr(guides, _u8p), N, H, W, _ptr(keys, _i32p),
                                 _ptr(key_styles, _u8p), len(keys), ctypes.byref(p),
                                 _ptr(out, _f32p))
    if rc != 0:
        raise ValueError("fbref_interpolate: bad arguments")
    return out


def interpolate_frame(guides, key_idx, key_styles, i: int, patch: int, iters: int,
                      levels: int = 1, r0: int = 0, seed: int = 0) -> np.ndarray:
    guides, key_styles = _u8(guides), _u8(key_styles)
    keys = np.ascontiguousarray(key_idx, dtype=np.int32)
    N, H, W = guides.shape[:3]
    out = np.zeros((H, W, 3), np.float32)
    p = params(patch, iters, levels, r0, seed)
    rc = lib().fbref_interpolate_frame(_ptr(guides, _u8p), N, H, W, _ptr(keys, _i32p),
                                       _ptr(key_styles, _u8p), len(keys), ctypes.byref(p), i,
                                       _ptr(out, _f32p))
    if rc != 0:
        raise ValueError("fbref_interpolate_frame: bad arguments")
    return out


# ----------------------------------------------------------------------------------
# Sec. 3.4 improved loss ("balanced mode")
# ----------------------------------------------------------------------------------
def shat(style, nnf, patch: int) -> np.ndarray:
    """The remap (Alg. 2) of `style` through `nnf`, rounded to 8-bit values."""
    style = _u8(style)
    H, W = style.shape[:2]
    nnf = np.ascontiguousarray(nnf, dtype=np.int32)
    out = np.zeros((H, W, 3), np.uint8)
    lib().fbref_shat(_ptr(style, _u8p), _ptr(nnf, _i32p), H, W, patch, _ptr(out, _u8p))
    return out


def nnf_balanced(src_guide, tgt_guide, src_style, patch: int, iters: int, alpha: int,
                 r0: int = 0, seed: int = 0, pair_tag: int = 0, init=None):
    """Alg. 1 under the improved loss; returns (F, E, S^ of the last iteration)."""
    gs, gt, ss = _u8(src_guide), _u8(tgt_guide), _u8(src_style)
    H, W = gs.shape[:2]
    F = np.zeros((H, W, 2), np.int32)
    E = np.zeros((H, W), np.uint32)
    S = np.zeros((H, W, 3), np.uint8)
    p = params(patch, iters, 1, r0, seed)
    ip = None
    if init is not None:
        init = np.ascontiguousarray(init, dtype=np.int32)
        ip = _ptr(init, _i32p)
    rc = lib().fbref_nnf_balanced(_ptr(gs, _u8p), _ptr(gt, _u8p), _ptr(ss, _u8p), H, W,
                                  ctypes.byref(p), alpha, pair_tag, ip, _ptr(F, _i32p),
                                  _ptr(E, _u32p), _ptr(S, _u8p))
    if rc != 0:
        raise ValueError("fbref_nnf_balanced: bad arguments")
    return F, E, S


def blend_frame_balanced(guides, styles, window: int, i: int, patch: int, iters: int,
                         alpha: int, seed: int = 0):
    g, s = _u8(guides), _u8(styles)
    N, H, W = g.shape[:3]
    out = np.zeros((H, W, 3), np.float32)
    p = params(patch, iters, 1, 0, seed)
    rc = lib().fbref_blend_frame_balanced(_ptr(g, _u8p), _ptr(s, _u8p), N, H, W, window,
                                          ctypes.byref(p), alpha, i, _ptr(out, _f32p))
    if rc != 0:
        raise ValueError("fbref_blend_frame_balanced: bad arguments")
    return out


def blend_window_balanced(guides, styles, window: int, patch: int, iters: int, alpha: int,
                          seed: int = 0):
    g, s = _u8(guides), _u8(styles)
    N, H, W = g.shape[:3]
    out = np.zeros((N, H, W, 3), np.float32)
    p = params(patch, iters, 1, 0, seed)
    rc = lib().fbref_blend_window_balanced(_ptr(g, _u8p), _ptr(s, _u8p), N, H, W, window,
                                           ctypes.byref(p), alpha, _ptr(out, _f32p))
    if rc != 0:
        raise ValueError("fbref_blend_window_balanced: bad arguments")
    return out


# ----------------------------------------------------------------------------------
# Sec. 3.4 fast mode (Algs. 3-5)
# ----------------------------------------------------------------------------------
def blend_frame_fast(guides, styles, window: int, i: int, patch: int, iters: int, seed: int = 0):
    g, s = _u8(guides), _u8(styles)
    N, H, W = g.shape[:3]
    out = np.zeros((H, W, 3), np.float32)
    p = params(patch, iters, 1, 0, seed)
    rc = lib().fbref_blend_frame_fast(_ptr(g, _u8p), _ptr(s, _u8p), N, H, W, window,
                                      ctypes.byref(p), i, _ptr(out, _f32p))
    if rc != 0:
        raise ValueError("fbref_blend_frame_fast: bad arguments")
    return out


def blend_window_fast(guides, styles, window: int, patch: int, iters: int, seed: int = 0):
    g, s = _u8(guides), _u8(styles)
    N, H, W = g.shape[:3]
    out = np.zeros((N, H, W, 3), np.float32)
    p = params(patch, iters, 1, 0, seed)
    rc = lib().fbref_blend_window_fast(_ptr(g, _u8p), _ptr(s, _u8p), N, H, W, window,
                                       ctypes.byref(p), _ptr(out, _f32p))
    if rc != 0:
        raise ValueError("fbref_blend_window_fast: bad arguments")
    return out


# ----------------------------------------------------------------------------------
# Sec. 3.4 quality improvement ("accurate mode")
# ----------------------------------------------------------------------------------
def blend_frame_accurate(guides, styles, window: int, i: int, patch: int, iters: int, alpha: int,
                         seed: int = 0):
    """Output frame i, the mean remapped frame Tbar_i of the last iteration and the final
    fields of the pairs (j -> i), j ascending: (out, tbar, F (pairs, H, W, 2))."""
    g, s = _u8(guides), _u8(styles)
    N, H, W = g.shape[:3]
    M = (window - 1) // 2
    n_pairs = min(N - 1, i + M) - max(0, i - M)
    out = np.zeros((H, W, 3), np.float32)
    tbar = np.zeros((H, W, 3), np.uint8)
    F = np.zeros((max(n_pairs, 1), H, W, 2), np.int32)
    p = params(patch, iters, 1, 0, seed)
    rc = lib().fbref_blend_frame_accurate(_ptr(g, _u8p), _ptr(s, _u8p), N, H, W, window,
                                          ctypes.byref(p), alpha, i, _ptr(out, _f32p),
                                          _ptr(tbar, _u8p), _ptr(F, _i32p))
    if rc != 0:
        raise ValueError("fbref_blend_frame_accurate: bad arguments")
    return out, tbar, F[:n_pairs]


def blend_window_accurate(guides, styles, window: int, patch: int, iters: int, alpha: int,
                          seed: int = 0):
    g, s = _u8(guides), _u8(styles)
    N, H, W = g.shape[:3]
    out = np.zeros((N, H, W, 3), np.float32)
    p = params(patch, iters, 1, 0, seed)
    rc = lib().fbref_blend_window_accurate(_ptr(g, _u8p), _ptr(s, _u8p), N, H, W, window,
                                           ctypes.byref(p), alpha, _ptr(out, _f32p))
    if rc != 0:
        raise ValueError("fbref_blend_window_accurate: bad arguments")
    return out


# ----------------------------------------------------------------------------------
# Sec. 3.5.1 tracking
# ----------------------------------------------------------------------------------
def nnf_chain(src, tgts, patch: int, iters: int, tags, r0: int = 0, seed: int = 0, init=None):
    """NNFs from `src` to the consecutive frames `tgts` (n, H, W, 3) with tracking;
    returns (F (n, H, W, 2), E (n, H, W))."""
    src, tgts = _u8(src), _u8(tgts)
    n, H, W = tgts.shape[:3]
    F = np.zeros((n, H, W, 2), np.int32)
    E = np.zeros((n, H, W), np.uint32)
    t = np.ascontiguousarray(tags, dtype=np.uint32)
    p = params(patch, iters, 1, r0, seed)
    ip = None
    if init is not None:
        init = np.ascontiguousarray(init, dtype=np.int32)
        ip = _ptr(init, _i32p)
    rc = lib().fbref_nnf_chain(_ptr(src, _u8p), _ptr(tgts, _u8p), n, H, W, ctypes.byref(p),
                               _ptr(t, _u32p), ip, _ptr(F, _i32p), _ptr(E, _u32p))
    if rc != 0:
        raise ValueError("fbref_nnf_chain: bad arguments")
    return F, E


def nnf_segment(guide_l, guide_r, style_l, style_r, tgts, patch: int, iters: int, alpha: int,
                tags_l, tags_r, tracking: bool = False, r0: int = 0, seed: int = 0, init=None):
    """Coupled NNFs of Eq. 10 from keys l and r to the frames `tgts` (n, H, W, 3) between
    them; returns (F (2, n, H, W, 2), E (2, n, H, W)), index 0 the left key's fields."""
    gl, gr, sl, sr, tgts = (_u8(a) for a in (guide_l, guide_r, style_l, style_r, tgts))
    n, H, W = tgts.shape[:3]
    F = np.zeros((2, n, H, W, 2), np.int32)
    E = np.zeros((2, n, H, W), np.uint32)
    tl = np.ascontiguousarray(tags_l, dtype=np.uint32)
    tr = np.ascontiguousarray(tags_r, dtype=np.uint32)
    p = params(patch, iters, 1, r0, seed)
    ip = None
    if init is not None:
        init = np.ascontiguousarray(init, dtype=np.int32)
        ip = _ptr(init, _i32p)
    rc = lib().fbref_nnf_segment(_ptr(gl, _u8p), _ptr(gr, _u8p), _ptr(sl, _u8p), _ptr(sr, _u8p),
                                 _ptr(tgts, _u8p), n, H, W, ctypes.byref(p), alpha, int(tracking),
                                 _ptr(tl, _u32p), _ptr(tr, _u32p), ip, _ptr(F, _i32p),
                                 _ptr(E, _u32p))
    if rc != 0:
        raise ValueError("fbref_nnf_segment: bad arguments")
    return F, E


def interpolate_aligned(guides, key_idx, key_styles, patch: int, iters: int, alpha: int,
                        tracking: bool = False, seed: int = 0):
    g, ks = _u8(guides), _u8(key_styles)
    N, H, W = g.shape[:3]
    keys = np.ascontiguousarray(key_idx, dtype=np.int32)
    out = np.zeros((N, H, W, 3), np.float32)
    p = params(patch, iters, 1, 0, seed)
    rc = lib().fbref_interpolate_aligned(_ptr(g, _u8p), N, H, W, _ptr(keys, _i32p),
                                         _ptr(ks, _u8p), len(keys), ctypes.byref(p), alpha,
                                         int(tracking), _ptr(out, _f32p))
    if rc != 0:
        raise ValueError("fbref_interpolate_aligned: bad arguments")
    return out


def interpolate_tracking(guides, key_idx, key_styles, patch: int, iters: int, seed: int = 0):
    g, ks = _u8(guides), _u8(key_styles)
    N, H, W = g.shape[:3]
    keys = np.ascontiguousarray(key_idx, dtype=np.int32)
    out = np.zeros((N, H, W, 3), np.float32)
    p = params(patch, iters, 1, 0, seed)
    rc = lib().fbref_interpolate_tracking(_ptr(g, _u8p), N, H, W, _ptr(keys, _i32p), _ptr(ks, _u8p),
                                          len(keys), ctypes.byref(p), _ptr(out, _f32p))
    if rc != 0:
        raise ValueError("fbref_interpolate_tracking: bad arguments")
    return out


def blend_window_tracking(guides, styles, window: int, patch: int, iters: int, seed: int = 0):
    """Eq. 2 blend whose NNFs from each source frame to the targets before / after it are
    computed as two tracking chains (Sec. 3.5.1, one level)."""
    g, s = _u8(guides), _u8(styles)
    N, H, W = g.shape[:3]
    out = np.zeros((N, H, W, 3), np.float32)
    p = params(patch, iters, 1, 0, seed)
    rc = lib().fbref_blend_window_tracking(_ptr(g, _u8p), _ptr(s, _u8p), N, H, W, window,
                                           ctypes.byref(p), _ptr(out, _f32p))
    if rc != 0:
        raise ValueError("fbref_blend_window_tracking: bad arguments")
    return out
