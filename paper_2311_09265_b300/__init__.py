"""FastBlend hot path (arXiv 2311.09265) on B300 -- Python binding of libfb.so.

This module only marshals arguments: every step of the path (patch matching, remap,
blend, interpolation) runs in the CUDA kernels of libfb.so behind the C ABI declared
in include/fb.h.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if libfb.so is missing or cannot load, every call raises.

Names follow the C ABI: fb_nnf, fb_remap, fb_blend_window, fb_interpolate, plus
Context (fb_ctx_*) and Params (fb_params).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

from ._build import LIB_PATH, build  # noqa: F401  (build is re-exported)

FB_OK, FB_ERR_ARG, FB_ERR_CUDA, FB_ERR_OOM, FB_ERR_TIMEOUT, FB_ERR_UNSUPPORTED = range(6)

HEADER_FUNCTIONS = ("fb_ctx_create", "fb_ctx_destroy", "fb_ctx_sync", "fb_last_error",
                    "fb_status_string", "fb_ctx_launches", "fb_ctx_scratch_bytes",
                    "fb_ctx_profile", "fb_ctx_profile_read", "fb_probe_dp4a", "fb_probe_ssd_mix",
                    "fb_debug_candidates_considered", "fb_pair_tag",
                    "fb_nnf", "fb_nnf_balanced", "fb_nnf_segment", "fb_remap", "fb_blend_window", "fb_interpolate",
                    "fb_blend_window_range", "fb_interpolate_range", "fb_shard_plan", "fb_pair_plan_range",
                    "fb_blend_window_noalloc", "fb_blend_batch", "fb_batch_plan", "fb_fast_plan", "fb_pair_plan",
                    "fb_ctx_batch_variant", "fb_ctx_batch_claim", "fb_ctx_batch_mode", "fb_ctx_set_pair_budget",
                    "fb_initnet_create", "fb_initnet_destroy", "fb_initnet_last_error",
                    "fb_initnet_param_count", "fb_initnet_get_params", "fb_initnet_set_params",
                    "fb_initnet_get_grads", "fb_initnet_forward", "fb_initnet_init_nnf", "fb_conv_gemm_path",
                    "fb_initnet_get_optimizer", "fb_initnet_set_optimizer",
                    "fb_initnet_train_step", "fb_initnet_status", "fb_conv3x3_forward",
                    "fb_conv3x3_backward", "fb_ctx_set_initnet", "fb_ctx_energy",
                    "fb_initnet_targets", "fb_debug_set_wait_limit", "fb_nnf_step", "fb_check_status", "fb_probe_gather")

FB_FLAG_LEARNED_INIT = 0x1
FB_FLAG_REPORT_ENERGY = 0x2
FB_FLAG_BALANCED = 0x4
FB_FLAG_FAST = 0x8
FB_FLAG_ACCURATE = 0x10
FB_FLAG_TRACKING = 0x20
FB_FLAG_ALIGN = 0x40

FB_BATCH_NO_GRAPH = 0x1

# Device-side check sites of the checked build (fb_check_status).
FB_CHECK_CANDIDATE, FB_CHECK_SNAPSHOT, FB_CHECK_ENERGY, FB_CHECK_SLOT, FB_CHECK_TABLE, FB_CHECK_REMAP = range(1, 7)


def FB_BATCH_CLAIM(c: int) -> int:
    return (int(c) & 0xFF) << 16


def FB_BATCH_VARIANT(v: int) -> int:
    """Flag that forces tile variant v (0..3) of the batched path."""
    return (v + 1) << 8

# fb_kernel_kind, in header order.
KERNEL_KINDS = ("prep", "downsample", "style", "init", "iter", "unpack", "pack", "combine",
                "initnet", "shat", "energy", "table")


class Params(ctypes.Structure):
    """fb_params: Alg. 1 parameters (patch k, iterations, pyramid levels, r0, seed)."""
    _fields_ = [("patch", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("r0", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("pair_tag", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("alpha", ctypes.c_uint32)]

    @classmethod
    def make(cls, patch: int, iters: int, levels: int = 1, r0: int = 0, seed: int = 0,
             pair_tag: int = 0, flags: int = 0, alpha: int = 0) -> "Params":
        return cls(patch, iters, levels, r0, seed & 0xFFFFFFFFFFFFFFFF, pair_tag & 0xFFFFFFFF,
                   flags, alpha)


class PairInfo(ctypes.Structure):
    """fb_pair_info: one NNF of a blend or interpolation call."""
    _fields_ = [("src", ctypes.c_int32), ("tgt", ctypes.c_int32), ("tag", ctypes.c_uint32),
                ("weight", ctypes.c_uint32), ("prev", ctypes.c_int32), ("next", ctypes.c_int32),
                ("partner", ctypes.c_int32), ("out_frame", ctypes.c_int32)]


class ClipDesc(ctypes.Structure):
    """fb_clip_desc: one clip of a batched submission (device pointers)."""
    _fields_ = [("guides", ctypes.c_void_p), ("styles", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("N", ctypes.c_int32), ("H", ctypes.c_int32),
                ("W", ctypes.c_int32), ("window", ctypes.c_int32), ("patch", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class FastBlendError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_STATUS_NAMES = {0: "FB_OK", 1: "FB_ERR_ARG", 2: "FB_ERR_CUDA", 3: "FB_ERR_OOM",
                 4: "FB_ERR_TIMEOUT", 5: "FB_ERR_UNSUPPORTED"}

_lib: Optional[ctypes.CDLL] = None
_vp = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Load libfb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "or python -m paper_2311_09265_b300._build")
        L = ctypes.CDLL(LIB_PATH)
        L.fb_ctx_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int]
        L.fb_ctx_destroy.argtypes = [_vp]
        L.fb_ctx_sync.argtypes = [_vp, _vp]
        L.fb_last_error.argtypes = [_vp]
        L.fb_last_error.restype = ctypes.c_char_p
        L.fb_status_string.argtypes = [ctypes.c_int]
        L.fb_status_string.restype = ctypes.c_char_p
        L.fb_ctx_launches.argtypes = [_vp]
        L.fb_ctx_launches.restype = ctypes.c_uint64
        L.fb_ctx_scratch_bytes.argtypes = [_vp]
        L.fb_ctx_scratch_bytes.restype = ctypes.c_size_t
        L.fb_ctx_profile.argtypes = [_vp, ctypes.c_int]
        L.fb_ctx_profile_read.argtypes = [_vp, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_uint64)]
        L.fb_probe_dp4a.argtypes = [_vp, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]
        L.fb_probe_dp4a.restype = ctypes.c_int
        L.fb_probe_ssd_mix.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
        L.fb_probe_ssd_mix.restype = ctypes.c_int
        L.fb_probe_gather.argtypes = [_vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
        L.fb_probe_gather.restype = ctypes.c_int
        L.fb_debug_candidates_considered.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]
        L.fb_debug_candidates_considered.restype = ctypes.c_int
        L.fb_pair_tag.argtypes = [ctypes.c_int, ctypes.c_int]
        L.fb_pair_tag.restype = ctypes.c_uint32
        P = ctypes.POINTER(Params)
        L.fb_nnf.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, P, _vp, _vp, _vp, _vp]
        L.fb_nnf_step.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, _vp, _vp,
                                  _vp, _vp, _vp]
        L.fb_nnf_step.restype = ctypes.c_int
        L.fb_check_status.argtypes = [ctypes.POINTER(ctypes.c_uint64)] * 3 + [ctypes.c_int]
        L.fb_check_status.restype = ctypes.c_int
        L.fb_nnf_segment.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                     _vp, _vp, _vp, _vp]
        L.fb_nnf_balanced.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, P, _vp, _vp,
                                      _vp, _vp, _vp]
        L.fb_fast_plan.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.POINTER(ctypes.c_uint64)] * 3
        L.fb_conv_gemm_path.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
        L.fb_pair_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                   ctypes.c_uint32, ctypes.POINTER(PairInfo), ctypes.c_size_t,
                                   ctypes.POINTER(ctypes.c_size_t)]
        L.fb_remap.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]
        L.fb_blend_window.argtypes = [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, P, _vp, _vp]
        L.fb_interpolate.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp,
                                     _vp, ctypes.c_int, P, _vp, _vp]
        L.fb_blend_window_noalloc.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, P, _vp, _vp]
        ci = ctypes.c_int
        L.fb_blend_window_range.argtypes = [_vp, _vp, _vp, ci, ci, ci, ci, P, ci, ci, ci, ci, _vp, _vp]
        L.fb_blend_window_range.restype = ctypes.c_int
        L.fb_interpolate_range.argtypes = [_vp, _vp, ci, ci, ci, _vp, _vp, ci, P, ci, ci, _vp, _vp]
        L.fb_interpolate_range.restype = ctypes.c_int
        L.fb_shard_plan.argtypes = [ci, ci, ci, ci] + [ctypes.POINTER(ci)] * 4
        L.fb_shard_plan.restype = ctypes.c_int
        L.fb_pair_plan_range.argtypes = [ci, ci, ctypes.POINTER(ctypes.c_int32), ci, ctypes.c_uint32, ci, ci,
                                         ctypes.POINTER(PairInfo), ctypes.c_size_t,
                                         ctypes.POINTER(ctypes.c_size_t)]
        L.fb_pair_plan_range.restype = ctypes.c_int
        L.fb_blend_window_noalloc.restype = ctypes.c_int
        CP = ctypes.POINTER(ClipDesc)
        L.fb_blend_batch.argtypes = [_vp, CP, ctypes.c_int, P, ctypes.c_uint32, _vp]
        L.fb_blend_batch.restype = ctypes.c_int
        L.fb_batch_plan.argtypes = [CP, ctypes.c_int, P, ctypes.c_size_t,
                                    ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                    ctypes.POINTER(ctypes.c_int)]
        L.fb_batch_plan.restype = ctypes.c_int
        L.fb_initnet_create.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int]
        L.fb_initnet_destroy.argtypes = [_vp]
        L.fb_initnet_last_error.argtypes = [_vp]
        L.fb_initnet_last_error.restype = ctypes.c_char_p
        L.fb_initnet_param_count.argtypes = [_vp]
        L.fb_initnet_param_count.restype = ctypes.c_size_t
        for f in ("fb_initnet_get_params", "fb_initnet_set_params", "fb_initnet_get_grads"):
            getattr(L, f).argtypes = [_vp, _vp]
        L.fb_initnet_get_optimizer.argtypes = [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_uint64)]
        L.fb_initnet_set_optimizer.argtypes = [_vp, _vp, _vp, ctypes.c_uint64]
        L.fb_initnet_forward.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp]
        L.fb_initnet_init_nnf.argtypes = [_vp, ctypes.c_int, _vp, _vp]
        L.fb_initnet_train_step.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, ctypes.c_float,
                                            ctypes.c_float, _vp, _vp]
        L.fb_initnet_status.argtypes = [_vp]
        L.fb_debug_set_wait_limit.argtypes = [ctypes.c_int64]
        L.fb_debug_set_wait_limit.restype = ctypes.c_int
        L.fb_conv3x3_forward.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _vp, _vp, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _vp, _vp, _vp, _vp]
        L.fb_conv3x3_backward.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                          _vp, _vp, _vp]
        for f in ("fb_initnet_create", "fb_initnet_destroy", "fb_initnet_get_params",
                  "fb_initnet_set_params", "fb_initnet_get_grads", "fb_initnet_forward",
                  "fb_initnet_init_nnf", "fb_initnet_train_step", "fb_initnet_status",
                  "fb_initnet_get_optimizer", "fb_initnet_set_optimizer",
                  "fb_conv3x3_forward", "fb_conv3x3_backward"):
            getattr(L, f).restype = ctypes.c_int
        L.fb_ctx_set_initnet.argtypes = [_vp, _vp]
        L.fb_ctx_set_initnet.restype = ctypes.c_int
        L.fb_ctx_energy.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64)]
        L.fb_ctx_energy.restype = ctypes.c_int
        L.fb_initnet_targets.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         _vp, _vp, _vp]
        L.fb_initnet_targets.restype = ctypes.c_int
        L.fb_ctx_set_pair_budget.argtypes = [_vp, ctypes.c_size_t]
        L.fb_ctx_set_pair_budget.restype = ctypes.c_int
        L.fb_ctx_batch_variant.argtypes = [_vp, ctypes.c_int]
        L.fb_ctx_batch_variant.restype = ctypes.c_int
        L.fb_ctx_batch_claim.argtypes = [_vp, ctypes.c_int]
        L.fb_ctx_batch_claim.restype = ctypes.c_int
        L.fb_ctx_batch_mode.argtypes = [_vp, ctypes.c_int]
        L.fb_ctx_batch_mode.restype = ctypes.c_int
        for f in ("fb_ctx_create", "fb_ctx_destroy", "fb_ctx_sync", "fb_ctx_profile",
                  "fb_ctx_profile_read", "fb_nnf", "fb_remap",
                  "fb_blend_window", "fb_interpolate"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def fb_fast_plan(N: int, window: int):
    """(distinct NNFs, blending-table entries, query pieces) of the fast mode (host only)."""
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    rc = lib().fb_fast_plan(N, window, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_fast_plan")
    return int(a.value), int(b.value), int(c.value)


def fb_pair_plan(N: int, window: int = 0, keys=None, flags: int = 0):
    """The NNFs a blend (window > 0) or interpolation (keys) call enumerates, in its order
    (host only): a list of dicts with src, tgt, tag, weight, prev, next, partner, out_frame."""
    karr, nk = None, 0
    if keys is not None:
        nk = len(keys)
        karr = (ctypes.c_int32 * max(nk, 1))(*keys)
    n = ctypes.c_size_t()
    rc = lib().fb_pair_plan(N, window, karr, nk, flags, None, 0, ctypes.byref(n))
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_pair_plan")
    out = (PairInfo * max(n.value, 1))()
    rc = lib().fb_pair_plan(N, window, karr, nk, flags, out, n.value, ctypes.byref(n))
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_pair_plan")
    return [{f: getattr(out[q], f) for f, _ in PairInfo._fields_} for q in range(n.value)]


def fb_pair_plan_range(N: int, out_first: int, n_out: int, window: int = 0, keys=None,
                       flags: int = 0):
    """The NNFs of a range call over output frames [out_first, out_first + n_out) of an
    N-frame clip (host only), as fb_pair_plan lists them (clip frame indices)."""
    karr, nk = None, 0
    if keys is not None:
        nk = len(keys)
        karr = (ctypes.c_int32 * max(nk, 1))(*keys)
    n = ctypes.c_size_t()
    rc = lib().fb_pair_plan_range(N, window, karr, nk, flags, out_first, n_out, None, 0, ctypes.byref(n))
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_pair_plan_range")
    out = (PairInfo * max(n.value, 1))()
    rc = lib().fb_pair_plan_range(N, window, karr, nk, flags, out_first, n_out, out, n.value, ctypes.byref(n))
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_pair_plan_range")
    return [{f: getattr(out[q], f) for f, _ in PairInfo._fields_} for q in range(n.value)]


def fb_shard_plan(N: int, window: int, n_shards: int, shard: int) -> dict:
    """Shard `shard` of an N-frame clip split over n_shards GPUs (host only): its output
    frames [out_first, out_first + n_out) and input frames [frame_base, frame_base + n_in)."""
    v = [ctypes.c_int() for _ in range(4)]
    rc = lib().fb_shard_plan(N, window, n_shards, shard, *[ctypes.byref(x) for x in v])
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_shard_plan")
    return dict(zip(("frame_base", "n_in", "out_first", "n_out"), (int(x.value) for x in v)))


def fb_conv_gemm_path(mode: int = -1) -> int:
    """Set the forward convolutions' operand staging (0: TMA where eligible, 1: cp.async
    gathers; -1: unchanged); returns the number of TMA-staged launches so far."""
    n = ctypes.c_uint64()
    rc = lib().fb_conv_gemm_path(mode, ctypes.byref(n))
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_conv_gemm_path")
    return int(n.value)


def fb_debug_candidates_considered(reset: bool = False) -> int:
    """Candidates considered by the per-call NNF kernels since the last reset (debug
    builds, libfb_debug.so, only; the product library raises FB_ERR_UNSUPPORTED)."""
    v = ctypes.c_uint64()
    rc = lib().fb_debug_candidates_considered(ctypes.byref(v), 1 if reset else 0)
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_debug_candidates_considered")
    return int(v.value)


def fb_check_status(reset: bool = False):
    """(first failure word, failed checks, visits) of the device-side checks of a checked
    build (libfb_checked.so); the first failure word is (site << 56) | (a << 28) | b, 0 if
    none.  The product library raises FB_ERR_UNSUPPORTED."""
    first, failed, evaluated = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    rc = lib().fb_check_status(ctypes.byref(first), ctypes.byref(failed), ctypes.byref(evaluated),
                               1 if reset else 0)
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_check_status")
    return int(first.value), int(failed.value), int(evaluated.value)


def fb_debug_set_wait_limit(polls: int) -> None:
    """Polls of the tensor-core kernels' progress waits on the current device (0: give up
    at once; < 0: the default); for exercising the timeout path."""
    rc = lib().fb_debug_set_wait_limit(int(polls))
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_debug_set_wait_limit")


def fb_pair_tag(j: int, i: int) -> int:
    return lib().fb_pair_tag(j, i)


class Context:
    """fb_ctx: owns device scratch for one CUDA device.  Not thread-safe."""

    def __init__(self, device: int = 0):
        h = _vp()
        rc = lib().fb_ctx_create(ctypes.byref(h), device)
        if rc != FB_OK:
            raise FastBlendError(rc, lib().fb_last_error(None).decode())
        self._h = h
        self.device = device

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().fb_ctx_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc: int) -> None:
        if rc != FB_OK:
            raise FastBlendError(rc, lib().fb_last_error(self._h).decode())

    @property
    def launches(self) -> int:
        return int(lib().fb_ctx_launches(self._h))

    @property
    def scratch_bytes(self) -> int:
        return int(lib().fb_ctx_scratch_bytes(self._h))

    def profile(self, enable: bool) -> None:
        """Start (clearing earlier records) or stop per-launch CUDA-event timing."""
        self.check(lib().fb_ctx_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{kernel kind: (total ms, launches)} recorded since profiling was enabled."""
        n = len(KERNEL_KINDS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_uint64 * n)()
        self.check(lib().fb_ctx_profile_read(self._h, ms, cnt))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_KINDS)}

    def probe_dp4a(self):
        """(dp4a instructions per second, kernel ms) of a register-only probe."""
        rate, ms = ctypes.c_double(), ctypes.c_double()
        self.check(lib().fb_probe_dp4a(self._h, ctypes.byref(rate), ctypes.byref(ms)))
        return rate.value, ms.value

    def probe_ssd_mix(self, patch: int = 5):
        """(Eq. 1 byte pairs per second, kernel ms) of a register-only probe of the patch-k
        kernels' per-candidate instruction sequence (k = 5 or 7)."""
        rate, ms = ctypes.c_double(), ctypes.c_double()
        self.check(lib().fb_probe_ssd_mix(self._h, patch, ctypes.byref(rate), ctypes.byref(ms)))
        return rate.value, ms.value

    def probe_gather(self, nbytes: int):
        """(32-byte sectors/s, ms) of scattered 256-bit loads over an nbytes buffer."""
        rate, ms = ctypes.c_double(), ctypes.c_double()
        self.check(lib().fb_probe_gather(self._h, int(nbytes), ctypes.byref(rate), ctypes.byref(ms)))
        return rate.value, ms.value

    def set_initnet(self, net) -> None:
        """Attach the learned initialiser used with FB_FLAG_LEARNED_INIT (None detaches)."""
        self.check(lib().fb_ctx_set_initnet(self._h, net.handle if net is not None else None))

    def energy(self):
        """(sum, count) of final Eq. 1 errors of the last FB_FLAG_REPORT_ENERGY call."""
        s, c = ctypes.c_double(), ctypes.c_uint64()
        self.check(lib().fb_ctx_energy(self._h, ctypes.byref(s), ctypes.byref(c)))
        return s.value, c.value

    def set_pair_budget(self, nbytes: int) -> None:
        """Bytes of NNF scratch per chunk of pairs (0 = library default)."""
        self.check(lib().fb_ctx_set_pair_budget(self._h, int(nbytes)))

    def sync(self, stream: Optional[torch.cuda.Stream] = None) -> None:
        self.check(lib().fb_ctx_sync(self._h, _stream_handle(stream, self.device)))


def _stream_handle(stream, device) -> int:
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return stream.cuda_stream


def _ptr(t: Optional[torch.Tensor], dtype: torch.dtype, name: str):
    if t is None:
        return None
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _shape(t: torch.Tensor, want: Sequence[int], name: str) -> None:
    if tuple(t.shape) != tuple(want):
        raise ValueError(f"{name} must have shape {tuple(want)}, got {tuple(t.shape)}")


def fb_nnf(ctx: Context, src_guide: torch.Tensor, tgt_guide: torch.Tensor, params: Params,
           init_nnf: Optional[torch.Tensor] = None, nnf_out: Optional[torch.Tensor] = None,
           err_out: Optional[torch.Tensor] = None, stream=None):
    """Alg. 1 NNF(src -> tgt) for one pair of H x W x 3 uint8 CUDA tensors.
    Returns (nnf (H,W,2) int32, err (H,W) int32 holding uint32 values)."""
    H, W = int(src_guide.shape[0]), int(src_guide.shape[1])
    _shape(src_guide, (H, W, 3), "src_guide")
    _shape(tgt_guide, (H, W, 3), "tgt_guide")
    dev = src_guide.device
    if nnf_out is None:
        nnf_out = torch.empty((H, W, 2), dtype=torch.int32, device=dev)
    if err_out is None:
        err_out = torch.empty((H, W), dtype=torch.int32, device=dev)
    if init_nnf is not None:
        _shape(init_nnf, (H, W, 2), "init_nnf")
    rc = lib().fb_nnf(ctx.handle, _ptr(src_guide, torch.uint8, "src_guide"),
                      _ptr(tgt_guide, torch.uint8, "tgt_guide"), H, W, ctypes.byref(params),
                      _ptr(init_nnf, torch.int32, "init_nnf"),
                      _ptr(nnf_out, torch.int32, "nnf_out"), _ptr(err_out, torch.int32, "err_out"),
                      _stream_handle(stream, ctx.device))
    ctx.check(rc)
    return nnf_out, err_out


def fb_nnf_step(ctx: Context, src_guide: torch.Tensor, tgt_guide: torch.Tensor, params: Params,
                it: int, nnf_in: torch.Tensor, err_in: torch.Tensor, stream=None):
    """One Jacobi iteration (index it) of Alg. 1 from the snapshot (nnf_in (H,W,2) int32,
    err_in (H,W) int32 holding uint32 errors).  Returns (nnf, err) after the step."""
    H, W = int(src_guide.shape[0]), int(src_guide.shape[1])
    _shape(src_guide, (H, W, 3), "src_guide")
    _shape(tgt_guide, (H, W, 3), "tgt_guide")
    _shape(nnf_in, (H, W, 2), "nnf_in")
    _shape(err_in, (H, W), "err_in")
    dev = src_guide.device
    nnf_out = torch.empty((H, W, 2), dtype=torch.int32, device=dev)
    err_out = torch.empty((H, W), dtype=torch.int32, device=dev)
    rc = lib().fb_nnf_step(ctx.handle, _ptr(src_guide, torch.uint8, "src_guide"),
                           _ptr(tgt_guide, torch.uint8, "tgt_guide"), H, W, ctypes.byref(params), int(it),
                           _ptr(nnf_in, torch.int32, "nnf_in"), _ptr(err_in, torch.int32, "err_in"),
                           _ptr(nnf_out, torch.int32, "nnf_out"), _ptr(err_out, torch.int32, "err_out"),
                           _stream_handle(stream, ctx.device))
    ctx.check(rc)
    return nnf_out, err_out


def fb_nnf_balanced(ctx: Context, src_guide: torch.Tensor, tgt_guide: torch.Tensor,
                    src_style: torch.Tensor, params: Params, init_nnf: Optional[torch.Tensor] = None,
                    stream=None):
    """Alg. 1 under the improved loss of Sec. 3.4 for one pair (params.alpha weighs the
    guide term).  Returns (nnf (H,W,2) int32, err (H,W) int32 holding uint32 values,
    S^ of the last iteration (H,W,3) uint8)."""
    H, W = int(src_guide.shape[0]), int(src_guide.shape[1])
    _shape(src_guide, (H, W, 3), "src_guide")
    _shape(tgt_guide, (H, W, 3), "tgt_guide")
    _shape(src_style, (H, W, 3), "src_style")
    dev = src_guide.device
    nnf_out = torch.empty((H, W, 2), dtype=torch.int32, device=dev)
    err_out = torch.empty((H, W), dtype=torch.int32, device=dev)
    shat_out = torch.empty((H, W, 3), dtype=torch.uint8, device=dev)
    if init_nnf is not None:
        _shape(init_nnf, (H, W, 2), "init_nnf")
    rc = lib().fb_nnf_balanced(ctx.handle, _ptr(src_guide, torch.uint8, "src_guide"),
                               _ptr(tgt_guide, torch.uint8, "tgt_guide"),
                               _ptr(src_style, torch.uint8, "src_style"), H, W, ctypes.byref(params),
                               _ptr(init_nnf, torch.int32, "init_nnf"),
                               _ptr(nnf_out, torch.int32, "nnf_out"), _ptr(err_out, torch.int32, "err_out"),
                               _ptr(shat_out, torch.uint8, "shat_out"), _stream_handle(stream, ctx.device))
    ctx.check(rc)
    return nnf_out, err_out, shat_out


def fb_nnf_segment(ctx: Context, guides: torch.Tensor, key_styles: torch.Tensor, params: Params,
                   init: Optional[torch.Tensor] = None, with_err: bool = True, stream=None):
    """Fields of a clip segment (key l, n frames, key r) under params.flags
    (FB_FLAG_ALIGN / FB_FLAG_TRACKING).  Returns (nnf (2n,H,W,2) int32, err (2n,H,W)
    int32 holding uint32 values, or None), the left key's fields first."""
    n2, H, W = int(guides.shape[0]), int(guides.shape[1]), int(guides.shape[2])
    n = n2 - 2
    _shape(guides, (n2, H, W, 3), "guides")
    _shape(key_styles, (2, H, W, 3), "key_styles")
    if init is not None:
        _shape(init, (2 * max(n, 0), H, W, 2), "init")
    dev = guides.device
    nnf_out = torch.empty((2 * max(n, 0), H, W, 2), dtype=torch.int32, device=dev)
    err_out = torch.empty((2 * max(n, 0), H, W), dtype=torch.int32, device=dev) if with_err else None
    rc = lib().fb_nnf_segment(ctx.handle, _ptr(guides, torch.uint8, "guides"),
                              _ptr(key_styles, torch.uint8, "key_styles"), n, H, W,
                              ctypes.byref(params), _ptr(init, torch.int32, "init"),
                              _ptr(nnf_out, torch.int32, "nnf_out"),
                              _ptr(err_out, torch.int32, "err_out"), _stream_handle(stream, ctx.device))
    ctx.check(rc)
    return nnf_out, err_out


def fb_remap(ctx: Context, src_style: torch.Tensor, nnf: torch.Tensor, patch: int,
             out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Alg. 2 remap of an H x W x 3 uint8 style through an (H,W,2) int32 NNF."""
    H, W = int(src_style.shape[0]), int(src_style.shape[1])
    _shape(src_style, (H, W, 3), "src_style")
    _shape(nnf, (H, W, 2), "nnf")
    if out is None:
        out = torch.empty((H, W, 3), dtype=torch.float32, device=src_style.device)
    rc = lib().fb_remap(ctx.handle, _ptr(src_style, torch.uint8, "src_style"),
                        _ptr(nnf, torch.int32, "nnf"), H, W, patch,
                        _ptr(out, torch.float32, "out"), _stream_handle(stream, ctx.device))
    ctx.check(rc)
    return out


def fb_blend_window(ctx: Context, guides: torch.Tensor, styles: torch.Tensor, window: int,
                    params: Params, out: Optional[torch.Tensor] = None,
                    stream=None) -> torch.Tensor:
    """Eq. 2 window blend.  guides/styles (N,H,W,3) uint8, both CUDA (async) or both
    CPU (the library stages them; synchronous).  Returns (N,H,W,3) float32."""
    N, H, W = (int(s) for s in guides.shape[:3])
    _shape(guides, (N, H, W, 3), "guides")
    _shape(styles, (N, H, W, 3), "styles")
    if out is None:
        out = torch.empty((N, H, W, 3), dtype=torch.float32, device=guides.device,
                          pin_memory=(not guides.is_cuda))
    rc = lib().fb_blend_window(ctx.handle, _ptr(guides, torch.uint8, "guides"),
                               _ptr(styles, torch.uint8, "styles"), N, H, W, window,
                               ctypes.byref(params), _ptr(out, torch.float32, "out"),
                               _stream_handle(stream, ctx.device))
    ctx.check(rc)
    return out


def fb_blend_window_range(ctx: Context, guides: torch.Tensor, styles: torch.Tensor, window: int,
                          params: Params, n_total: int, frame_base: int, out_first: int, n_out: int,
                          out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Output frames [out_first, out_first + n_out) of the Eq. 2 blend of an n_total-frame
    clip, from its frames [frame_base, frame_base + len(guides)) (CUDA or CPU tensors, as
    fb_blend_window).  Returns (n_out,H,W,3) float32, equal to those frames of the
    whole-clip blend."""
    n_in, H, W = (int(s) for s in guides.shape[:3])
    _shape(guides, (n_in, H, W, 3), "guides")
    _shape(styles, (n_in, H, W, 3), "styles")
    if out is None:
        out = torch.empty((n_out, H, W, 3), dtype=torch.float32, device=guides.device,
                          pin_memory=(not guides.is_cuda))
    _shape(out, (n_out, H, W, 3), "out")
    rc = lib().fb_blend_window_range(ctx.handle, _ptr(guides, torch.uint8, "guides"),
                                     _ptr(styles, torch.uint8, "styles"), n_in, H, W, window,
                                     ctypes.byref(params), n_total, frame_base, out_first, n_out,
                                     _ptr(out, torch.float32, "out"), _stream_handle(stream, ctx.device))
    ctx.check(rc)
    return out


def fb_interpolate(ctx: Context, guides: torch.Tensor, key_idx: Sequence[int],
                   key_styles: torch.Tensor, params: Params, out: Optional[torch.Tensor] = None,
                   stream=None) -> torch.Tensor:
    """Sec. 3.5.2 keyframe interpolation.  guides (N,H,W,3) uint8, key_styles
    (n_keys,H,W,3) uint8, key_idx a host sequence of increasing frame indices."""
    N, H, W = (int(s) for s in guides.shape[:3])
    _shape(guides, (N, H, W, 3), "guides")
    keys = (ctypes.c_int32 * len(key_idx))(*[int(k) for k in key_idx])
    _shape(key_styles, (len(key_idx), H, W, 3), "key_styles")
    if out is None:
        out = torch.empty((N, H, W, 3), dtype=torch.float32, device=guides.device,
                          pin_memory=(not guides.is_cuda))
    rc = lib().fb_interpolate(ctx.handle, _ptr(guides, torch.uint8, "guides"), N, H, W,
                              ctypes.cast(keys, _vp), _ptr(key_styles, torch.uint8, "key_styles"),
                              len(key_idx), ctypes.byref(params), _ptr(out, torch.float32, "out"),
                              _stream_handle(stream, ctx.device))
    ctx.check(rc)
    return out


def fb_interpolate_range(ctx: Context, guides: torch.Tensor, key_idx: Sequence[int],
                         key_styles: torch.Tensor, params: Params, out_first: int, n_out: int,
                         out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Output frames [out_first, out_first + n_out) of fb_interpolate over the whole clip
    (guides: all N frames).  Returns (n_out,H,W,3) float32."""
    N, H, W = (int(s) for s in guides.shape[:3])
    _shape(guides, (N, H, W, 3), "guides")
    keys = (ctypes.c_int32 * len(key_idx))(*[int(k) for k in key_idx])
    _shape(key_styles, (len(key_idx), H, W, 3), "key_styles")
    if out is None:
        out = torch.empty((n_out, H, W, 3), dtype=torch.float32, device=guides.device,
                          pin_memory=(not guides.is_cuda))
    _shape(out, (n_out, H, W, 3), "out")
    rc = lib().fb_interpolate_range(ctx.handle, _ptr(guides, torch.uint8, "guides"), N, H, W,
                                    ctypes.cast(keys, _vp), _ptr(key_styles, torch.uint8, "key_styles"),
                                    len(key_idx), ctypes.byref(params), out_first, n_out,
                                    _ptr(out, torch.float32, "out"), _stream_handle(stream, ctx.device))
    ctx.check(rc)
    return out


def fb_blend_batch(ctx: Context, clips, params: Params, flags: int = 0, stream=None):
    """Eq. 2 blends of several clips in one submission.  `clips` is a sequence of
    (guides, styles, window, patch[, out]) with (N,H,W,3) uint8 CUDA tensors; returns
    the list of (N,H,W,3) float32 outputs (bit-identical to fb_blend_window per clip)."""
    descs = (ClipDesc * len(clips))()
    outs, keep = [], []
    for i, c in enumerate(clips):
        g, s, window, patch = c[0], c[1], int(c[2]), int(c[3])
        N, H, W = (int(v) for v in g.shape[:3])
        _shape(g, (N, H, W, 3), "guides")
        _shape(s, (N, H, W, 3), "styles")
        out = c[4] if len(c) > 4 and c[4] is not None else torch.empty(
            (N, H, W, 3), dtype=torch.float32, device=g.device)
        descs[i] = ClipDesc(_ptr(g, torch.uint8, "guides"), _ptr(s, torch.uint8, "styles"),
                            _ptr(out, torch.float32, "out"), N, H, W, window, patch, 0)
        outs.append(out)
        keep += [g, s]
    rc = lib().fb_blend_batch(ctx.handle, descs, len(clips), ctypes.byref(params), flags,
                              _stream_handle(stream, ctx.device))
    ctx.check(rc)
    return outs


def fb_batch_plan(shapes, params: Params, budget_bytes: int = 0):
    """Host-only plan of a batch given (N, H, W, window, patch) tuples:
    (number of NNFs, work items of 32x8 tiles per iteration, chunks)."""
    descs = (ClipDesc * len(shapes))()
    for i, (N, H, W, window, patch) in enumerate(shapes):
        descs[i] = ClipDesc(None, None, None, N, H, W, window, patch, 0)
    n_pairs, n_items, n_chunks = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int()
    rc = lib().fb_batch_plan(descs, len(shapes), ctypes.byref(params), budget_bytes,
                             ctypes.byref(n_pairs), ctypes.byref(n_items), ctypes.byref(n_chunks))
    if rc != FB_OK:
        raise FastBlendError(rc, lib().fb_last_error(None).decode())
    return n_pairs.value, n_items.value, n_chunks.value


def fb_ctx_batch_variant(ctx: Context, patch: int) -> int:
    return int(lib().fb_ctx_batch_variant(ctx.handle, patch))


FB_BATCH_PERSISTENT = 1 << 24
FB_BATCH_PER_CLIP = 2 << 24


def fb_ctx_batch_mode(ctx: Context, patch: int) -> int:
    """Launch mode the batch autotuner chose for patch size k: 0 persistent, 1 per-clip, -1 none."""
    return int(lib().fb_ctx_batch_mode(ctx.handle, patch))


def fb_ctx_batch_claim(ctx: Context, patch: int) -> int:
    """Tiles per iteration claim the batch autotuner chose for patch size k (-1: none)."""
    return int(lib().fb_ctx_batch_claim(ctx.handle, patch))


BATCH_VARIANT_NAMES = ("tile 32x8, 5 blocks/SM", "tile 32x4, 10 blocks/SM",
                       "tile 32x16, 2 blocks/SM", "tile 32x8, 4 blocks/SM")


def batch_variant_name(v: int) -> str:
    return BATCH_VARIANT_NAMES[v] if 0 <= v < len(BATCH_VARIANT_NAMES) else "untuned"


# ----------------------------------------------------------------------------------
# Learned NNF initialiser
# ----------------------------------------------------------------------------------
class InitNet:
    """fb_initnet: the BF16 conv pyramid that proposes initial NNFs (tensor-core kernels)."""

    def __init__(self, ctx: Context, max_pairs: int, H: int, W: int, downscale: int = 8):
        h = _vp()
        rc = lib().fb_initnet_create(ctx.handle, ctypes.byref(h), max_pairs, H, W, downscale)
        if rc != FB_OK:
            raise FastBlendError(rc, "fb_initnet_create")
        self._h, self.ctx, self.max_pairs, self.H, self.W = h, ctx, max_pairs, H, W
        self.ds = downscale
        self.n_params = int(lib().fb_initnet_param_count(h))

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().fb_initnet_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int) -> None:
        if rc != FB_OK:
            raise FastBlendError(rc, lib().fb_initnet_last_error(self._h).decode())

    def get_params(self):
        import numpy as np
        out = np.zeros(self.n_params, np.float32)
        self._check(lib().fb_initnet_get_params(self._h, out.ctypes.data))
        return out

    def set_params(self, p) -> None:
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        self._check(lib().fb_initnet_set_params(self._h, p.ctypes.data))

    def get_grads(self):
        import numpy as np
        out = np.zeros(self.n_params, np.float32)
        self._check(lib().fb_initnet_get_grads(self._h, out.ctypes.data))
        return out

    def get_optimizer(self):
        """(first moments, second moments, updates taken) of the Adam state."""
        import numpy as np
        m = np.zeros(self.n_params, np.float32)
        v = np.zeros(self.n_params, np.float32)
        step = ctypes.c_uint64()
        self._check(lib().fb_initnet_get_optimizer(self._h, m.ctypes.data, v.ctypes.data, ctypes.byref(step)))
        return m, v, int(step.value)

    def set_optimizer(self, m, v, step: int) -> None:
        import numpy as np
        m = np.ascontiguousarray(m, np.float32)
        v = np.ascontiguousarray(v, np.float32)
        if m.size != self.n_params or v.size != self.n_params:
            raise ValueError("optimizer state must have n_params entries")
        self._check(lib().fb_initnet_set_optimizer(self._h, m.ctypes.data, v.ctypes.data, int(step)))

    def forward(self, src: torch.Tensor, tgt: torch.Tensor, stream=None) -> torch.Tensor:
        n = int(src.shape[0])
        head = torch.empty((n, self.H // self.ds, self.W // self.ds, 8), dtype=torch.float32,
                           device=src.device)
        self._check(lib().fb_initnet_forward(self._h, _ptr(src, torch.uint8, "src"),
                                             _ptr(tgt, torch.uint8, "tgt"), n,
                                             _ptr(head, torch.float32, "head"),
                                             _stream_handle(stream, self.ctx.device)))
        return head

    def init_nnf(self, n: int, stream=None) -> torch.Tensor:
        out = torch.empty((n, self.H, self.W, 2), dtype=torch.int32, device="cuda")
        self._check(lib().fb_initnet_init_nnf(self._h, n, out.data_ptr(),
                                              _stream_handle(stream, self.ctx.device)))
        return out

    def train_step(self, src, tgt, target, weight=None, weight_sum=None, lr=1e-3,
                   loss_out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        n = int(src.shape[0])
        if loss_out is None:
            loss_out = torch.zeros(1, dtype=torch.float32, device=src.device)
        if weight_sum is None:
            weight_sum = float(weight.sum()) if weight is not None else float(
                n * (self.H // self.ds) * (self.W // self.ds))
        self._check(lib().fb_initnet_train_step(
            self._h, _ptr(src, torch.uint8, "src"), _ptr(tgt, torch.uint8, "tgt"), n,
            _ptr(target, torch.float32, "target"),
            _ptr(weight, torch.float32, "weight") if weight is not None else None,
            float(weight_sum), float(lr), _ptr(loss_out, torch.float32, "loss"),
            _stream_handle(stream, self.ctx.device)))
        return loss_out

    def status(self) -> int:
        return int(lib().fb_initnet_status(self._h))


def fb_initnet_targets(nnf: torch.Tensor, downscale: int = 8, stream=None):
    """Targets (n,H/D,W/D,2) and weights (n,H/D,W/D) from Alg. 1 fields (n,H,W,2) int32."""
    n, H, W = (int(v) for v in nnf.shape[:3])
    D = downscale
    target = torch.empty((n, H // D, W // D, 2), dtype=torch.float32, device=nnf.device)
    weight = torch.empty((n, H // D, W // D), dtype=torch.float32, device=nnf.device)
    rc = lib().fb_initnet_targets(_ptr(nnf, torch.int32, "nnf"), n, H, W, D, target.data_ptr(),
                                  weight.data_ptr(), _stream_handle(stream, nnf.device.index or 0))
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_initnet_targets")
    return target, weight


def conv3x3_forward(x: torch.Tensor, w: torch.Tensor, bias: torch.Tensor, stride: int, relu: bool,
                    out_f32: bool = False, status: Optional[torch.Tensor] = None):
    """One 3x3 conv layer on the tensor cores (bf16 NHWC x, bf16 [Cout,3,3,Cin] w)."""
    n, H, W, Cin = (int(v) for v in x.shape)
    Cout = int(w.shape[0])
    Ho, Wo = (H + stride - 1) // stride, (W + stride - 1) // stride
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=x.device)
    y = torch.empty((n, Ho, Wo, Cout), dtype=torch.float32 if out_f32 else torch.bfloat16,
                    device=x.device)
    rc = lib().fb_conv3x3_forward(_ptr(x, torch.bfloat16, "x"), n, H, W, Cin,
                                  _ptr(w, torch.bfloat16, "w"), _ptr(bias, torch.float32, "bias"),
                                  Cout, stride, int(relu),
                                  None if out_f32 else y.data_ptr(), y.data_ptr() if out_f32 else None,
                                  status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_conv3x3_forward")
    return y, status


def conv3x3_backward(x: torch.Tensor, wt: Optional[torch.Tensor], dz: torch.Tensor, stride: int,
                     status: Optional[torch.Tensor] = None, input_grad: bool = True,
                     weight_grad: bool = True):
    """(dx f32 or None, dw f32 or None) of one conv layer; wt = weights transposed to
    [Cin,3,3,Cout] bf16 (needed for dx only); input_grad / weight_grad select the two."""
    n, H, W, Cin = (int(v) for v in x.shape)
    Cout = int(dz.shape[-1])
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=x.device)
    dx = torch.empty((n, H, W, Cin), dtype=torch.float32, device=x.device) if input_grad else None
    dw = torch.zeros((Cout, 3, 3, Cin), dtype=torch.float32, device=x.device) if weight_grad else None
    rc = lib().fb_conv3x3_backward(_ptr(x, torch.bfloat16, "x"), n, H, W, Cin,
                                   _ptr(wt, torch.bfloat16, "wt") if input_grad else None, Cout, stride,
                                   _ptr(dz, torch.bfloat16, "dz"), dx.data_ptr() if input_grad else None,
                                   dw.data_ptr() if weight_grad else None, status.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    if rc != FB_OK:
        raise FastBlendError(rc, "fb_conv3x3_backward")
    return dx, dw, status
