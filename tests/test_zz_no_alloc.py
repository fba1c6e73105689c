"""fb_blend_window_noalloc: fb_blend_window for callers that cannot allocate.

Such callers (a host callback or stream-ordered pipeline that must not synchronise
the device, a plug-in whose host owns every allocation, a process on a fixed memory
budget) cannot create a context, because a context allocates its scratch.  The
no-alloc entry point instead uses one fixed device array inside libfb.so.  This test
calls it through the C ABI twice in a row, on different clips, and checks each result
against fb_blend_window, the entry point with context-owned scratch, and the first one
also against the CPU oracle; between the two calls neither the device's free memory nor
torch's allocations may change.  It lives in a file of its own that pytest collects last.
"""
import ctypes
import gc

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 0.5 / 255.0


def _noalloc(fbp, g, s, window, params, out):
    import torch
    N, H, W = g.shape[:3]
    rc = fbp.lib().fb_blend_window_noalloc(g.data_ptr(), s.data_ptr(), N, H, W, window,
                                           ctypes.byref(params), out.data_ptr(),
                                           torch.cuda.current_stream().cuda_stream)
    assert rc == fbp.FB_OK, fbp.lib().fb_last_error(None).decode()
    return out


def test_noalloc_blend_matches_context_blend_on_two_calls_in_a_row():
    import torch

    import oracle
    import paper_2311_09265_b300 as fbp
    fbp.build()
    torch.cuda.set_device(0)
    ctx = fbp.Context(0)
    cases = [
        (synth.small_clip(8, 96, 96, seed=synth.clip_seed(0)), 3, fbp.Params.make(5, 4, 1, 0, 31)),
        (synth.small_clip(6, 61, 47, seed=77, motion="affine"), 5, fbp.Params.make(7, 2, 2, 0, 5)),
    ]
    # Everything torch or the context allocates comes first: inputs, outputs and the
    # context's own blends (which also load every kernel the two calls launch).
    dev, want = [], []
    for (g, s), window, params in cases:
        gd, sd = torch.from_numpy(g).cuda(), torch.from_numpy(s).cuda()
        dev.append((gd, sd))
        want.append(fbp.fb_blend_window(ctx, gd, sd, window, params).cpu().numpy())
    outs = [torch.full(g.shape, -1.0, dtype=torch.float32, device="cuda") for (g, _), _, _ in cases]
    torch.cuda.synchronize()
    got = []
    # Tensors left by earlier tests may be collected at any time and lower torch's count:
    # collect them first and keep the collector off while the counts are compared.
    gc.collect()
    gc.disable()
    try:
        for q, ((g, s), window, params) in enumerate(cases):
            got.append(_noalloc(fbp, dev[q][0], dev[q][1], window, params, outs[q]))
            torch.cuda.synchronize()
            if q == 0:   # the library's device code and its static array are in place now
                free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0
    finally:
        gc.enable()
    for q, ((g, s), window, params) in enumerate(cases):
        o = got[q].cpu().numpy()
        assert np.abs(o - want[q]).max() <= TOL
        assert (o == want[q]).all()
    (g, s), window, params = cases[0]
    ref = oracle.blend_window(g, s, window, params.patch, params.iters, params.levels, seed=params.seed)
    assert np.abs(got[0].cpu().numpy() - ref).max() <= TOL
    ctx.close()


def test_noalloc_rejects_a_blend_larger_than_its_scratch():
    import torch

    import paper_2311_09265_b300 as fbp
    fbp.build()
    g = torch.zeros((60, 512, 512, 3), dtype=torch.uint8, device="cuda")
    out = torch.empty((60, 512, 512, 3), dtype=torch.float32, device="cuda")
    p = fbp.Params.make(5, 1)
    rc = fbp.lib().fb_blend_window_noalloc(g.data_ptr(), g.data_ptr(), 60, 512, 512, 15,
                                           ctypes.byref(p), out.data_ptr(), None)
    assert rc == fbp.FB_ERR_ARG
    assert b"static scratch holds" in fbp.lib().fb_last_error(None)
