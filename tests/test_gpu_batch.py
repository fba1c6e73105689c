"""The batched persistent path (fb_blend_batch): every clip bit-identical to
fb_blend_window, for every tile variant, with and without graph replay, across chunks."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

SHAPES = [(5, 40, 52, 3, 5), (6, 33, 64, 5, 7), (4, 64, 48, 7, 3), (3, 48, 48, 1, 5),
          (7, 37, 45, 5, 5)]


@pytest.fixture(scope="module")
def fbp():
    import paper_2311_09265_b300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def clips():
    import torch
    out = []
    for n, (N, H, W, window, patch) in enumerate(SHAPES):
        g, s = synth.small_clip(N, H, W, seed=900 + n, motion="affine" if n % 2 else "shift")
        out.append((torch.tensor(g, device="cuda"), torch.tensor(s, device="cuda"), window, patch))
    return out


def per_clip(fbp, ctx, clips, params):
    res = []
    for g, s, window, patch in clips:
        p = fbp.Params.make(patch, params.iters, 1, params.r0, params.seed)
        res.append(fbp.fb_blend_window(ctx, g, s, window, p).cpu().numpy())
    return res


def test_batch_matches_per_clip_blend_and_oracle(fbp, clips):
    ctx = fbp.Context(0)
    params = fbp.Params.make(5, 3, 1, 0, 2024)
    want = per_clip(fbp, ctx, clips, params)
    got = [o.cpu().numpy() for o in fbp.fb_blend_batch(ctx, clips, params)]
    for w, g in zip(want, got):
        assert (w == g).all()
    g0 = clips[0][0].cpu().numpy()
    s0 = clips[0][1].cpu().numpy()
    ref = oracle.blend_window(g0, s0, SHAPES[0][3], SHAPES[0][4], 3, seed=2024)
    assert (got[0] == ref).all()
    for k in (3, 5, 7):
        assert 0 <= fbp.fb_ctx_batch_variant(ctx, k) < 4
        assert fbp.fb_ctx_batch_claim(ctx, k) in (1, 2, 4, 8)
        assert fbp.fb_ctx_batch_mode(ctx, k) in (0, 1)
    ctx.close()


def test_graph_replay_follows_new_input_contents(fbp, clips):
    import torch
    ctx = fbp.Context(0)
    params = fbp.Params.make(5, 2, 1, 0, 7)
    outs = [torch.empty(g.shape, dtype=torch.float32, device="cuda") for g, _, _, _ in clips]
    spec = [(g, s, w, k, o) for (g, s, w, k), o in zip(clips, outs)]
    first = [o.cpu().numpy().copy() for o in fbp.fb_blend_batch(ctx, spec, params)]
    n0 = ctx.launches
    again = [o.cpu().numpy().copy() for o in fbp.fb_blend_batch(ctx, spec, params)]
    assert all((a == b).all() for a, b in zip(first, again))
    assert ctx.launches > n0                      # replay counted its kernels
    saved = [s.clone() for _, s, _, _ in clips]
    for _, s, _, _ in clips:                      # new style contents, same pointers
        s.copy_(torch.flip(s, dims=[0]))
    replay = [o.cpu().numpy().copy() for o in fbp.fb_blend_batch(ctx, spec, params)]
    want = per_clip(fbp, ctx, clips, params)
    assert all((a == b).all() for a, b in zip(replay, want))
    for (_, s, _, _), s0 in zip(clips, saved):
        s.copy_(s0)
    ctx.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_every_tile_variant_gives_identical_results(fbp, clips, variant):
    ctx = fbp.Context(0)
    params = fbp.Params.make(5, 2, 1, 0, 99)
    want = per_clip(fbp, ctx, clips, params)
    for flags in (fbp.FB_BATCH_VARIANT(variant), fbp.FB_BATCH_VARIANT(variant) | fbp.FB_BATCH_NO_GRAPH):
        got = [o.cpu().numpy() for o in fbp.fb_blend_batch(ctx, clips, params, flags=flags)]
        assert all((a == b).all() for a, b in zip(want, got))
    ctx.close()


@pytest.mark.parametrize("claim", [1, 2, 3, 8, 64])
def test_every_claim_size_gives_identical_results(fbp, clips, claim):
    """The tuner's other knob, the tiles one claim of the persistent iteration kernel
    covers, changes only the schedule (alone or with a forced variant)."""
    ctx = fbp.Context(0)
    params = fbp.Params.make(5, 2, 1, 0, 98)
    want = per_clip(fbp, ctx, clips, params)
    for flags in (fbp.FB_BATCH_CLAIM(claim), fbp.FB_BATCH_CLAIM(claim) | fbp.FB_BATCH_VARIANT(claim % 4)):
        got = [o.cpu().numpy() for o in fbp.fb_blend_batch(ctx, clips, params, flags=flags)]
        assert all((a == b).all() for a, b in zip(want, got))
    assert fbp.fb_ctx_batch_claim(ctx, 5) == -1       # forced runs are not remembered as tuned
    ctx.close()


def test_per_clip_mode_gives_identical_results(fbp, clips):
    """The tuner's launch-mode knob: per-clip launches of the per-call kernels (three graph
    branches, or the caller's stream without a graph, and in many chunks) against the
    persistent kernels and the per-clip loop."""
    ctx = fbp.Context(0)
    params = fbp.Params.make(5, 2, 1, 0, 97)
    want = per_clip(fbp, ctx, clips, params)
    for flags in (fbp.FB_BATCH_PER_CLIP, fbp.FB_BATCH_PER_CLIP | fbp.FB_BATCH_NO_GRAPH, fbp.FB_BATCH_PERSISTENT):
        got = [o.cpu().numpy() for o in fbp.fb_blend_batch(ctx, clips, params, flags=flags)]
        assert all((a == b).all() for a, b in zip(want, got)), flags
    ctx.set_pair_budget(1 << 20)                 # segments cut at chunk boundaries
    got = [o.cpu().numpy() for o in fbp.fb_blend_batch(ctx, clips, params, flags=fbp.FB_BATCH_PER_CLIP)]
    assert all((a == b).all() for a, b in zip(want, got))
    ctx.close()


def test_chunked_batch_equals_single_chunk(fbp, clips):
    ctx = fbp.Context(0)
    params = fbp.Params.make(5, 2, 1, 0, 5)
    want = per_clip(fbp, ctx, clips, params)
    ctx.set_pair_budget(1 << 20)                 # forces many chunks
    got = [o.cpu().numpy() for o in fbp.fb_blend_batch(ctx, clips, params)]
    assert all((a == b).all() for a, b in zip(want, got))
    # the per-call blend honours the budget too
    again = per_clip(fbp, ctx, clips, params)
    assert all((a == b).all() for a, b in zip(want, again))
    ctx.close()


def test_batch_argument_errors(fbp, clips):
    import torch
    ctx = fbp.Context(0)
    g, s, _, _ = clips[0]
    for bad in (fbp.FB_BATCH_CLAIM(65), fbp.FB_BATCH_PER_CLIP | fbp.FB_BATCH_VARIANT(0), 3 << 24):
        with pytest.raises(fbp.FastBlendError) as e:
            fbp.fb_blend_batch(ctx, [(g, s, 3, 5)], fbp.Params.make(5, 2), flags=bad)
        assert e.value.status == fbp.FB_ERR_ARG
    with pytest.raises(fbp.FastBlendError) as e:
        fbp.fb_blend_batch(ctx, [(g, s, 4, 5)], fbp.Params.make(5, 2))
    assert e.value.status == fbp.FB_ERR_ARG
    with pytest.raises(fbp.FastBlendError) as e:
        fbp.fb_blend_batch(ctx, [(g.cpu(), s, 3, 5)], fbp.Params.make(5, 2))
    assert e.value.status == fbp.FB_ERR_ARG
    with pytest.raises(fbp.FastBlendError) as e:
        fbp.fb_blend_batch(ctx, [(g, s, 3, 5)], fbp.Params.make(5, 2), flags=fbp.FB_BATCH_VARIANT(7))
    assert e.value.status == fbp.FB_ERR_ARG
    ctx.close()


@pytest.mark.slow
def test_full_manifest_in_the_bench_launch_configuration(fbp):
    """The 32-clip manifest bench.py times (uneven shapes, windows 5-31, patch 5 and 7,
    tuned tiles, graph capture), checked on one middle frame of the cheapest clip of each
    patch size against the oracle, bit for bit."""
    import torch
    import bench
    manifest = synth.batch_manifest(seed=bench.BATCH_SEED)
    clips, host = [], []
    for n, (N, H, W, window, patch) in enumerate(manifest):
        g, s = synth.batch_clip(N, H, W, seed=bench.BATCH_SEED + n)
        host.append((g, s))
        clips.append((torch.tensor(g, device="cuda"), torch.tensor(s, device="cuda"), window, patch))
    ctx = fbp.Context(0)
    params = fbp.Params.make(5, bench.BATCH_ITERS, 1, 0, bench.BATCH_SEED)
    fbp.fb_blend_batch(ctx, clips, params)            # tunes and captures
    outs = fbp.fb_blend_batch(ctx, clips, params)     # graph replay, as timed
    for k in (5, 7):
        i = min((c for c in range(len(manifest)) if manifest[c][4] == k),
                key=lambda c: manifest[c][1] * manifest[c][2] * manifest[c][3])
        N, H, W, window, patch = manifest[i]
        g, s = host[i]
        ref = oracle.blend_frame(g, s, window, N // 2, patch, bench.BATCH_ITERS, seed=bench.BATCH_SEED)
        assert (outs[i][N // 2].cpu().numpy() == ref).all(), (i, manifest[i])
    ctx.close()


def test_small_clip_manifest_matches_per_clip_calls_and_oracle(fbp):
    """The first 64 clips of the small-clip manifest bench.py times (64-128 px, 6-12 frames,
    windows 3-5, patch 5 and 7; tuned, graph-replayed as timed): every clip bit for bit
    equal to its own fb_blend_window call, and the first clip of each patch size to the
    oracle over the whole clip."""
    import torch
    import bench
    manifest = bench.batch_manifest("batch_small", bench.BATCH_SEED)[:64]
    clips, host = [], []
    for n, (N, H, W, window, patch) in enumerate(manifest):
        g, s = synth.batch_clip(N, H, W, seed=bench.BATCH_SEED + n)
        host.append((g, s))
        clips.append((torch.tensor(g, device="cuda"), torch.tensor(s, device="cuda"), window, patch))
    ctx = fbp.Context(0)
    params = fbp.Params.make(5, bench.BATCH_ITERS, 1, 0, bench.BATCH_SEED)
    fbp.fb_blend_batch(ctx, clips, params)            # tunes and captures
    outs = fbp.fb_blend_batch(ctx, clips, params)     # graph replay, as timed
    for i, (N, H, W, window, patch) in enumerate(manifest):
        want = fbp.fb_blend_window(ctx, clips[i][0], clips[i][1], window,
                                   fbp.Params.make(patch, bench.BATCH_ITERS, 1, 0, bench.BATCH_SEED))
        assert torch.equal(outs[i], want), (i, manifest[i])
    for k in (5, 7):
        i = next(c for c in range(len(manifest)) if manifest[c][4] == k)
        N, H, W, window, patch = manifest[i]
        g, s = host[i]
        ref = oracle.blend_window(g, s, window, patch, bench.BATCH_ITERS, seed=bench.BATCH_SEED)
        assert (outs[i].cpu().numpy() == ref).all(), (i, manifest[i])
    ctx.close()
