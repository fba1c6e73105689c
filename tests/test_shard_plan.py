"""Splitting one clip across GPUs by output frame (host only, no GPU).

Eq. 2 (Sec. 3.4) makes output frame i depend only on the frames of its window
[i - M, i + M], and an interpolated frame only on its keys (Sec. 3.5.2).  So a clip shards
into contiguous ranges of output frames, each computed from its own frames plus an
M-frame halo on either side, with no exchange between the shards.  These tests check
the host side of that split against the definitions: the shards cover every output frame
once, carry about equal work, and each shard's input range holds every frame its NNFs
read; the NNFs of the range calls are exactly those of the whole-clip call, with the same
random streams.  The last test runs the planner as two gloo ranks (world size 2).
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def fbp():
    import paper_2311_09265_b300 as m
    m.build()
    return m


def _key(p):
    return (p["src"], p["tgt"], p["tag"], p["weight"], p["out_frame"])


def _work(N, window, i):
    if window == 0:
        return 1
    M = (window - 1) // 2
    return min(N - 1, i + M) - max(0, i - M) + 1


@pytest.mark.parametrize("N,window,n_shards", [
    (60, 15, 1), (60, 15, 2), (60, 15, 8), (16, 15, 3), (9, 3, 9), (100, 31, 7), (5, 1, 2),
    (48, 0, 4), (1, 1, 1)])
def test_shards_cover_the_clip_once_with_their_halo(fbp, N, window, n_shards):
    M = (window - 1) // 2 if window else 0
    plans = [fbp.fb_shard_plan(N, window, n_shards, s) for s in range(n_shards)]
    nxt = 0
    for s, pl in enumerate(plans):
        a, n = pl["out_first"], pl["n_out"]
        assert a == nxt and n >= 1, (s, pl)
        nxt = a + n
        if window:
            assert pl["frame_base"] == max(0, a - M)
            assert pl["frame_base"] + pl["n_in"] == min(N, a + n + M)
        else:
            assert (pl["frame_base"], pl["n_in"]) == (0, N)
    assert nxt == N
    # about equal work: no shard exceeds the ideal share by more than its largest frame
    total = sum(_work(N, window, i) for i in range(N))
    biggest = max(_work(N, window, i) for i in range(N))
    for pl in plans:
        w = sum(_work(N, window, i) for i in range(pl["out_first"], pl["out_first"] + pl["n_out"]))
        assert w <= total / n_shards + biggest, (pl, w, total)


@pytest.mark.parametrize("N,window,n_shards", [(60, 15, 2), (60, 15, 8), (16, 15, 3), (23, 5, 4),
                                               (7, 31, 3)])
def test_range_pairs_are_the_whole_clip_pairs(fbp, N, window, n_shards):
    whole = fbp.fb_pair_plan(N, window)
    got = []
    for s in range(n_shards):
        pl = fbp.fb_shard_plan(N, window, n_shards, s)
        lo, hi = pl["frame_base"], pl["frame_base"] + pl["n_in"]
        pr = fbp.fb_pair_plan_range(N, pl["out_first"], pl["n_out"], window=window)
        for p in pr:
            # every frame an NNF of the shard reads is inside the shard's input range
            assert lo <= p["src"] < hi and lo <= p["tgt"] < hi, (s, p, pl)
            assert pl["out_first"] <= p["out_frame"] < pl["out_first"] + pl["n_out"]
            assert p["tag"] == fbp.fb_pair_tag(p["src"], p["tgt"])
        got += [_key(p) for p in pr]
    # same NNFs, same streams, same order once the shards are concatenated
    assert got == [_key(p) for p in whole]


@pytest.mark.parametrize("keys,flags", [([0, 47], 0), ([0, 47], 0x40), ([5, 20, 33], 0x40), ([10], 0)])
def test_interpolation_ranges_are_the_whole_clip_pairs(fbp, keys, flags):
    N = 48
    whole = fbp.fb_pair_plan(N, 0, keys, flags)
    got = []
    for s in range(5):
        pl = fbp.fb_shard_plan(N, 0, 5, s)
        pr = fbp.fb_pair_plan_range(N, pl["out_first"], pl["n_out"], keys=keys, flags=flags)
        for q, p in enumerate(pr):
            if p["partner"] >= 0:  # the partner is the other key's NNF to the same frame
                o = pr[p["partner"]]
                assert o["tgt"] == p["tgt"] and o["src"] != p["src"] and o["partner"] == q
        got += [_key(p) for p in pr]
    assert got == [_key(p) for p in whole]


def test_planner_rejects_bad_requests(fbp):
    import paper_2311_09265_b300 as m
    for args in [(0, 3, 1, 0), (10, 4, 1, 0), (10, 3, 11, 0), (10, 3, 2, 2), (10, 3, 0, 0), (10, -1, 1, 0)]:
        with pytest.raises(m.FastBlendError):
            fbp.fb_shard_plan(*args)
    with pytest.raises(m.FastBlendError):
        fbp.fb_pair_plan_range(10, 8, 3, window=3)          # range past the clip end
    with pytest.raises(m.FastBlendError):
        fbp.fb_pair_plan_range(10, 0, 3, window=3, flags=0x20)  # tracking has no range form


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import json

    import torch.distributed as dist

    import paper_2311_09265_b300 as m
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N, window = 60, 15
    pl = m.fb_shard_plan(N, window, world, rank)
    mine = [_key(p) for p in m.fb_pair_plan_range(N, pl["out_first"], pl["n_out"], window=window)]
    lo, hi = pl["frame_base"], pl["frame_base"] + pl["n_in"]
    inside = all(lo <= k[0] < hi and lo <= k[1] < hi for k in mine)
    gathered = [None] * world
    dist.all_gather_object(gathered, {"plan": pl, "pairs": mine, "inside": inside})
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(gathered, f)


def test_two_gloo_ranks_split_one_clip(tmp_path, fbp):
    """Each rank plans its own shard; after an all-gather every rank holds the same view:
    the union of the shards' NNFs is the whole clip's list, and every shard's NNFs read only
    frames of its own input range (the halo included)."""
    import json
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    views = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert views[0] == views[1]
    whole = [list(_key(p)) for p in fbp.fb_pair_plan(60, 15)]
    union = [k for v in views[0] for k in v["pairs"]]
    assert union == whole
    assert all(v["inside"] for v in views[0])
    p0, p1 = views[0][0]["plan"], views[0][1]["plan"]
    assert p0["out_first"] == 0 and p0["out_first"] + p0["n_out"] == p1["out_first"]
    # the halo: rank 0's inputs reach 7 frames past its last output frame, rank 1's 7 before
    assert p0["frame_base"] + p0["n_in"] == p1["out_first"] + 7
    assert p1["frame_base"] == p1["out_first"] - 7
