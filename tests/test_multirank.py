"""The N > 1 bench path on CPU: two gloo ranks (world size 2, 127.0.0.1).

The hot path shards by output frame of one clip (each rank blends its range from its
frames plus the window's halo) or by clip (replicas); neither exchanges data, so what runs
across ranks is the bench's own plumbing: the barriers around the timed region, the
max-over-ranks timing, the whole-job aggregate, per-rank inputs (the same clip wherever it
is cut), and the reference arm that only rank 0 runs.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    grp = bench.RankGroup()
    assert (grp.rank, grp.world) == (rank, world)
    grp.barrier()
    slowest = grp.max(10.0 + 5.0 * rank)           # this rank's "timed region"
    w = synth.WORKLOADS["blend_tiny"]
    g, s = bench.make_inputs(w, bench.shard_seed(w.seed, rank))
    grp.barrier()
    grp.close()
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), slowest=slowest, g=g, s=s)


def test_two_gloo_ranks_share_timing_and_shard_inputs(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    # every rank sees the slowest rank's time
    assert [float(x["slowest"]) for x in r] == [15.0, 15.0]
    # rank 0 blends the named workload itself; rank 1 blends a different clip of the same shape
    g0, s0 = synth.make_clip("blend_tiny")
    assert np.array_equal(r[0]["g"], g0) and np.array_equal(r[0]["s"], s0)
    assert r[1]["g"].shape == g0.shape and r[1]["s"].shape == s0.shape
    assert not np.array_equal(r[1]["g"], g0)


def test_aggregate_counts_every_rank_over_the_slowest_time():
    # 2 ranks x 60 frames x 5 steps in 3 s of the slowest rank
    assert bench.aggregate(60, 5, 2, 3000.0) == pytest.approx(200.0)
    assert bench.aggregate(60, 5, 1, 3000.0) == pytest.approx(100.0)


def test_shard_seeds_are_distinct_and_rank0_is_the_workload():
    seeds = [bench.shard_seed(1234, r) for r in range(8)]
    assert seeds[0] == 1234 and len(set(seeds)) == 8


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_one_line():
    """bench.py --impl reference launched as two ranks: rank 0 alone runs the oracle and
    prints one JSON line, the other rank exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--workload", "blend_tiny", "--steps", "1", "--warmup", "0"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_window_override_keeps_the_named_clip():
    import dataclasses
    w = synth.WORKLOADS["blend_tiny"]
    g0, s0 = bench.make_inputs(w, w.seed)
    g1, s1 = bench.make_inputs(dataclasses.replace(w, window=5), w.seed)
    assert np.array_equal(g0, g1) and np.array_equal(s0, s1)


def _shard_rank_main(rank, world, port, out_dir):
    import dataclasses
    import json

    import paper_2311_09265_b300 as fbp
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    grp = bench.RankGroup()
    w = dataclasses.replace(synth.WORKLOADS["blend_512"], N=8, H=48, W=64)
    n_total = w.N * world
    pl = fbp.fb_shard_plan(n_total, w.window, world, rank)
    g, s = bench.shard_inputs(w, n_total, pl["frame_base"], pl["frame_base"] + pl["n_in"])
    total_in = grp.sum(g.nbytes + s.nbytes)
    grp.barrier()
    grp.close()
    np.savez(os.path.join(out_dir, f"shard{rank}.npz"), g=g, s=s, total_in=total_in)
    with open(os.path.join(out_dir, f"shard{rank}.json"), "w") as f:
        json.dump(pl, f)


def test_frame_shards_see_one_clip(tmp_path):
    """bench.py --shard frames: two gloo ranks plan their output ranges of one 16-frame
    clip (window 15) and draw only their own input frames, halo included; the frames both
    ranks hold are identical, and every rank's frames are those of the whole clip."""
    import dataclasses
    import json
    world = 2
    mp.start_processes(_shard_rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    pl = [json.load(open(tmp_path / f"shard{r}.json")) for r in range(world)]
    d = [np.load(tmp_path / f"shard{r}.npz") for r in range(world)]
    w = dataclasses.replace(synth.WORKLOADS["blend_512"], N=8, H=48, W=64)
    g_all, s_all = bench.shard_inputs(w, 16, 0, 16)
    for r in range(world):
        a, n = pl[r]["frame_base"], pl[r]["n_in"]
        assert np.array_equal(d[r]["g"], g_all[a:a + n]) and np.array_equal(d[r]["s"], s_all[a:a + n])
    assert pl[0]["out_first"] + pl[0]["n_out"] == pl[1]["out_first"]
    assert float(d[0]["total_in"]) == d[0]["g"].nbytes + d[0]["s"].nbytes + d[1]["g"].nbytes + d[1]["s"].nbytes
