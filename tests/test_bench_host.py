"""Host-side bookkeeping of bench.py that needs no GPU."""
import dataclasses
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def _pairs(N, keys):
    """Sec. 3.5.2 pair set by brute force: each non-key frame from its nearest key on
    either side."""
    out = set()
    for i in range(N):
        if i in keys:
            continue
        left = [k for k in keys if k < i]
        right = [k for k in keys if k > i]
        if left:
            out.add((max(left), i))
        if right:
            out.add((min(right), i))
    return out


@pytest.mark.parametrize("N,keys", [(48, (0, 47)), (10, (2, 5, 7)), (6, (3,)), (5, (0, 1, 2, 3, 4)),
                                    (9, (0, 2, 4, 6, 8)), (7, (6,))])
def test_tracking_neighbour_refs_count_chain_neighbours(N, keys):
    w = dataclasses.replace(synth.WORKLOADS["interp_1024x576"], N=N, keys=keys)
    pairs = _pairs(N, set(keys))
    brute = sum(((src, tgt - 1) in pairs) + ((src, tgt + 1) in pairs) for src, tgt in pairs)
    assert bench.tracking_neighbour_refs(w) == brute
    assert len(pairs) == w.pairs()


@pytest.mark.parametrize("N,window", [(60, 15), (5, 15), (9, 3), (7, 5), (1, 7)])
def test_tracking_neighbour_refs_of_a_blend(N, window):
    w = dataclasses.replace(synth.WORKLOADS["blend_512"], N=N, window=window)
    M = window // 2
    pairs = {(j, i) for i in range(N) for j in range(max(0, i - M), min(N - 1, i + M) + 1) if j != i}
    brute = sum(((src, tgt - 1) in pairs) + ((src, tgt + 1) in pairs) for src, tgt in pairs)
    assert bench.tracking_neighbour_refs(w) == brute
    assert len(pairs) == w.pairs()


def test_mode_workloads_run_on_their_clip():
    assert bench.base_workload("tracking_1024x576") == "interp_1024x576"
    assert bench.base_workload("aligned_1024x576") == "interp_1024x576"
    for m in ("balanced_512", "fast_512", "accurate_512", "learned_512", "initnet_512", "tracking_512"):
        assert bench.base_workload(m) == "blend_512"
    assert bench.base_workload("blend_512_16f") == "blend_512_16f"


@pytest.mark.parametrize("N,keys,expect", [(48, (0, 47), 92), (10, (2, 5, 7), 6), (6, (3,), 0),
                                           (5, (0, 1, 2, 3, 4), 0), (9, (0, 4, 8), 12)])
def test_aligned_pairs_are_the_pairs_between_keys(N, keys, expect):
    w = dataclasses.replace(synth.WORKLOADS["interp_1024x576"], N=N, keys=keys)
    between = sum(2 for i in range(N) if i not in keys and keys[0] < i < keys[-1])
    assert bench.aligned_pairs(w) == between == expect


def test_frames_override_truncates_a_two_key_interpolation():
    w = synth.WORKLOADS["interp_1024x576"]
    g = np.zeros((w.N, 4, 4, 3), np.uint8)
    g[:, 0, 0, 0] = np.arange(w.N)
    s = np.zeros((2, 4, 4, 3), np.uint8)
    w2, g2, s2 = bench.truncate_interpolation(w, g, s, 12)
    assert (w2.N, w2.keys) == (12, (0, 11)) and g2.shape[0] == 12 and s2 is s
    assert (g2[:, 0, 0, 0] == np.arange(12)).all() and w2.pairs() == 20
    assert bench.truncate_interpolation(w, g, s, 0)[0] is w
    with pytest.raises(ValueError):
        bench.truncate_interpolation(w, g, s, 1)


def test_workload_labels_state_the_sizes_run():
    w = synth.WORKLOADS["blend_512"]
    assert bench.workload_label("blend_512", w) == w.name
    w5 = dataclasses.replace(w, window=5)
    assert "w5" in bench.workload_label("blend_512", w5) and w.name in bench.workload_label("blend_512", w5)
    assert "60x512x512 k5 w15 n6" in bench.workload_label("balanced_512", w)
    wi = synth.WORKLOADS["interp_1024x576"]
    assert "48x576x1024 k7 keys 0,47 n8" in bench.workload_label("aligned_1024x576", wi)
    wt = dataclasses.replace(wi, N=12, keys=(0, 11))
    assert "12x576x1024 k7 keys 0,11 n8" in bench.workload_label("aligned_1024x576", wt)
