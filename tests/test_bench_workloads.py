"""Every frame workload bench.py offers builds, names its configuration, and its
CPU baseline (the oracle on a bounded sample) runs: the bench cannot fail on
the GPU machine for want of a key or an oracle argument."""
import argparse
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

KEYS = ("scene", "array", "angles", "n_rays", "seed", "max_bounces", "max_path", "x_px", "z_px", "dyn_range_db")


@pytest.mark.parametrize("name", sorted(bench.FRAME_WORKLOADS))
def test_frame_workload_builds_and_its_baseline_runs(name):
    w = bench.frame_workload(argparse.Namespace(workload=name))
    for k in KEYS:
        assert k in w, (name, k)
    n_tx = len(np.atleast_1d(w["angles"]))
    if w.get("transmits") is not None:
        assert len(w["transmits"]) == n_tx
    assert isinstance(bench.FRAME_WORKLOADS[name], str) and len(bench.FRAME_WORKLOADS[name]) > 40
    # a sample small enough for the CPU suite: 1024 rays per transmit, a 16 x 16 image
    w = dict(w, n_rays=1024, x_px=w["x_px"][::max(1, len(w["x_px"]) // 16)],
             z_px=w["z_px"][::max(1, len(w["z_px"]) // 16)])
    rate, n, dt, threads = bench.oracle_rate(w, 0.05, threads=4)
    assert rate > 0 and n == 1024 and dt > 0 and threads == 4


def test_mixed_workload_mixes_and_mesh_workload_has_triangles():
    a = argparse.Namespace
    assert bench.frame_workload(a(workload="mixed"))["mix"] is True
    assert not bench.frame_workload(a(workload="paper")).get("mix")
    tri, med = bench.frame_workload(a(workload="mesh"))["scene"]["triangles"]
    assert tri.shape == (5120 + 2 * 96 * 4, 9) and med.shape == (tri.shape[0], 2)
    syn = bench.frame_workload(a(workload="synthetic"))
    assert all(k == 3 for k, _, _ in syn["transmits"]) and syn["n_rays"] * len(syn["transmits"]) == 10_000_000
