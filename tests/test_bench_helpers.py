"""Host-side helpers of bench.py (no GPU): the dominant stage's kernel name, the DRAM-traffic
record guarded by the kernel source's SHA-1, and the whole-job throughput."""
import hashlib
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stage_kernel_names():
    assert bench._stage_kernel("knn_tile", "learned_bf16_tc", {"tc_variant": "staged"}) == "knn_tc_kernel"
    assert bench._stage_kernel("knn_tile", "fp16_tc", {"tc_variant": "pipelined"}) == "knn_tcp_kernel"
    assert bench._stage_kernel("knn_tile", "plain_fp32", {}) == "knn_tile_kernel"
    assert bench._stage_kernel("knn_retry", "learned_fp32", {}) == "knn_tile_kernel"
    assert bench._stage_kernel("sweep_density", "plain_fp32", {}) == "sweep57_kernel"
    assert bench._stage_kernel("graph", "plain_fp32", {}) == "graph"


def test_traffic_record_follows_the_source_hash():
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, r in rec.items():
        stage, form, workload = key.split("/")
        current = hashlib.sha1(open(os.path.join(ROOT, r["source"]), "rb").read()).hexdigest()
        got = bench._traffic(stage, form, workload)
        # the recorded bytes while the kernel's source is the one captured, else no figure
        assert got == (r["dram_bytes_per_launch"] if current == r["source_sha1"] else None), key
    assert bench._traffic("knn_tile", "no_such_form", "no_such_workload") is None


def test_job_throughput_counts_every_rank_over_the_slowest():
    # 2 ranks, 10 steps of 1,000,000 points each, the slowest rank taking 0.5 s in all
    assert bench.job_throughput(1_000_000, 10, 2, 0.5) == 40_000_000
