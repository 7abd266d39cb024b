"""Host-side pieces of bench.py that need no GPU (CPU).

The recorded DRAM traffic is reported only while the kernel sources keep the
hashes they had when the counters were taken; the defaults run one GPU with
at least three warm-up steps; both arms report the same workload.
"""
import copy

import bench


def test_traffic_reported_only_for_the_captured_sources(monkeypatch):
    # with the hashes of the sources as they are now, the bytes are reported
    import hashlib
    import os
    current = copy.deepcopy(bench.TRAFFIC_TCX)
    for src in current["sources"]:
        with open(os.path.join(bench.ROOT, src), "rb") as f:
            current["sources"][src] = hashlib.sha1(f.read()).hexdigest()
    monkeypatch.setattr(bench, "TRAFFIC_TCX", current)
    assert bench.traffic_bytes(True) == current["bytes"]
    changed = copy.deepcopy(current)
    src = next(iter(changed["sources"]))
    changed["sources"][src] = "0" * 40
    monkeypatch.setattr(bench, "TRAFFIC_TCX", changed)
    assert bench.traffic_bytes(True) is None
    missing = copy.deepcopy(current)
    missing["sources"] = {"no/such/file.cu": "0" * 40}
    monkeypatch.setattr(bench, "TRAFFIC_TCX", missing)
    assert bench.traffic_bytes(True) is None


def test_defaults_one_gpu_and_three_warmup_steps():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and 1 <= a.steps <= 20
    assert a.impl == "libkrr"
    r = bench.parse_args(["--impl", "reference", "--steps", "2", "--warmup", "3"])
    assert r.impl == "reference" and (r.steps, r.warmup) == (2, 3)


def test_both_arms_report_the_same_workload():
    cfg = bench.bench_config(1)
    assert set(cfg) == {"workload", "l2", "parallelism"}
    assert "N=1048576" in cfg["workload"] and "d=3" in cfg["workload"]
    assert bench.bench_config(4)["workload"] == cfg["workload"]
