"""Host logic of bench.py, on the CPU: the sample windows of the CPU
baseline, the replica arithmetic, the traffic record's source check and the
reference arm's JSON line (its oracle timing replaced by a stand-in, so the
test takes no measurable time)."""
import argparse
import json
import os

import pytest

import bench
from conftest import ROOT
from paper_2310_19373_gb300 import inputs


def test_random_windows_are_distinct_aligned_and_in_range():
    wins = bench.random_windows(40, 22, 64, seed=3)
    assert len(wins) == 64 and len({lo for lo, _ in wins}) == 64
    for lo, hi in wins:
        assert hi - lo == 1 << 22 and lo % (1 << 22) == 0 and 0 <= lo and hi <= 1 << 40
    # more windows than the range holds: every window once
    assert sorted(bench.random_windows(6, 3, 100, seed=0)) == [(i << 3, (i + 1) << 3) for i in range(8)]
    # the same seed gives the same sample, another seed another one
    assert bench.random_windows(40, 22, 8, 5) == bench.random_windows(40, 22, 8, 5)
    assert bench.random_windows(40, 22, 8, 5) != bench.random_windows(40, 22, 8, 6)


def test_replica_arithmetic_without_a_process_group():
    assert bench.max_over_ranks(2.5, None) == 2.5
    assert bench.replica_throughput(4, 2.0 ** 40, 0.05) == pytest.approx(4 * 2.0 ** 40 / 0.05)


def test_cpu_baseline_times_at_least_one_window():
    r = bench.cpu_baseline(inputs.config_n40_f32(0), target_s=0.0, seed=1)
    assert r["kind"] == "oracle" and r["unit"] == "states/s"
    assert r["value"] > 0 and r["cores"] >= 1
    assert "1 windows of 2^22 states" in r["sample"]


def test_traffic_record_is_dropped_when_its_sources_change(tmp_path, monkeypatch):
    kernel = "walk_defer2_min_kernel<7>"
    assert bench.load_traffic(kernel) is not None  # committed record, unchanged sources
    assert bench.load_traffic("no_such_kernel") is None
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    rec[kernel]["source_sha256"] = "0" * 64
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    for src in rec[kernel]["sources"]:
        dst = tmp_path / src
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, src), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic(kernel) is None


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    calls = []

    def fake_baseline(Q, target_s=12.0, seed=0):
        calls.append(seed)
        return {"value": 4.0e7, "unit": "states/s", "cores": 16, "kind": "oracle",
                "cpu_model": "test", "sample": "stand-in"}

    monkeypatch.setattr(bench, "cpu_baseline", fake_baseline)
    args = argparse.Namespace(gpus=1, steps=2, warmup=3)
    bench.run_reference(args, rank=0)
    line = json.loads(capsys.readouterr().out.strip().split("\n")[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] == 4.0e7 and line["unit"] == "states/s" and line["higher_is_better"]
    assert line["ms_per_step"] == pytest.approx(2.0 ** 40 / 4.0e7 * 1e3)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 16
    assert line["e2e"] == {"value": 4.0e7, "unit": "states/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.WORKLOAD
    assert len(calls) == 5  # three warm-up samples, two timed
    # only rank 0 prints
    bench.run_reference(args, rank=1)
    assert capsys.readouterr().out == ""
