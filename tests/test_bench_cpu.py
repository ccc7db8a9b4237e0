"""The benchmark's roofline bookkeeping on the host: DRAM traffic per launch
is taken from a committed capture only while the kernel sources hash to the
capture's value and only for the pass role that dominates the run; the
batched uneven exec counts one read and one write of every value it
transforms per launch (the one-launch form both phases, phase 0 the single
passes and four-step columns).  No GPU."""
import json
import os

import pytest

import bench


@pytest.fixture
def traffic_file(tmp_path, monkeypatch):
    os.makedirs(tmp_path / "profiles")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: "h1")

    def write(d):
        with open(tmp_path / "profiles" / "traffic.json", "w") as f:
            json.dump(d, f)
    return write


def test_traffic_entry_needs_the_current_kernel_hash_and_the_pass(traffic_file):
    traffic_file({"w": {"kernel_hash": "h1", "pass": "axis2", "dram_bytes_per_launch": 7},
                  "stale": {"kernel_hash": "h0", "pass": "axis2", "dram_bytes_per_launch": 9}})
    assert bench.load_traffic("w")["dram_bytes_per_launch"] == 7
    assert bench.load_traffic("w", "axis2")["dram_bytes_per_launch"] == 7
    assert bench.load_traffic("w", "axis1") is None
    assert bench.load_traffic("stale") is None
    assert bench.load_traffic("absent") is None


def test_traffic_entries_per_pass_role(traffic_file):
    traffic_file({"u": [{"kernel_hash": "h1", "pass": "many.uneven", "dram_bytes_per_launch": 11},
                        {"kernel_hash": "h1", "pass": "many.uneven.phase0", "dram_bytes_per_launch": 5}]})
    assert bench.load_traffic("u", "many.uneven")["dram_bytes_per_launch"] == 11
    assert bench.load_traffic("u", "many.uneven.phase0")["dram_bytes_per_launch"] == 5
    assert bench.load_traffic("u", "many.uneven.phase1") is None


def test_no_traffic_file_means_no_traffic(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic("w") is None


def test_uneven_roofline_bytes_per_launch_form(traffic_file):
    traffic_file({})
    peaks = {"hbm_gbs": 1.0, "source": "measured"}  # the helper rounds GB/s to 0.01 and fractions to 1e-4
    lens = [1000, 4096, 65536] * 1000
    bytes_step = float(sum(16 * n for n in lens))
    rows = float(sum(16 * n for n in lens if n > 2048))
    # one launch of 2 ms per exec, 10 execs profiled
    r = bench.uneven_roofline([("many.uneven", 20.0, 10)], 10, lens, bytes_step, 2.0, 1, "u", peaks)
    assert r["kernel_pass"] == "many.uneven"
    assert r["algorithmic_bytes_per_launch"] == bytes_step + rows
    assert r["achieved"] == pytest.approx((bytes_step + rows) / 2e-3 / 1e9, abs=0.01)
    assert r["traffic"] is None
    # two launches: phase 0 dominates, its bytes are one pass over every value
    r = bench.uneven_roofline([("many.uneven.phase0", 12.0, 10), ("many.uneven.phase1", 9.0, 10)], 10, lens,
                              bytes_step, 2.1, 2, "u", peaks)
    assert r["kernel_pass"] == "many.uneven.phase0"
    assert r["algorithmic_bytes_per_launch"] == bytes_step
    assert r["frac"] == pytest.approx(bytes_step / 1.2e-3 / 1e9, abs=1e-3)
