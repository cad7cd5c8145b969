"""bench.py's host-side pieces (CPU): the recorded DRAM-traffic captures are
well formed and only ever reported for the sources they were taken on."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_captures_are_well_formed():
    entries = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert entries, "no capture recorded"
    for e in entries:
        for key in ("kernel", "workload", "config", "source_sha256", "dram_bytes_per_launch",
                    "algorithmic_bytes_per_launch", "command"):
            assert key in e, key
        assert e["dram_bytes_per_launch"] == e["dram_bytes_read"] + e["dram_bytes_write"]
        # every row is read once: the capture cannot be below the algorithmic bytes,
        # and re-reads beyond a few percent would be a regression worth a look
        ratio = e["dram_bytes_per_launch"] / e["algorithmic_bytes_per_launch"]
        assert 1.0 <= ratio < 1.05, ratio
        assert "--clock-control none" in e["command"]


def test_traffic_is_reported_only_for_matching_sources_workload_and_config():
    b = _bench()
    e = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[0]
    src = b.kernel_source_hash(e["kernel"])
    got = b.measured_traffic(e["kernel"], e["workload"], e["config"])
    if e["source_sha256"] == src:
        assert got == e["dram_bytes_per_launch"]
    else:  # sources changed since the capture: nothing is reported
        assert got is None
    assert b.measured_traffic(e["kernel"], e["workload"], "9,9,9,9,9") is None
    assert b.measured_traffic(e["kernel"], "another workload", e["config"]) is None
    assert b.measured_traffic("k_unknown", e["workload"], e["config"]) is None
