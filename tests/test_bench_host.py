"""Host logic of bench.py that needs no GPU: the FP32-vs-FP64 error
statistics, the clock record over the timed window, and the workload
descriptions both arms print."""
import importlib.util
import os
import types

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _run(weight, me2, passed):
    return types.SimpleNamespace(t={"weight": weight, "me2": me2, "pass": passed}, n_events=weight.numel())


def test_precision_error_statistics(bench):
    g = torch.Generator().manual_seed(3)
    n = 4000
    w64 = torch.rand(n, generator=g, dtype=torch.float64) + 0.5
    m64 = 2.0 * w64
    p64 = torch.ones(n, dtype=torch.uint8)
    p64[:100] = 0  # failing in both
    rel = torch.full((n,), 1e-6, dtype=torch.float64)
    rel[100:110] = 0.5  # a tail of ill-conditioned events
    w = w64 * (1.0 + rel)
    m64[200:230] = 1e-40  # vanishing helicity configurations: counted, not compared
    p = p64.clone()
    p[300:303] = 0  # cut decisions that differ
    st = bench.precision_error(torch, _run(w, m64, p), _run(w64, m64, p64))
    assert st["events"] == n
    assert st["cut_flips"] == 3
    assert st["vanishing"] == 30
    assert st["compared"] == n - 100 - 3 - 30
    assert st["median"] == pytest.approx(1e-6, rel=1e-6)
    assert st["max"] == pytest.approx(0.5, rel=1e-12)
    assert st["above_1e_2"] == 10
    assert 1e-6 * 0.999 <= st["p99"] <= 0.5


def test_precision_error_nothing_to_compare(bench):
    z = torch.zeros(8, dtype=torch.float64)
    st = bench.precision_error(torch, _run(z, z, torch.zeros(8, dtype=torch.uint8)),
                               _run(z, z, torch.zeros(8, dtype=torch.uint8)))
    assert st["compared"] == 0 and "median" not in st


def test_clock_summary_keeps_the_timed_window(bench):
    clk = bench.ClockSampler("0")
    idle = ["1100", "2070", "200.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]
    busy = ["2070", "2070", "900.0", "0x0", "Not Active", "Not Active", "Not Active", "Active"]
    hot = ["1500", "2070", "900.0", "0x0", "Not Active", "Active", "Not Active", "Not Active"]
    clk.rows = [(0.0, idle), (1.0, busy), (1.5, busy), (2.0, busy), (3.0, hot)]
    s = clk.summary([0.9, 2.1])
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    s_all = clk.summary()
    assert s_all["samples"] == 5 and "hw_thermal_slowdown" in s_all["reasons"]
    assert clk.summary([5.0, 6.0])["reasons"] == ["unsampled"]


def test_both_arms_describe_the_same_workload(bench):
    for name, wl in bench.WORKLOADS.items():
        cfg = bench.workload_config(name, wl, wl["n_events"])
        assert cfg["workload"].startswith(name) and cfg["events_per_gpu"] == wl["n_events"]
        assert cfg["n_gluons"] == wl["n"]
        assert isinstance(bench.workload_metric(wl), str) and bench.workload_metric(wl)


def test_traffic_record_lookup(bench, tmp_path, monkeypatch):
    """The committed DRAM-traffic record is used only for the kernel sources it
    was captured on and the variant it names, scaled to the launch size."""
    import json
    (tmp_path / "profiles").mkdir()
    h = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    rec = {"source_hash": h,
           "by_variant": {"4": {"kernel": "k", "events_per_launch": 1000, "dram_bytes_per_launch": 250_000}}}
    (tmp_path / "profiles" / "traffic_gg4g.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_traffic("gg4g", 4, 500) == 125_000
    assert bench.read_traffic("gg4g", 0, 500) is None      # no capture of this variant
    assert bench.read_traffic("gg8g", 4, 500) is None      # no record for this workload
    rec["source_hash"] = "0" * 64                            # kernels changed since the capture
    (tmp_path / "profiles" / "traffic_gg4g.json").write_text(json.dumps(rec))
    assert bench.read_traffic("gg4g", 4, 500) is None


def test_committed_traffic_records_are_well_formed(bench):
    """Every committed record names the source hash it was taken on and, per
    amplitude variant, a full launch's events and DRAM bytes (a record whose
    hash no longer matches is ignored by read_traffic, not an error)."""
    import glob
    import json
    import re
    files = glob.glob(os.path.join(ROOT, "profiles", "traffic_*.json"))
    assert files
    for f in files:
        rec = json.load(open(f))
        assert re.fullmatch(r"[0-9a-f]{64}", rec["source_hash"]), f
        assert rec["by_variant"]
        for v, e in rec["by_variant"].items():
            assert int(v) >= 0 and e["events_per_launch"] > 0 and e["dram_bytes_per_launch"] > 0
