"""Host-side helpers of bench.py (no GPU): the histogram throughput figure."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_onchip_rate():
    b = load_bench()
    r = b.onchip_rate(2_000_000_000, 1_000_000_000, 400.0, 1e10)
    assert r["pair_updates_per_s"] == 5e9 and r["elements_per_s"] == 2.5e9
    assert r["pair_updates"] == 2_000_000_000 and r["affinity_ms"] == 400.0
    assert r["frac"] == 0.25
    assert "frac" not in b.onchip_rate(10, 10, 1.0, None)
    assert b.onchip_rate(10, 10, 0, 1e9) is None and b.onchip_rate(10, 10, None, 1e9) is None


def test_traffic_record(tmp_path, monkeypatch):
    import hashlib
    import json
    b = load_bench()
    src = tmp_path / "k.cu"
    src.write_text("kernel")
    (tmp_path / "profiles").mkdir()
    rec = {"stage": "affinity", "kernel": "k", "dram_bytes": 300, "algorithmic_bytes": 100,
           "sources": ["k.cu"], "sources_sha256": hashlib.sha256(b"kernel").hexdigest()}
    (tmp_path / "profiles" / "roofline_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    assert b.traffic_record("affinity", 1000) == (3000.0, "k")
    assert b.traffic_record("gains", 1000) == (None, None)
    src.write_text("kernel changed")
    assert b.traffic_record("affinity", 1000)[0] is None


def test_pinned_to_one_core_restores_affinity():
    b = load_bench()
    if not hasattr(os, "sched_getaffinity"):
        return
    before = os.sched_getaffinity(0)
    with b.PinnedToOneCore() as pin:
        assert os.sched_getaffinity(0) == {pin.cpu} and pin.cpu in before
    assert os.sched_getaffinity(0) == before


def test_host_cpu():
    h = load_bench().host_cpu()
    assert h["cpus"] == os.cpu_count() and (h["model"] is None or isinstance(h["model"], str))
