"""CPU checks of the bench's host-side helpers behind the JSON line's
roofline fields: bytes per stored rounded cost, the measured-peak lookup,
and the DRAM-traffic summary that stays valid only while the phase kernel's
sources are unchanged."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_helpers_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_bytes_per_rounded_cost_matches_the_byte_storage_limit():
    """The library stores rounded costs as bytes when floor(1/eps) <= 252."""
    b = load_bench()
    assert b.cbar_bytes(0.01) == 1 and b.cbar_bytes(0.1) == 1
    assert b.cbar_bytes(1 / 252) == 1 and b.cbar_bytes(1 / 253.5) == 2
    assert b.cbar_bytes(0.005) == 1 and b.cbar_bytes(0.003) == 2


def test_measured_peak_or_labelled_fallback(tmp_path, monkeypatch):
    b = load_bench()
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    peak, src = b.measured_peak()
    assert peak == 6800.0 and src.startswith("fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6779.0}))
    peak, src = b.measured_peak()
    assert peak == 6779.0 and src.startswith("measured")


def test_traffic_summary_only_for_unchanged_sources(monkeypatch):
    """The summary's bytes are reported while its hash equals the phase
    kernel's sources and null for any other hash (a changed kernel)."""
    b = load_bench()
    d = json.load(open(os.path.join(ROOT, "profiles", "k_phases_traffic.json")))
    assert d["dram_bytes_per_launch"] == d["dram_bytes_read"] + d["dram_bytes_write"]
    monkeypatch.setattr(b, "src_hash", lambda: d["src_hash"])
    assert b.ncu_traffic() == d["dram_bytes_per_launch"]
    monkeypatch.setattr(b, "src_hash", lambda: "0" * 16)
    assert b.ncu_traffic() is None


def test_latency_roofline_arithmetic():
    """Floor = barriers x (one barrier + three dependent L2 loads); the
    fraction is the floor over the measured phase-loop time."""
    import bench
    r = bench.latency_roofline(1000, 900.0, 150.0, 2.7)
    assert abs(r["floor_ms"] - 1000 * (900.0 + 3 * 150.0) * 1e-6) < 1e-12
    assert abs(r["frac"] - r["floor_ms"] / 2.7) < 1e-12
    assert r["bound"] == "latency" and r["barriers"] == 1000
