"""bench.py's DRAM traffic figure without a GPU: it comes from the committed
ncu summary of the roofline kernel, scaled by units, and is null once the
kernel sources hash differently from the capture."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_summaries_exist_and_parse():
    for name, rel in bench.TRAFFIC_PROFILES.items():
        f = bench.profile_fields(rel)
        assert f, rel
        for k in ("kernel source hash", "dram bytes read", "dram bytes write", "captured units"):
            assert k in f, (rel, k)
        assert int(f["dram bytes read"]) > 0 and int(f["dram bytes write"]) > 0
        assert float(f["captured units"]) > 0


def test_traffic_scales_by_units_and_follows_the_hash(monkeypatch):
    f = bench.profile_fields(bench.TRAFFIC_PROFILES["c4"])
    b = int(f["dram bytes read"]) + int(f["dram bytes write"])
    u = float(f["captured units"])
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: f["kernel source hash"])
    got, note = bench.measured_traffic("c4", u)
    assert got == b and "this launch" in note
    got, note = bench.measured_traffic("c4", 20 * u)
    assert got == 20 * b and "scaled" in note
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.measured_traffic("c4", u) == (None, "kernel changed since the capture")
    assert bench.measured_traffic("c1", u) == (None, "no capture")


def test_kernel_source_hash_covers_every_listed_file():
    for rel in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(ROOT, rel)), rel
    assert len(bench.kernel_source_hash()) == 16
