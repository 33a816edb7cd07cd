"""Committed ncu counters as the benchmark reads them (CPU): values come from a
profile summary's machine-readable block only while the hashed sources are
unchanged."""
import hashlib
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _write(root, src_text, sha=None):
    (root / "profiles").mkdir()
    (root / "k.cu").write_text(src_text)
    if sha is None:
        sha = hashlib.sha256(src_text.encode()).hexdigest()
    (root / "profiles" / "k_t5_x.md").write_text(
        "# summary\n\n| a | b |\n|---|---|\n\nkernel: t5\ndram_bytes_per_launch: 123\n"
        "fp32_flop_per_launch: 4.5e8\nsources: k.cu\nsources_sha256: " + sha + "\n")


def test_counters_follow_the_source_hash(tmp_path, monkeypatch):
    _write(tmp_path, "kernel source\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    c = bench.measured_counters("t5")
    assert c == {"dram_bytes_per_launch": 123.0, "fp32_flop_per_launch": 4.5e8}
    assert bench.measured_traffic("t5") == 123
    assert bench.measured_counters("t3") == {}
    (tmp_path / "k.cu").write_text("kernel source, edited\n")
    assert bench.measured_counters("t5") == {} and bench.measured_traffic("t5") is None


def test_counters_of_a_missing_source_are_dropped(tmp_path, monkeypatch):
    _write(tmp_path, "x\n", sha="0" * 64)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_counters("t5") == {}
    os.remove(tmp_path / "k.cu")
    assert bench.measured_traffic("t5") is None


def test_committed_profiles_match_the_current_sources():
    c = bench.measured_counters("t5")
    assert c.get("dram_bytes_per_launch", 0) > 1e6
    assert c.get("fp32_flop_per_launch", 0) > 1e8 and c.get("atom_inst_per_launch", 0) > 0
