"""Host logic of bench.py that decides what its JSON line claims.

The roofline's `traffic` comes from a committed ncu summary and is only valid while the
solve kernel's sources are the ones the counters were taken on: the summary lists their
sha256 digests, and `recorded_traffic` must return None as soon as one differs or is
missing.  The workload label must name the level count and the point count of the
hierarchy that was actually run.
"""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _tree(tmp_path, files, traffic=123456789.0, digests=None):
    csrc = tmp_path / "paper_2503_04914_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    lines = ["# a summary", ""]
    for name, body in files.items():
        (csrc / name).write_bytes(body)
        d = (digests or {}).get(name, hashlib.sha256(body).hexdigest())
        lines.append(f"kernel_source_sha256 {name}: {d}")
    lines.append(f"traffic_bytes_per_launch: {int(traffic)}")
    (tmp_path / "profiles" / "p.md").write_text("\n".join(lines) + "\n")
    return csrc


def test_traffic_gate_follows_the_kernel_sources(tmp_path, monkeypatch):
    csrc = _tree(tmp_path, {"a.cuh": b"kernel a\n", "b.cu": b"kernel b\n"})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("p.md") == 123456789.0
    (csrc / "b.cu").write_bytes(b"kernel b, changed\n")
    assert bench.recorded_traffic("p.md") is None
    (csrc / "b.cu").unlink()
    assert bench.recorded_traffic("p.md") is None
    assert bench.recorded_traffic("missing.md") is None


def test_traffic_gate_rejects_a_wrong_digest(tmp_path, monkeypatch):
    _tree(tmp_path, {"a.cuh": b"kernel a\n"}, digests={"a.cuh": "0" * 64})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("p.md") is None


def test_committed_traffic_line_is_current_or_withheld():
    v = bench.recorded_traffic()
    assert v is None or v > 0


def test_workload_label_names_the_run_hierarchy():
    from paper_2503_04914_gb300 import inputs
    assert bench.halton_points(8) == 1398080
    assert "8 levels" in bench.workload_label(8) and "1,398,080 points" in bench.workload_label(8)
    for L in (3, 5):
        w = inputs.halton_hierarchy(L=L)
        assert w.N == bench.halton_points(L)
        assert f"{L} levels" in bench.workload_label(L) and f"{w.N:,} points" in bench.workload_label(L)
