"""Host logic of bench.py that decides what its JSON line claims.

The roofline's `traffic` comes from a committed ncu summary (DRAM bytes per algorithmic byte
of a smaller case) and is only valid while the solve kernel's sources are the ones the
counters were taken on: the summary lists their sha256 digests, and `recorded_traffic` must
return None as soon as one differs or is missing.  The workload label must name the level
count, the point count and the configuration of the hierarchy that was actually run.  The CPU
baseline's extrapolation is a least-squares power law through its samples.
"""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _tree(tmp_path, files, traffic=0.8125, digests=None):
    csrc = tmp_path / "paper_2503_04914_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    lines = ["# a summary", ""]
    for name, body in files.items():
        (csrc / name).write_bytes(body)
        d = (digests or {}).get(name, hashlib.sha256(body).hexdigest())
        lines.append(f"kernel_source_sha256 {name}: {d}")
    lines.append(f"traffic_per_algorithmic_byte: {traffic}")
    (tmp_path / "profiles" / "p.txt").write_text("\n".join(lines) + "\n")
    return csrc


def test_traffic_gate_follows_the_kernel_sources(tmp_path, monkeypatch):
    csrc = _tree(tmp_path, {"a.cuh": b"kernel a\n", "b.cu": b"kernel b\n"})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("p.txt") == 0.8125
    (csrc / "b.cu").write_bytes(b"kernel b, changed\n")
    assert bench.recorded_traffic("p.txt") is None
    (csrc / "b.cu").unlink()
    assert bench.recorded_traffic("p.txt") is None
    assert bench.recorded_traffic("missing.txt") is None


def test_traffic_gate_rejects_a_wrong_digest(tmp_path, monkeypatch):
    _tree(tmp_path, {"a.cuh": b"kernel a\n"}, digests={"a.cuh": "0" * 64})
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("p.txt") is None


def test_committed_traffic_line_is_current_or_withheld():
    v = bench.recorded_traffic()
    assert v is None or v > 0


def test_workload_label_names_the_run_hierarchy():
    from paper_2503_04914_gb300 import inputs
    assert bench.halton_points(8) == 1398080
    assert "8 levels" in bench.workload_label(8) and "1,398,080 points" in bench.workload_label(8)
    # the headline is the learned-preconditioner configuration: delta = 8 h, phi_{2,2}
    assert bench.workload_label(8).startswith("halton8_d2_nu8_w22")
    assert "phi_{2,2}" in bench.workload_label(8) and "delta_j=8*" in bench.workload_label(8)
    assert bench.workload_label(8, 4.0, (2, 1)).startswith("halton8_d2_nu4_w21")
    for L in (3, 5):
        w = inputs.halton_hierarchy(L=L, nu=bench.HEAD_NU, wendland=bench.HEAD_W)
        assert w.N == bench.halton_points(L)
        assert w.name == bench.workload_label(L).split(":")[0]
        assert f"{L} levels" in bench.workload_label(L) and f"{w.N:,} points" in bench.workload_label(L)


def test_power_law_extrapolation():
    # exact on a power law, and the exponent it reports
    est, b = bench.power_law([(1000, 2.0), (4000, 32.0)], 16000)
    assert abs(b - 2.0) < 1e-12 and abs(est - 512.0) < 1e-9
    est, b = bench.power_law([(10, 1.0), (100, 10.0), (1000, 100.0)], 1e6)
    assert abs(b - 1.0) < 1e-12 and abs(est - 1e5) < 1e-6
