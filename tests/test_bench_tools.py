"""Host-side pieces of bench.py that need no GPU: the traffic figure read from
a committed ncu summary (only while its recorded source hash matches), the
measured-peak lookup and the serving stream's Poisson arrivals."""
import hashlib
import os
import sys
import types

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _fake_root(tmp_path, source_text, recorded_hash, value="1234567"):
    (tmp_path / "paper_1702_03484_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "paper_1702_03484_gb300" / "csrc" / "join.cu").write_text(source_text)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dense_write_skewed_join.md").write_text(
        f"# x\n\n- source: join.cu\n- source_sha256: {recorded_hash}\n- dram_bytes_per_launch: {value}\n")
    return str(tmp_path)


def test_traffic_read_while_the_source_hash_matches(tmp_path, monkeypatch):
    src = "kernel source v1\n"
    digest = hashlib.sha256(src.encode()).hexdigest()[:16]
    monkeypatch.setattr(bench, "ROOT", _fake_root(tmp_path, src, digest))
    assert bench.ncu_traffic("dense_write", "skewed_join") == 1234567.0
    assert bench.ncu_traffic("join_write", "skewed_join") is None  # no summary for that kernel


def test_traffic_dropped_once_the_kernel_changed(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", _fake_root(tmp_path, "kernel source v2\n", "0123456789abcdef"))
    assert bench.ncu_traffic("dense_write", "skewed_join") is None


def test_committed_summaries_name_their_command_and_source():
    prof = os.path.join(ROOT, "profiles")
    names = [n for n in os.listdir(prof) if n.endswith(".md")]
    assert names
    for n in names:
        text = open(os.path.join(prof, n)).read()
        assert "- command: `" in text and "ncu " in text and "--clock-control none" in text, n
        assert "- source_sha256: " in text, n


def test_measured_peak_is_used_when_present():
    peak, kind = bench.measured_peaks()
    assert peak > 1000 and kind in ("measured", "fallback")


def test_serving_arrivals_are_poisson_and_seeded():
    w = bench.Serving.__new__(bench.Serving)  # only the stream parameters, no graph
    w.seed, w.rate, w.step_s, w.bgps = 5, 2000.0, 1.5, list(range(64))
    t, idx = w.stream(4, part=2)
    t2, idx2 = w.stream(4, part=2)
    assert np.array_equal(t, t2) and np.array_equal(idx, idx2)
    assert np.all(np.diff(t) > 0) and t[-1] < 6.0
    assert abs(t.shape[0] / 6.0 - 2000.0) < 3 * np.sqrt(2000.0 * 6.0) / 6.0  # rate within 3 sigma
    gaps = np.diff(t)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05  # exponential gaps: unit coefficient of variation
    assert idx.min() >= 0 and idx.max() < 64


def test_small_sizes_exist_for_profiled_joins():
    a = types.SimpleNamespace(workload="skewed_join", size="small")
    w = bench.make_workload(a)
    assert w.A.nrows == 1 << 24 and w.B.nrows == 1 << 22
