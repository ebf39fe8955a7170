"""Host logic of bench.py (no GPU): the end-to-end step timer's step count
and statistics, and the traffic lookup keyed by the kernel sources' hash."""
import os
import sys
import time

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_timed_host_steps_counts_and_stats():
    calls = []

    def one():
        calls.append(1)
        time.sleep(0.002)

    steps, total = bench._timed_host_steps(one, 3, 1, min_seconds=0.05, max_steps=100)
    # one warm-up, one sizing step, then `steps` timed steps
    assert len(calls) == steps + 2
    assert 3 <= steps <= 100
    st = bench._timed_host_steps.last
    assert total >= steps * 0.002
    assert st["step_ms_min"] <= st["step_ms_median"] <= 1e3 * total


def test_timed_host_steps_bounds():
    steps, _ = bench._timed_host_steps(lambda: time.sleep(0.03), 3, 0, min_seconds=0.01)
    assert steps == 3  # at least min_steps
    steps, _ = bench._timed_host_steps(lambda: None, 3, 0, min_seconds=10.0, max_steps=7)
    assert steps == 7  # at most max_steps


def test_traffic_lookup_only_on_current_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench._src_hash()  # of the (empty) sources under the patched root
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.txt").write_text(
        "# comment\n"
        f"d20_int64 interp_pass 55.0e9 {h}\n"
        "d18_fp32 interp_pass 3.0e9 000000000000\n")
    assert bench._traffic_from_profiles("d20_int64", "interp_pass") == pytest.approx(55.0e9)
    assert bench._traffic_from_profiles("d18_fp32", "interp_pass") is None  # other sources
    assert bench._traffic_from_profiles("batched", "batched_interp") is None
