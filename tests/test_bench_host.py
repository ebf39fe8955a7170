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


class _FakeWorkload:
    """The parts of bench.Workload that the roofline reads."""

    def __init__(self, name, D, alg, bound="hbm"):
        self.name, self.D, self.D_override = name, D, None
        self._alg, self._bound = alg, bound

    def kernel_alg(self, kname, launches_per_step):
        return self._alg / launches_per_step, self._bound


def test_roofline_of_the_dominant_kernel(monkeypatch):
    """The kernel with the largest traced time is the dominant one; achieved
    = its algorithmic bytes per launch over its mean launch time, against the
    measured HBM peak."""
    monkeypatch.setattr(bench, "_peaks", lambda: (6000.0, "measured"))
    monkeypatch.setattr(bench, "_traffic_from_profiles", lambda w, k: None)
    wl = _FakeWorkload("d20_int64", 20, alg=2 * 60e9)  # per step, two launches
    prof = {"interp_pass": (20, 200.0), "tile_conv": (10, 60.0)}  # (launches, total ms)
    r = bench._roofline(wl, prof, steps=10)
    assert r["kernel"] == "interp_pass" and r["bound"] == "hbm"
    assert r["ms_per_launch"] == pytest.approx(10.0)
    assert r["achieved"] == pytest.approx(60e9 / 10e-3 / 1e9)  # GB/s
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    assert bench._roofline(wl, {}, steps=10) is None


def test_roofline_alu_bound_takes_the_measured_fp64_rate(monkeypatch):
    monkeypatch.setattr(bench, "_fp64_peak", lambda: (0.5e12, "measured probe"))
    wl = _FakeWorkload("d16_fp64", 16, alg=3e9, bound="alu")
    r = bench._roofline(wl, {"tile_conv": (4, 40.0)}, steps=4)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(0.5)
    assert r["achieved"] == pytest.approx(3e9 / 10e-3 / 1e12)
    assert r["frac_of_nominal"] == pytest.approx(r["achieved"] / 0.625)


def test_brief_keeps_the_reported_fields():
    res = {"ms_per_step": 1.23456789, "value": 3.0e11, "alg_hbm_frac": 0.123456,
           "roofline": {"kernel": "interp_pass", "bound": "hbm", "achieved": 5000.123456,
                        "frac": 0.7512345, "peak": 6780.7, "unit": "GB/s",
                        "ms_per_launch": 10.5, "traffic": None, "peak_source": "x"},
           "kernels": {"interp_pass": {"launches": 2, "ms": 21.0}}, "gpu_launches": 2,
           "clocks": {"sm_mhz": 2070.0}}
    b = bench._brief(res)
    assert b["ms_per_step"] == pytest.approx(1.23457)
    assert b["dominant"]["kernel"] == "interp_pass" and b["dominant"]["frac"] == 0.7512
    assert "peak_source" not in b["dominant"]
    assert b["kernels"] == res["kernels"] and b["clocks"] == res["clocks"]


def test_roofline_float_float_slab_takes_the_measured_fp32_rate(monkeypatch):
    """The float-float chunk kernels are arithmetic-bound: their roofline is
    binary32 operations per launch against the probe's binary32 rate."""
    monkeypatch.setattr(bench, "_fp32_peak", lambda: (30e12, "measured probe"))
    wl = _FakeWorkload("d16_mixed", 16, alg=5e9, bound="alu32")
    r = bench._roofline(wl, {"slab": (4, 2.0), "interp_pass": (4, 1.0)}, steps=4)
    assert r["kernel"] == "slab" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["peak"] == pytest.approx(30.0)
    assert r["achieved"] == pytest.approx(5e9 / 0.5e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 30.0)


def test_float_float_slab_operation_count():
    """The counted operations of the chunked-bulk kernel for the float-float
    forms: tile evaluation, products and interpolation of the unit's axes
    (D = 16, C = 8, m = 6 middle axes, 3^2 units)."""
    wl = bench.Workload.__new__(bench.Workload)
    wl.D, wl.sched = 16, {}
    wl.schedule_geometry = lambda: (3, 8, 6, 2, 8)
    for name, ea, mu in (("d16_mixed", 1, 1), ("d16_ff", 11, 9)):
        wl.name = name
        ops, bound = bench.Workload.kernel_alg(wl, "slab", 1)
        tile = 2 * (3 ** 8 - 2 ** 8) * ea + 3 ** 8 * mu
        assert bound == "alu32"
        assert ops == 9 * (3 ** 6 * tile + 14 * 3 ** 13 * 22)


def test_maxconv_kernel_bytes():
    """The max-convolution's own kernels: the root reads the (D + e)-axis
    convolution once and writes the 3^D maxima; the spread reads x, y and
    writes the two limb cubes; the convolution's kernels are counted on its
    D + e axes."""
    wl = bench.Workload.__new__(bench.Workload)
    wl.name, wl.D, wl.conv_D, wl.sched = "maxconv", 14, 18, {}
    b, bound = bench.Workload.kernel_alg(wl, "maxconv_root", 1)
    assert bound == "hbm" and b == 8 * (3 ** 18 + 3 ** 14)
    b, _ = bench.Workload.kernel_alg(wl, "maxconv_spread", 1)
    assert b == 8 * (2 * 2 ** 14 + 2 * 2 ** 18)
    b, _ = bench.Workload.kernel_alg(wl, "interp_pass", 2)
    assert b == 2 * 3 ** 18 * 8
