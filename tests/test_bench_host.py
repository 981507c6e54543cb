"""Host-side logic of bench.py (no GPU): the summary of the nvidia-smi clock samples
taken during the timed region, the look-up of the recorded ncu traffic of the
dominant kernel (used only while the kernel sources are the ones it was taken on),
and the moment stack that the end-to-end step moves."""
import importlib.util
import json
import os

import numpy as np
import pytest

from paper_2101_03055_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary_takes_the_median_and_the_active_reasons(bench):
    s = bench.ClockSampler(0)
    s.samples = [
        ["0", "2070", "2070", "950.1", "0x0000000000000000", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "1950", "2070", "1390.0", "0x0000000000000004", "Not Active", "Not Active", "Not Active", "Active"],
        ["0", "2010", "2070", "1200.5", "0x0000000000000000", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["0", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]"],
    ]
    out = s.summary()
    assert out["sm_mhz"] == 2010.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 4
    s.samples.append(["0", "1500", "2070", "800", "0x8", "Active", "Not Active", "Active", "Not Active"])
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["nvidia-smi unavailable"]


def test_recorded_traffic_is_used_only_for_the_sources_it_was_taken_on(bench, monkeypatch):
    with open(os.path.join(ROOT, "profiles", "step_kernel_traffic.json")) as fh:
        records = json.load(fh)
    name, rec = "batched_plume_sweep_256", records["batched_plume_sweep_256"]
    current = rec["kernel_hash"] == bench.kernel_source_hash(bench.KERNEL_SOURCES_2D)
    got = bench.recorded_profile(name, rec["kernel"] + " x 256 instance chains")
    assert (got is not None) == current
    if current:
        assert got["dram_bytes_per_launch"] == rec["dram_bytes_per_launch"]
    # another kernel, or sources that changed since the capture: no record
    assert bench.recorded_profile(name, "step_kernel_flat<2,float>") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda files=None: "0000000000000000")
    assert bench.recorded_profile(name, rec["kernel"]) is None
    assert bench.recorded_profile("no_such_workload", rec["kernel"]) is None


def test_moment_stack_of_a_problem(bench):
    pb = I.chemotaxis_plume(40, 24, seed=3)
    st = bench.moment_stack(pb)
    assert st.shape == (pb.m + 3, 24, 40) and st.dtype == np.float32
    np.testing.assert_array_equal(st[:pb.m], np.asarray(pb.phi0, np.float32))
    np.testing.assert_array_equal(st[pb.m:pb.m + 2], np.asarray(pb.u0, np.float32))
    if pb.p0 is None:
        assert np.all(st[pb.m + 2] == 0.0)
