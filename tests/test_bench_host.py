"""Host-side logic of bench.py, without a GPU: the clock sampler's window
and throttle-reason summary (on sample lines written by hand), the committed
per-agent traffic lookup, the kernel count per step, and the workload
naming of a precision override."""
import datetime

import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


class _Thread:
    def join(self, timeout=None):
        pass


def _sampler(lines):
    s = object.__new__(bench.ClockSampler)
    s.lines = lines
    s.proc = _Proc()
    s.t = _Thread()
    return s


def _line(t, sm, reasons=("Not Active",) * 4, power="250.0"):
    stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")
    return ", ".join([stamp, "0", str(sm), "2070", power, "0x0"] + list(reasons))


def test_clock_window_inside_the_timed_region():
    t0 = 1_000_000.0
    lines = [_line(t0 - 1.0, 1000)] + [_line(t0 + 0.1 * k, 2070) for k in range(1, 6)] + [_line(t0 + 5.0, 900)]
    got = _sampler(lines).stop(t0, t0 + 0.6)
    assert got["window"] == "timed region"
    assert got["samples"] == 5 and got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == [] and got["power_w_max"] == 250.0


def test_clock_window_extends_over_the_passes_after_a_short_region():
    t0 = 1_000_000.0
    lines = [_line(t0 + 0.01, 2070)] + [_line(t0 + 0.1 * k, 2055) for k in range(1, 5)]
    got = _sampler(lines).stop(t0, t0 + 0.02, t0 + 0.5)
    assert got["window"].startswith("timed region + the timing and end-to-end passes")
    assert got["samples"] == 5 and got["sm_mhz"] == 2055.0


def test_clock_window_adjacent_samples_and_reasons():
    t0 = 1_000_000.0
    slow = ("Active", "Not Active", "Not Active", "Active")
    lines = [_line(t0 - 0.2, 1900, slow), _line(t0 + 0.3, 1950), _line(t0 + 9.0, 800)]
    got = _sampler(lines).stop(t0, t0 + 0.01)
    assert got["window"] == "adjacent" and got["samples"] == 2
    assert got["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert got["sm_mhz"] == 1925.0


def test_clock_sampler_without_samples():
    assert _sampler([]).stop(0.0, 1.0) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_committed_traffic_lookup():
    for p in ("bf16", "fp8", "fp32"):
        rec = bench.committed_traffic("paper-1024x1024-65536slots-371-64-64-9-" + p)
        assert rec is not None and rec["dram_bytes_per_agent"] > 0 and "ncu" in rec["source"]
    per = {p: bench.committed_traffic("paper-1024x1024-65536slots-371-64-64-9-" + p)["dram_bytes_per_agent"]
           for p in ("bf16", "fp8", "fp32")}
    # the measured bytes sit within a few percent above the algorithmic ones
    for p, alg in (("fp32", 114212), ("bf16", 57380), ("fp8", 29512)):
        assert alg <= per[p] <= 1.05 * alg, p
    assert bench.committed_traffic("no-such-workload") is None


def test_kernels_per_step():
    assert bench.kernels_per_step(0, "simple") == 2
    assert bench.kernels_per_step(0, "terrain") == 2
    assert bench.kernels_per_step(1, "simple") == 9
    assert bench.kernels_per_step(1, "terrain") == 11


def test_precision_override_renames_the_workload():
    class A:
        workload = "paper"
        precision = "fp8"
        side = slots = founders = None

    (w,) = bench.make_workloads(A, 0)
    assert w["precision"] == "fp8" and w["name"].endswith("-fp8") and "bf16" not in w["name"]

    class B(A):
        side, slots, founders = 256, 4096, 3000

    (w,) = bench.make_workloads(B, 1)
    assert w["side"] == 256 and w["slots"] == 4096 and w["precision"] == "fp8"
