"""The bench's clock sampler on CPU, fed by a stand-in for nvidia-smi that
prints rows in the same CSV layout: only rows stamped inside the timed region
are summarised, throttle reasons are read per row, priming stops once the
sampler is live, and buffered output is still placed by its own timestamps."""
import sys
import time

import pytest

import bench

FAKE = r"""
import datetime, signal, sys, time
period, reason, buffered = float(sys.argv[1]), sys.argv[2], sys.argv[3] == "1"
signal.signal(signal.SIGTERM, lambda *a: sys.exit(0))
mhz = 1980
while True:
    ts = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    cap = "Active" if reason == "cap" else "Not Active"
    print(f"{ts}, 0, {mhz}, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, {cap}",
          flush=not buffered)
    mhz = 2070 if mhz == 1980 else 1980
    time.sleep(period)
"""


class FakeSampler(bench.ClockSampler):
    def __init__(self, period=0.01, reason="none", buffered=False, missing=False):
        super().__init__(0)
        self.args = [str(period), reason, "1" if buffered else "0"]
        self.missing = missing

    def command(self):
        if self.missing:
            return ["/nonexistent/nvidia-smi-stand-in"]
        return [sys.executable, "-c", FAKE] + self.args


def _region(clk, seconds, prime=None, wait_s=3.0):
    clk.start(prime=prime, wait_s=wait_s)
    with clk:
        time.sleep(seconds)
    return clk.summary()


def test_rows_inside_the_region_only():
    calls = []
    res = _region(FakeSampler(period=0.01), 0.3, prime=lambda: (calls.append(1),
                                                                 time.sleep(0.005)))
    assert res["samples"] >= 5
    assert res["sm_mhz"] in (1980.0, 2025.0, 2070.0)
    assert res["sm_max_mhz"] == 2070.0
    assert res["reasons"] == []
    assert res["prime_steps"] == len(calls) >= 1
    assert 290 <= res["region_ms"] < 1000


def test_active_reason_is_reported_and_not_active_is_not():
    res = _region(FakeSampler(period=0.01, reason="cap"), 0.2, prime=lambda: time.sleep(0.005))
    assert res["reasons"] == ["sw_power_cap"]


def test_region_shorter_than_the_period_reports_the_nearest_row():
    res = _region(FakeSampler(period=0.5), 0.001, prime=lambda: time.sleep(0.005))
    assert res["samples"] == 0
    assert res["nearest_ms"] >= 0
    assert res["sm_mhz"] is not None


def test_buffered_output_is_placed_by_its_timestamps():
    # nothing arrives before exit: priming gives up after wait_s, rows are still dated
    res = _region(FakeSampler(period=0.01, buffered=True), 0.3,
                  prime=lambda: time.sleep(0.01), wait_s=0.3)
    assert res["prime_steps"] >= 10
    assert res["samples"] >= 5


def test_missing_sampler_reports_unsampled():
    res = _region(FakeSampler(missing=True), 0.01)
    assert res == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_sampler_without_start_still_works():
    clk = FakeSampler(period=0.01)
    with clk:
        time.sleep(0.3)
    res = clk.summary()
    assert "prime_steps" not in res
    assert res["sm_mhz"] is not None


def test_unparsed_stamps_fall_back_to_arrival_time():
    clk = FakeSampler(period=0.01)
    clk.start(prime=lambda: time.sleep(0.005))
    with clk:
        time.sleep(0.2)
    clk.lines = [(t, "garbled" + line[line.index(","):]) for t, line in clk.lines]
    res = clk.summary()
    assert res["samples"] >= 3


def test_gpu_found_by_uuid_not_by_cuda_index():
    listing = ("0, GPU-11111111-aaaa-bbbb-cccc-000000000000\n"
               "1, GPU-22222222-aaaa-bbbb-cccc-000000000000\n")
    # the process sees one GPU (CUDA index 0) that nvidia-smi numbers 1
    assert bench.smi_index_of("22222222-AAAA-bbbb-cccc-000000000000", listing, "0") == "1"
    assert bench.smi_index_of("GPU-11111111-aaaa-bbbb-cccc-000000000000", listing, "5") == "0"
    assert bench.smi_index_of("33333333-aaaa-bbbb-cccc-000000000000", listing, "0") == "0"
    assert bench.smi_index_of("", listing, "2") == "2"
    assert bench.smi_index_of("x", "garbled", "3") == "3"


def test_smi_index_falls_back_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("needs a machine without a GPU")
    assert bench.smi_index(torch.device("cuda", 3)) == "3"


def test_failing_prime_stops_the_sampler():
    clk = FakeSampler(period=0.01, buffered=True)     # no row arrives early: prime runs

    def prime():
        raise RuntimeError("step failed")
    with pytest.raises(RuntimeError):
        clk.start(prime=prime)
    assert clk.proc.poll() is not None
