"""Host logic of bench.py without a GPU: the clock record that decides
whether a timed run saw a throttling reason (NVML reason bits, or the
nvidia-smi CSV fallback), fed by fakes; nothing here queries or changes a
GPU."""
import os

import pytest


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


class _FakeNvml:
    sm_max = 2070.0

    def __init__(self, samples):
        self.s = list(samples)

    def sample(self):
        return self.s.pop(0) if self.s else None


def test_nvml_reasons_and_clocks(bench):
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.nvml = _FakeNvml([])
    cs.samples = [(2070.0, 0x0, 150.0), (1980.0, 0x4, 900.0), (2070.0, 0x4 | 0x40, 1200.0)]
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_min_mhz"] == 1980.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert s["power_w_max"] == 1200.0 and s["samples"] == 3
    cs.samples = [(2070.0, 0x8, 100.0)]
    assert cs.summary()["reasons"] == ["hw_slowdown"]
    cs.samples = []
    assert cs.summary()["reasons"] == ["unsampled"]


def test_nvml_sampling_thread(bench):
    """__enter__/__exit__ take a first and a last sample around the polling."""
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.nvml = _FakeNvml([(2070.0, 0, 100.0)] * 5)
    cs.period = 0.001
    with cs:
        pass
    assert 2 <= len(cs.samples) <= 5
    assert cs.summary()["reasons"] == []


def test_nvidia_smi_csv_fallback(bench, tmp_path):
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.nvml = None
    cs.proc = object()
    cs.path = os.path.join(tmp_path, "clocks.csv")
    with open(cs.path, "w") as f:
        f.write("0, 2070, 2070, 500.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1500, 2070, 900.0, 0x4, Not Active, Not Active, Active, Active\n")
        f.write("garbage line\n")
        f.write("0, 2070, 2070, 800.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]
