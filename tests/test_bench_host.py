"""Host logic of bench.py that needs no GPU: reading nvidia-smi clock samples
for the right device, and the throttle reasons that make a run invalid."""
import bench

LINES = """0, 2070, 2070, 950.1, 0x0, Not Active, Not Active, Not Active, Not Active
3, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active
0, 2055, 2070, 955.0, 0x0, Not Active, Not Active, Not Active, Not Active
3, 1965, 2070, 1399.0, 0x4, Not Active, Not Active, Not Active, Active
3, 1950, 2070, 1400.0, 0x8, Not Active, Active, Not Active, Active
garbage line
"""


def test_clocks_of_the_device_in_use(monkeypatch):
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES", raising=False)
    c = bench._parse_clocks(LINES, 0)
    assert c == {"sm_mhz": 2062.5, "sm_max_mhz": 2070.0, "samples": 2, "reasons": []}
    c = bench._parse_clocks(LINES, 3)
    assert c["samples"] == 3 and c["sm_mhz"] == 1965.0
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clocks_follow_cuda_visible_devices(monkeypatch):
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "3,0")
    assert bench._parse_clocks(LINES, 0)["samples"] == 3      # CUDA device 0 is GPU 3
    assert bench._parse_clocks(LINES, 1)["samples"] == 2
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "GPU-1234abcd")
    only3 = "\n".join(l for l in LINES.splitlines() if l.startswith("3,"))
    assert bench._parse_clocks(only3, 0)["samples"] == 3      # the one GPU sampled
    assert bench._parse_clocks("", 0) is None
