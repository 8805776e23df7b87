"""The benchmark's clock sampler, run against a stand-in ``nvidia-smi`` that
writes a fixed CSV log: the median SM clock, the maximum clock and the active
throttle reasons come out of the rows of the benchmarked GPU only."""
import os
import stat
import sys
import time

import bench

ROWS = [
    # index, uuid, sm, max sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    "0, GPU-aaa, 1965, 2032, 700.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, GPU-aaa, 2032, 2032, 650.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, GPU-aaa, 2010, 2032, 690.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "1, GPU-bbb, 1200, 2032, 300.0, 0x0000000000000020, Not Active, Active, Not Active, Not Active",
    "0, GPU-aaa, [N/A], 2032, 640.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
]


def _fake_smi(tmp_path):
    log = "\\n".join(ROWS) + "\\n"
    script = tmp_path / "nvidia-smi"
    script.write_text(f"""#!{sys.executable}
import sys, time
path = sys.argv[sys.argv.index("-f") + 1]
open(path, "w").write("{log}")
time.sleep(60)
""")
    script.chmod(script.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def _sample(tmp_path, monkeypatch, uuid):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(uuid)
    s.start()
    time.sleep(1.0)
    return s.stop()


def test_clock_summary_of_the_benchmarked_gpu(tmp_path, monkeypatch):
    c = _sample(tmp_path, monkeypatch, "GPU-aaa")
    assert c == {"sm_mhz": 2010.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"], "samples": 4}


def test_clock_summary_without_a_uuid_takes_every_row(tmp_path, monkeypatch):
    c = _sample(tmp_path, monkeypatch, None)
    assert c["samples"] == 5 and c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert c["sm_mhz"] == 1987.5  # median of 1965, 2032, 2010, 1200


def test_missing_nvidia_smi_gives_no_clock_record(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(None)
    s.start()
    assert s.stop() is None
