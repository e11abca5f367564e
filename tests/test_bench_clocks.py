"""bench.py's clock sampler on CPU, against a stand-in nvidia-smi on PATH that prints
the query's CSV lines every 20 ms: only the samples taken between start() and stop()
are reported (the median SM clock, the maximum clock, the throttle reasons seen), and
a region shorter than the sampling interval reports the sample taken just before it
with samples = 0."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FAKE = """#!{py}
import sys, time
lines = {lines!r}
i = 0
while True:
    sys.stdout.write(lines[min(i, len(lines) - 1)] + "\\n")
    sys.stdout.flush()
    i += 1
    time.sleep({period})
"""


def install_fake(tmp_path, monkeypatch, lines, period):
    exe = tmp_path / "nvidia-smi"
    exe.write_text(FAKE.format(py=sys.executable, lines=lines, period=period))
    exe.chmod(exe.stat().st_mode | stat.S_IXUSR)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))


def sampler():
    sys.path.insert(0, ROOT)
    import bench
    return bench.ClockSampler(0)


def row(mhz, power_cap="Not Active", thermal="Not Active"):
    return "0, %d, 2070, 900.0, 0x0, Not Active, Not Active, %s, %s" % (mhz, thermal, power_cap)


def test_samples_inside_the_region_only(tmp_path, monkeypatch):
    # the first line (a low clock) is printed before start() returns and is not reported
    lines = [row(600)] + [row(2070)] * 3 + [row(1980, power_cap="Active")] * 200
    install_fake(tmp_path, monkeypatch, lines, 0.02)
    s = sampler()
    s.start()
    time.sleep(0.3)
    c = s.stop()
    assert c["samples"] >= 5
    assert c["sm_max_mhz"] == 2070.0 and c["sm_mhz"] in (1980.0, 2070.0)
    assert c["reasons"] == ["sw_power_cap"]


def test_short_region_reports_the_sample_before_it(tmp_path, monkeypatch):
    install_fake(tmp_path, monkeypatch, [row(2070, thermal="Active")], 5.0)
    s = sampler()
    s.start()
    c = s.stop()
    assert c["samples"] == 0
    assert c["sm_mhz"] == 2070.0 and c["reasons"] == ["sw_thermal_slowdown"]


def test_missing_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = sampler()
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
