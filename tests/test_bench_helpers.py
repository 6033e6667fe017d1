"""Host-side helpers of the benchmark on CPU: the recorded DRAM traffic is
used only while the kernel source it was captured on is unchanged, and the
clock record summarises nvidia-smi samples of this GPU under load (median
SM clock, maximum clock, every throttle reason seen)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_recorded_traffic_follows_the_kernel_source(tmp_path):
    note = tmp_path / "summary.md"
    note.write_text(f"text\ntraffic_bytes_per_launch: 1.5e9 source_hash: {bench.kernel_source_hash()}\n")
    assert bench.recorded_traffic(str(note)) == 1.5e9
    note.write_text("traffic_bytes_per_launch: 1.5e9 source_hash: 0123456789ab\n")
    assert bench.recorded_traffic(str(note)) is None            # taken on another source
    note.write_text("no record here\n")
    assert bench.recorded_traffic(str(note)) is None
    assert bench.recorded_traffic(str(tmp_path / "missing.md")) is None
    # the committed summary carries a record in the expected form
    with open(bench.PROFILE_NOTE) as f:
        assert "traffic_bytes_per_launch:" in f.read()


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_summary():
    s = bench.ClockSampler("GPU-aaaa")
    s.file.write(
        "0, GPU-aaaa, 2032, 2032, 900.5, 0x0, Not Active, Not Active, Not Active, Active\n"
        "0, GPU-aaaa, 1900, 2032, 1000.0, 0x8, Active, Not Active, Not Active, Not Active\n"
        "0, GPU-aaaa, 2010, 2032, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "1, GPU-bbbb, 800, 2032, 900.0, 0x0, Active, Active, Active, Active\n"      # another GPU
        "0, GPU-aaaa, 345, 2032, 80.0, 0x0, Not Active, Active, Not Active, Not Active\n"  # idle
        "garbage line\n")
    s.proc = _Proc()
    out = s.stop()
    assert out == dict(sm_mhz=2010.0, sm_max_mhz=2032.0, reasons=["hw_slowdown", "sw_power_cap"], samples=3)
    assert not os.path.exists(s.file.name)


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler("")
    assert s.stop() is None                                       # never started
    os.unlink(s.file.name)
