"""The benchmark's CPU legs run the oracle unchanged: on one core, and as one spawned
replica per core behind a start barrier.  Checked on a small lattice with two replicas:
the aggregate rate is the replicas' flops over the common wall time."""
import pytest


def test_oracle_replicas_report_aggregate_rate():
    import bench
    dims, ns = (4, 4, 2, 4), 4
    gf, wall, cores = bench.oracle_on_all_cores(dims, ns, warmup=0, reps=2, cores=2)
    assert cores == 2 and wall > 0
    n = dims[0] * dims[1] * dims[2] * dims[3] // 2 * ns
    assert gf == pytest.approx(2 * 2 * bench.flops_ccdag(n, ns) / wall / 1e9)


def test_host_cores_is_positive():
    import bench
    assert bench.host_cores() >= 1


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_reports_median_clock_and_active_reasons():
    """The clocks object of the bench line: median SM clock under load, the maximum, and
    every throttle reason seen active in any sample (nvidia-smi csv, noheader, nounits)."""
    import bench
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = ["0, 2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "0, 2055, 2070, 1398.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
               "garbage line", ""]
    c = s.stop()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    s.lines.append("0, 1500, 2070, 700.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active")
    assert "hw_slowdown" in s.stop()["reasons"]


def test_clock_sampler_without_nvidia_smi():
    import bench
    c = bench.ClockSampler(0).stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]
