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
