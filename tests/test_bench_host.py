"""Host helpers of bench.py on the CPU: the batch of trial points is the
workload theta and neighbours one step away along a single transformed
coordinate of Sec. 5 (as a simplex would ask for), all admissible; the
whole-job rate divides every rank's units by the slowest rank's time.
bench is imported inside the tests: importing it sets a CUDA environment
variable, which must not leak into the collection of the GPU tests."""
import numpy as np

import oracle


def test_batch_thetas_are_single_coordinate_neighbours():
    import bench
    theta = tuple(bench.WORKLOAD["theta"])
    ths = bench.batch_thetas(theta, 32)
    assert len(ths) == 32 and ths[0] == theta
    x0 = np.array(oracle.untransform(theta))
    for k, th in enumerate(ths[1:]):
        assert all(np.isfinite(th)) and th[0] > 0 and 0 < th[1] <= 20 and th[2] > 0 and th[3] > 0
        dx = np.array(oracle.untransform(th)) - x0
        moved = np.flatnonzero(np.abs(dx) > 1e-9)
        assert list(moved) == [k % 4]
        step = 0.25 * (1 if (k // 4) % 2 == 0 else -1) * (1 + k // 8)
        assert abs(dx[k % 4] - step) < 1e-9
    assert len(set(ths)) == 32


def test_job_rate_uses_the_slowest_rank():
    import bench
    assert bench.job_rate(4, 96, 2000.0) == 4 * 96 / 2.0
