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


def test_oracle_extrapolation_is_exact_for_its_model_and_falls_back_to_cubic():
    import bench
    a, b = 3e-8, 2e-12
    t = lambda m: a * m ** 2 + b * m ** 3
    est, how = bench.extrapolate_seconds(t(8192), t(16384), 16384, 65536)
    assert abs(est - t(65536)) <= 1e-9 * t(65536) and "both sizes" in how
    # pure cubic growth is the model with a = 0
    est, _ = bench.extrapolate_seconds(1.0, 8.0, 16384, 65536)
    assert abs(est - 512.0) < 1e-9
    # times that no a m^2 + b m^3 with a, b >= 0 fits: the larger size, cubed
    for t_half, t_full in ((1.0, 3.0), (1.0, 9.0)):
        est, how = bench.extrapolate_seconds(t_half, t_full, 16384, 65536)
        assert est == t_full * 64.0 and "larger size" in how
