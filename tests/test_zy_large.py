"""The large configuration's size, n = 2,000,000, with an exact reference.

The dense oracle cannot run at this size (32 TB).  On sorted collinear
points the exponential kernel (nu = 1/2 in Eq. 2) is an Ornstein-Uhlenbeck
process, so Eq. 1 has an exact O(n) form: the prediction-error decomposition
of a scalar Kalman filter (oracle.kalman_exponential), and a draw from the
model is an O(n) recursion (oracle.simulate_exponential_line, the Cholesky
factor of the covariance applied to xi).  The H-matrix path runs unchanged on
this degenerate 2-D geometry with the large configuration's options (leaf
128, eta 2, ACA eps 1e-5, rank capacity 48, oversampling 16, theta (0.02,
1/2, 1, 1e-3)), and must reach |dL| / n <= 1e-6 (FP64) against the exact
value; the mixed forms reach q to 1e-6 per point through PCG.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_07146_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 2_000_000
THETA = (0.02, 0.5, 1.0, 1e-3)


@pytest.fixture(scope="module")
def line():
    locs = synth.locations_collinear(N, seed=71)
    Z = oracle.simulate_exponential_line(locs[:, 0], THETA, synth.normal(72, N), synth.normal(73, N))
    ref = oracle.kalman_exponential(locs[:, 0], Z, THETA[0], THETA[2], THETA[3])
    return locs, Z, ref


@pytest.mark.parametrize("precision,bound", [(0, 1e-6), (1, 1e-5)], ids=["fp64", "mixed_fp32"])
def test_two_million_points_on_a_line_match_kalman(hmle_lib, line, precision, bound):
    from paper_2104_07146_gb300 import hmle
    locs, Z, ref = line
    ctx = hmle.Context()
    tree = hmle.Tree(ctx, locs, leaf_size=128, eta=2.0, aca_eps=1e-5, max_rank=48, oversample=16,
                     precision=precision)
    ll, info = tree.loglik(THETA, Z)
    print("n=%d precision %d: L=%.6f ref=%.6f |dL|/n=%.2e q/n=%.4f ranks c/l %d/%d pcg %d"
          % (N, precision, ll, ref, abs(ll - ref) / N, info.quad / N, info.max_rank_c,
             info.max_rank_l, info.pcg_iters))
    assert abs(ll - ref) / N <= bound, (ll, ref)
    # a draw from the model: q / n is chi^2_n / n, 1 +- 5 sqrt(2 / n)
    assert abs(info.quad / N - 1.0) <= 5 * math.sqrt(2.0 / N)
    tree.close()
