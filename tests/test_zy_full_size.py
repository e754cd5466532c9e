"""A property that holds at any size, checked on the benchmark's own workload
(n = 65,536: 70% uniform + 30% in 8 blobs, leaf 64, eta 2, ACA eps 1e-6) in
the batched launch configuration that bench.py times.

Scaling sigma2 and tau2 by 4 multiplies C by 4 (Eq. 2).  Every decision of
the method is relative (ACA pivots and stopping rule, the pivoted QR, the
Jacobi rotations, the truncation threshold) and a factor of 4 is exact in
binary floating point, so C~ scales by exactly 4 and L~ by 2.  Eq. 1 then
gives log|4 C~| = log|C~| + n log 4 and Z^T (4 C~)^{-1} Z = q / 4, which
checks log|C~| and q separately at full size, where the dense oracle does
not run.
"""
import math

import pytest

from paper_2104_07146_gb300 import synth

pytestmark = pytest.mark.gpu


def test_scaling_invariant_on_the_benchmark_workload(hmle_lib):
    from paper_2104_07146_gb300 import hmle
    n = 65536
    locs = synth.locations_blobs(n, 2, 0.3, 8, 0.03, seed=1001)    # the benchmark's inputs
    Z = synth.normal(1002, n)
    ctx = hmle.Context()
    tree = hmle.Tree(ctx, locs, leaf_size=64, eta=2.0, aca_eps=1e-6)
    th = (0.05, 0.5, 1.0, 1e-3)
    th4 = (th[0], th[1], 4.0 * th[2], 4.0 * th[3])
    ll, st = tree.loglik_batch([th, th4], Z, concurrency=2)
    assert [int(s) for s in st] == [0, 0]
    l1, i1 = tree.loglik(th, Z)
    l4, i4 = tree.loglik(th4, Z)
    # the batched evaluations are the single ones
    assert abs(ll[0] - l1) <= 1e-12 * abs(l1) and abs(ll[1] - l4) <= 1e-12 * abs(l4)
    assert abs(i4.logdet - (i1.logdet + n * math.log(4.0))) <= 1e-10 * n
    assert abs(i4.quad - i1.quad / 4.0) <= 1e-12 * i1.quad
    expect = l1 - 0.5 * n * math.log(4.0) - 0.5 * i1.quad * (0.25 - 1.0)
    assert abs(l4 - expect) <= 1e-9 * n
    assert (i4.max_rank_c, i4.max_rank_l) == (i1.max_rank_c, i1.max_rank_l)
    tree.close()
