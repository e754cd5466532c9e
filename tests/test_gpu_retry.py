"""Retried evaluations of a multi-instance call (hmle_loglik_multi_retry)
through the C ABI.

A task that fails is evaluated again on a tree derived from its own (same
points and cluster tree, a new plan with other options).  The derived tree
must give exactly the result of a tree built from scratch with those options
(the same kernels, plan and order of sums), and that result must meet the
oracle bound.  Failures are provoked on the host side of the method only: a
rank capacity too small for the requested accuracy (RANK_OVERFLOW), and a
mixed-form PCG limited to one iteration at an unreachable tolerance
(NOT_CONVERGED).
"""
import numpy as np
import pytest

import oracle
from paper_2104_07146_gb300 import synth

pytestmark = pytest.mark.gpu

N = 3000
THETA = (0.1, 0.5, 1.0, 1e-2)


@pytest.fixture(scope="module")
def ctx(hmle_lib):
    from paper_2104_07146_gb300 import hmle
    return hmle.Context()


@pytest.fixture(scope="module")
def field():
    locs = synth.locations_uniform(N, 2, seed=4242)
    Z = synth.normal(4243, N)
    return locs, Z


def _tree(ctx, locs, **kw):
    from paper_2104_07146_gb300 import hmle
    return hmle.Tree(ctx, locs, leaf_size=32, **kw)


def test_rank_overflow_is_retried_at_the_largest_capacity(ctx, field):
    locs, Z = field
    small = _tree(ctx, locs, aca_eps=1e-8, max_rank=8, oversample=8)
    ll0, st0 = ctx.loglik_multi([(small, THETA, Z)])
    assert st0[0] == 5 and ll0[0] == -np.inf          # RANK_OVERFLOW at capacity 8
    ll, st, info = ctx.loglik_multi_retry([(small, THETA, Z), (small, THETA, Z)], max_retries=3)
    assert list(st) == [0, 0]
    assert info[0] == {"retries": 1, "max_rank": 56, "precision": 0, "aca_eps": 1e-8}
    big = _tree(ctx, locs, aca_eps=1e-8, max_rank=56, oversample=8)
    ref, st_ref = ctx.loglik_multi([(big, THETA, Z)])
    assert st_ref[0] == 0
    assert ll[0] == ref[0] and ll[1] == ref[0]
    L = oracle.loglik_dense(locs, Z, THETA)[0]
    assert abs(ll[0] - L) / N <= 1e-6
    # no retries: the plain call
    ll_n, st_n, info_n = ctx.loglik_multi_retry([(small, THETA, Z)], max_retries=0)
    assert st_n[0] == 5 and info_n[0]["retries"] == 0 and info_n[0]["max_rank"] == 8
    small.close()
    big.close()


def test_unconverged_mixed_pcg_is_retried_in_fp64(ctx, field):
    locs, Z = field
    mixed = _tree(ctx, locs, aca_eps=1e-7, precision=1, pcg_tol=1e-15, pcg_max_iter=1)
    _, st0 = ctx.loglik_multi([(mixed, THETA, Z)])
    assert st0[0] == 7                                   # NOT_CONVERGED, reported per task
    ll, st, info = ctx.loglik_multi_retry([(mixed, THETA, Z)], max_retries=1)
    assert st[0] == 0 and info[0]["retries"] == 1 and info[0]["precision"] == 0
    fp64 = _tree(ctx, locs, aca_eps=1e-7)
    ref, _ = ctx.loglik_multi([(fp64, THETA, Z)])
    assert ll[0] == ref[0]
    mixed.close()
    fp64.close()


def test_tasks_that_succeed_are_not_retried(ctx, field):
    locs, Z = field
    t = _tree(ctx, locs, aca_eps=1e-6, max_rank=32, oversample=8)
    ths = [THETA, (0.05, 1.0, 2.0, 1e-3)]
    ll0, st0 = ctx.loglik_multi([(t, th, Z) for th in ths])
    ll, st, info = ctx.loglik_multi_retry([(t, th, Z) for th in ths], max_retries=3)
    assert list(st0) == [0, 0] and list(st) == [0, 0]
    assert np.array_equal(ll, ll0)
    assert all(r["retries"] == 0 and r["max_rank"] == 32 for r in info)
    t.close()


def test_retry_count_is_checked(ctx, field):
    from paper_2104_07146_gb300 import hmle
    locs, Z = field
    t = _tree(ctx, locs)
    with pytest.raises(hmle.HmleError):
        ctx.loglik_multi_retry([(t, THETA, Z)], max_retries=9)
    t.close()
