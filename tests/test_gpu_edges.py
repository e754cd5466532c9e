"""Degenerate and boundary inputs through the C ABI, against the oracle.

- A tree of one leaf (n <= leaf size): the block tree is the single dense
  diagonal block, so the H-Cholesky is the dense Cholesky and L, C^{-1} Z
  and the kriging prediction are exact up to rounding and the Matern
  table's accuracy (1e-13 per entry).
- A two-leaf tree whose blocks are all dense (leaf-level admissible blocks
  stay dense): the same exactness across a leaf boundary.
- The smallest n (2), empty batches, and inputs the library must reject;
  the context stays usable after each rejection.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2104_07146_gb300 import synth

pytestmark = pytest.mark.gpu

TH = (0.2, 0.8, 1.0, 0.05)


@pytest.fixture(scope="module")
def ctx(hmle_lib):
    from paper_2104_07146_gb300 import hmle
    return hmle.Context()


def _tree(ctx, locs, **kw):
    from paper_2104_07146_gb300 import hmle
    return hmle.Tree(ctx, locs, **kw)


def _exact(ctx, locs, leaf, n_leaves):
    n = locs.shape[0]
    Z = synth.normal(900 + n, n)
    t = _tree(ctx, locs, leaf_size=leaf)
    i = t.info()
    assert (i.n_leaves, i.n_lowrank) == (n_leaves, 0)
    ll, info = t.loglik(TH, Z)
    ref, ld, q = oracle.loglik_dense(locs, Z, TH)
    assert abs(info.logdet - ld) <= 1e-9 * n, (info.logdet, ld)
    assert abs(info.quad - q) <= 1e-9 * max(q, 1.0), (info.quad, q)
    assert abs(ll - ref) <= 1e-9 * n, (ll, ref)
    f = t.assemble(TH).factor(Z)
    X = f.solve(Z)
    Xd = np.linalg.solve(oracle.matern_matrix(locs, TH), Z)
    assert np.linalg.norm(X - Xd) <= 1e-9 * np.linalg.norm(Xd)
    locs2 = synth.locations_uniform(7, locs.shape[1], seed=901 + n)
    pred = f.predict(Z, locs2)
    pref = oracle.predict(locs, Z, locs2, TH)
    assert np.abs(pred - pref).max() <= 1e-9 * max(np.abs(pref).max(), 1.0)
    return t


@pytest.mark.parametrize("n,leaf,d", [(2, 16, 2), (40, 64, 2), (128, 128, 3)])
def test_single_leaf_tree_is_the_dense_cholesky(ctx, n, leaf, d):
    locs = synth.locations_uniform(n, d, seed=800 + n)
    _exact(ctx, locs, leaf, 1)


def test_all_dense_two_leaf_tree(ctx):
    # n = 100, leaf 64: two leaves of 50, blocks (0,0), (1,1), (1,0) all dense
    locs = synth.locations_uniform(100, 2, seed=811)
    _exact(ctx, locs, 64, 2)


def test_single_leaf_simulation_has_the_xi_norm(ctx):
    # Z = P^T L P xi  =>  Z^T C^{-1} Z = |xi|^2, with C the dense matrix here
    n = 60
    locs = synth.locations_uniform(n, 2, seed=821)
    xi = synth.normal(822, n)
    Z = _tree(ctx, locs, leaf_size=64).simulate(TH, xi)
    _, _, q = oracle.loglik_dense(locs, Z, TH)
    assert abs(q - xi @ xi) <= 1e-9 * (xi @ xi)


def test_empty_batches_return_at_once(ctx):
    locs = synth.locations_uniform(300, 2, seed=831)
    t = _tree(ctx, locs, leaf_size=32)
    ll, st = t.loglik_batch([], synth.normal(832, 300))
    assert ll.shape == (0,) and st.shape == (0,)
    ll, st = ctx.loglik_multi([])
    assert ll.shape == (0,) and st.shape == (0,)


def _rejects(fn):
    from paper_2104_07146_gb300 import hmle
    with pytest.raises(hmle.HmleError) as e:
        fn()
    assert e.value.status == 1, e.value


def test_invalid_inputs_are_rejected_and_the_context_stays_usable(ctx):
    ok = synth.locations_uniform(200, 2, seed=841)
    _rejects(lambda: _tree(ctx, ok[:1]))                               # n = 1
    _rejects(lambda: _tree(ctx, synth.locations_uniform(50, 1, seed=842)))   # d = 1
    _rejects(lambda: _tree(ctx, synth.locations_uniform(50, 4, seed=843)))   # d = 4
    bad = ok.copy()
    bad[17, 1] = math.nan
    _rejects(lambda: _tree(ctx, bad))                                  # non-finite point
    bad[17, 1] = math.inf
    _rejects(lambda: _tree(ctx, bad))
    _rejects(lambda: _tree(ctx, ok, leaf_size=24))                     # not a multiple of 16
    _rejects(lambda: _tree(ctx, ok, leaf_size=256))
    _rejects(lambda: _tree(ctx, ok, aca_eps=0.0))
    _rejects(lambda: _tree(ctx, ok, max_rank=64, oversample=8))        # capacity above 64
    t = _tree(ctx, ok, leaf_size=32)
    Z = synth.normal(844, 200)
    _rejects(lambda: t.loglik((0.0, 0.5, 1.0, 0.01), Z))               # ell = 0
    _rejects(lambda: t.loglik((0.1, 21.0, 1.0, 0.01), Z))              # nu > 20
    _rejects(lambda: t.loglik((0.1, 0.5, -1.0, 0.01), Z))              # sigma2 < 0
    _rejects(lambda: t.loglik((0.1, 0.5, 1.0, math.nan), Z))
    f = t.assemble(TH).factor(Z)
    _rejects(lambda: f.predict(Z, np.zeros((0, 2))))                   # m = 0
    ll, _ = t.loglik(TH, Z)
    ref, _, _ = oracle.loglik_dense(ok, Z, TH)
    assert abs(ll - ref) / 200 <= 1e-6


def test_phase_work_of_a_single_leaf(ctx):
    # one dense diagonal block of m = n points: n^2 Matern entries of
    # 3d + 68 flops, and a solve reads its lower triangle once per sweep
    n = 40
    locs = synth.locations_uniform(n, 2, seed=851)
    Z = synth.normal(852, n)
    f = _tree(ctx, locs, leaf_size=64).assemble(TH).factor(Z)
    fa, sb = f.phase_work()
    assert fa == n * n * (3 * 2 + 68)
    assert sb == 2 * 8 * n * (n + 1) / 2
