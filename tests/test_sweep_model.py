"""The factorisation schedule, executed by a numpy interpreter
(tests/sweep_model.py), reproduces the H-Cholesky factor of Sec. 2 on the
CPU: L~ L~^T matches C to the truncation accuracy, and log|C~| and
Z^T C~^{-1} Z (the right-hand side carried through the W-panels as the root
panel) match the dense oracle at the contract bound |delta| / n <= 1e-6.
This checks the planner's lists as a computation (targets, pairs, panel
solves and deferred updates in their order), independently of the kernels.
"""
import numpy as np
import pytest

import oracle
import sweep_model
from paper_2104_07146_gb300 import synth


@pytest.mark.parametrize("n,d,leaf,theta,geometry", [
    (1200, 2, 32, (0.1, 0.8, 1.0, 0.01), "uniform"),
    (900, 2, 16, (0.05, 0.5, 1.0, 1e-3), "blobs"),
    (700, 3, 32, (0.2, 1.3, 1.5, 0.02), "uniform"),
])
def test_schedule_computes_the_h_cholesky_factor(n, d, leaf, theta, geometry):
    if geometry == "blobs":
        locs = synth.locations_blobs(n, d, 0.3, 8, 0.03, seed=31)
    else:
        locs = synth.locations_uniform(n, d, seed=32)
    Z = synth.normal(33, n)
    ld, q, L, C, perm, nlr, kmax = sweep_model.execute(locs, Z, theta, leaf=leaf, eps=1e-9)
    assert nlr > 0 and kmax <= 48                 # the low-rank machinery was exercised
    _, ld0, q0 = oracle.loglik_from_matrix(C, Z[perm])
    assert abs(ld - ld0) / n <= 1e-6, (ld, ld0)
    assert abs(q - q0) / n <= 1e-6, (q, q0)
    assert np.linalg.norm(L @ L.T - C) <= 1e-7 * np.linalg.norm(C)
    # the schedule's forward solve is L~^{-1} P Z itself
    w = np.linalg.solve(L, Z[perm])
    assert abs(w @ w - q) <= 1e-9 * q


@pytest.mark.parametrize("n,d,leaf,theta,geometry", [
    (1200, 2, 32, (0.1, 0.8, 1.0, 0.01), "uniform"),
    (900, 2, 16, (0.05, 0.5, 1.0, 1e-3), "blobs"),
])
def test_ldlt_form_on_the_same_schedule(n, d, leaf, theta, geometry):
    # Sec. 2's factorisation without square roots run on the same lists: the
    # blocks held as M = L D and every product over a column index weighted
    # by 1 / d.  It must give the dense oracle's log|C| and q, and its
    # L D^(1/2) must be the H-Cholesky factor of the L L^T form (the same
    # truncations, so the same factor up to rounding).
    if geometry == "blobs":
        locs = synth.locations_blobs(n, d, 0.3, 8, 0.03, seed=31)
    else:
        locs = synth.locations_uniform(n, d, seed=32)
    Z = synth.normal(33, n)
    ld, q, L, C, perm, nlr, _ = sweep_model.execute(locs, Z, theta, leaf=leaf, eps=1e-9, form="ldlt")
    assert nlr > 0
    _, ld0, q0 = oracle.loglik_from_matrix(C, Z[perm])
    assert abs(ld - ld0) / n <= 1e-6, (ld, ld0)
    assert abs(q - q0) / n <= 1e-6, (q, q0)
    assert np.linalg.norm(L @ L.T - C) <= 1e-7 * np.linalg.norm(C)
    ld1, q1, L1, *_ = sweep_model.execute(locs, Z, theta, leaf=leaf, eps=1e-9, form="llt")
    assert abs(ld - ld1) <= 1e-9 * n and abs(q - q1) <= 1e-9 * q1
    assert np.linalg.norm(L - L1) <= 1e-6 * np.linalg.norm(L1)
