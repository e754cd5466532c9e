"""Planted mistakes in the oracle (on the CPU) must be caught by the pins.

Each case rebuilds one step of Eq. 1 / Eq. 2 with a plausible error and
checks that the pin used in test_oracle_pins rejects it.
"""
import math

import numpy as np

import oracle
from paper_2104_07146_gb300 import synth

LOG2PI = math.log(2 * math.pi)


def _ll(C, Z, drop_2pi=False, logdet_sign=-0.5, transpose=False):
    n = C.shape[0]
    L = np.linalg.cholesky(C)
    logdet = 2 * np.sum(np.log(np.diag(L)))
    w = oracle.forward_solve(L.T.copy() if transpose else L, Z)
    q = float(w @ w)
    return (0 if drop_2pi else -0.5 * n * LOG2PI) + logdet_sign * logdet - 0.5 * q


def test_dropped_2pi_term_fails_nugget_pin():
    n, t2 = 40, 0.3
    Z = synth.normal(1, n)
    C = t2 * np.eye(n)
    ref = -0.5 * n * LOG2PI - 0.5 * n * math.log(t2) - float(Z @ Z) / (2 * t2)
    assert abs(_ll(C, Z) - ref) < 1e-10
    assert abs(_ll(C, Z, drop_2pi=True) - ref) > 1.0


def test_wrong_logdet_sign_fails_scaling_pin():
    n = 80
    locs = synth.locations_uniform(n, 2, seed=2)
    Z = synth.normal(3, n)
    C = oracle.matern_matrix(locs, (0.2, 0.9, 1.0, 0.05))
    c = 2.5
    good = _ll(c * C, Z) - _ll(C, Z)
    bad = _ll(c * C, Z, logdet_sign=0.5) - _ll(C, Z, logdet_sign=0.5)
    q = float(np.linalg.solve(C, Z) @ Z)
    expect = -0.5 * n * math.log(c) - 0.5 * q * (1 / c - 1)
    assert abs(good - expect) < 1e-9 * abs(expect) + 1e-9
    assert abs(bad - expect) > 1.0


def test_transposed_factor_fails_kalman_pin():
    n = 200
    locs = synth.locations_collinear(n, seed=4)
    Z = synth.normal(5, n)
    C = oracle.matern_matrix(locs, (0.1, 0.5, 1.0, 0.01))
    ok = _ll(C, Z)
    bad = _ll(C, Z, transpose=True)
    assert abs(ok - bad) > 1.0


def test_sqrt2nu_scaling_fails_half_integer_pin():
    # the sqrt(2 nu) h / ell convention is a different parameterisation than
    # Eq. 2; at nu = 1.5 it does not give (1 + x) e^{-x}
    x = 0.7
    alt = oracle.matern_unit(1.5, math.sqrt(3.0) * x)
    assert abs(alt - (1 + x) * math.exp(-x)) > 1e-2


def _ll_ldlt(C, Z, drop_d=False, sqrt_d=False):
    # Eq. 1 through C = L D L^T with a planted mistake: q without the 1/d_i
    # weights, or log|C| from sqrt(d_i) as if d held Cholesky diagonals
    n = C.shape[0]
    L, d = oracle.ldlt(C)
    w = np.linalg.solve(L, Z)
    q = float(np.sum(w * w) if drop_d else np.sum(w * w / d))
    logdet = float(np.sum(np.log(np.sqrt(d)) if sqrt_d else np.log(d)))
    return -0.5 * n * LOG2PI - 0.5 * logdet - 0.5 * q


def test_ldlt_mistakes_fail_nugget_and_cholesky_pins():
    n, t2 = 40, 0.3
    Z = synth.normal(6, n)
    ref = -0.5 * n * LOG2PI - 0.5 * n * math.log(t2) - float(Z @ Z) / (2 * t2)
    assert abs(_ll_ldlt(t2 * np.eye(n), Z) - ref) < 1e-10
    assert abs(_ll_ldlt(t2 * np.eye(n), Z, drop_d=True) - ref) > 1.0
    locs = synth.locations_uniform(60, 2, seed=7)
    C = oracle.matern_matrix(locs, (0.2, 0.9, 1.0, 0.05))
    Z = synth.normal(8, 60)
    good = oracle.loglik_from_matrix(C, Z)[0]
    assert abs(_ll_ldlt(C, Z) - good) < 1e-9 * abs(good)
    assert abs(_ll_ldlt(C, Z, sqrt_d=True) - good) > 1.0


def test_prediction_error_mistakes_fail_the_joint_covariance_pin():
    # Eq. 5-6: a flipped sign of the cross term, or the approximated model's
    # covariance in the quadratic term, changes E_t[(Z_a - Z)^2] away from
    # the variance w^T J_t w of the predictor's error
    rng = np.random.default_rng(22)
    locs1 = rng.uniform(size=(60, 2))
    s = rng.uniform(size=(1, 2))
    tht, tha = (0.15, 0.8, 1.0, 0.02), (0.25, 1.4, 1.5, 0.05)
    n = len(locs1)
    Jt = oracle.matern_matrix(np.vstack([locs1, s]), tht)
    Ja = oracle.matern_matrix(np.vstack([locs1, s]), tha)
    ct, ca = Jt[:n, n], Ja[:n, n]
    la = np.linalg.solve(Ja[:n, :n], ca)
    vt = tht[2] + tht[3]
    w = np.append(la, -1.0)
    ref = w @ Jt @ w
    good = vt - 2.0 * la @ ct + la @ Jt[:n, :n] @ la
    flipped = vt + 2.0 * la @ ct + la @ Jt[:n, :n] @ la
    wrong_c = vt - 2.0 * la @ ct + la @ Ja[:n, :n] @ la
    assert abs(good - ref) <= 1e-10 * vt
    assert abs(flipped - ref) > 1e-3 * vt
    assert abs(wrong_c - ref) > 1e-3 * vt
