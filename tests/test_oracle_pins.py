"""Pins of the CPU oracle against facts fixed by mathematics and the paper.

None of these re-derive the oracle's own formula: closed forms of
half-integer Bessel functions, the recurrence and Wronskian of K_nu, brute
force determinants, the exact O(n) likelihood of the exponential kernel on a
line (Kalman filter), invariances of Eq. 1, and Nelder-Mead on functions
with known minima.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2104_07146_gb300 import synth

XS = np.logspace(-6, 2.5, 41)
HALF_PI = math.pi / 2.0


# --- K_nu and the Matern function (Eq. 2) ------------------------------------

@pytest.mark.parametrize("nu,poly", [
    (0.5, lambda x: 1.0),
    (1.5, lambda x: 1.0 + 1.0 / x),
    (2.5, lambda x: 1.0 + 3.0 / x + 3.0 / (x * x)),
])
def test_besselk_half_integer_closed_forms(nu, poly):
    # K_{n+1/2}(x) = sqrt(pi/(2x)) e^{-x} * (finite polynomial in 1/x)
    for x in XS:
        ref = math.sqrt(HALF_PI / x) * poly(x)          # e^x K_nu(x)
        got = oracle.besselk_scaled(nu, x)
        assert abs(got - ref) <= 1e-13 * ref, (nu, x, got, ref)


@pytest.mark.parametrize("nu,f", [
    (0.5, lambda x: math.exp(-x)),
    (1.5, lambda x: (1.0 + x) * math.exp(-x)),
    (2.5, lambda x: (1.0 + x + x * x / 3.0) * math.exp(-x)),
])
def test_matern_half_integer_closed_forms(nu, f):
    for x in np.concatenate([XS, [0.0]]):
        ref = f(x)
        got = oracle.matern_unit(nu, x)
        assert abs(got - ref) <= 1e-13 * max(ref, 1e-300) + 1e-300, (nu, x, got, ref)


@pytest.mark.parametrize("nu", [0.3, 0.8, 1.3, 2.2])
def test_besselk_recurrence(nu):
    # K_{nu+1}(x) = K_{nu-1}(x) + (2 nu / x) K_nu(x), with K_{-mu} = K_mu
    for x in np.logspace(-3, 2, 21):
        lhs = oracle.besselk_scaled(nu + 1, x)
        rhs = oracle.besselk_scaled(abs(nu - 1), x) + 2 * nu / x * oracle.besselk_scaled(nu, x)
        assert abs(lhs - rhs) <= 1e-13 * lhs, (nu, x)


def _besseli(nu, x, terms=200):
    s, k = 0.0, 0
    while k < terms:
        s += math.exp((2 * k + nu) * math.log(x / 2) - math.lgamma(k + 1) - math.lgamma(k + nu + 1))
        k += 1
    return s


@pytest.mark.parametrize("nu", [0.3, 0.75, 1.6, 2.4])
def test_besselk_wronskian(nu):
    # I_nu K_{nu+1} + I_{nu+1} K_nu = 1/x  (power series for I in the test)
    for x in [0.05, 0.3, 1.0, 3.0, 8.0, 15.0]:
        k0 = oracle.besselk(nu, x)
        k1 = oracle.besselk(nu + 1, x)
        w = _besseli(nu, x) * k1 + _besseli(nu + 1, x) * k0
        assert abs(w * x - 1.0) <= 1e-12, (nu, x, w * x)


@pytest.mark.parametrize("nu", [0.3, 0.5, 1.0, 2.5])
def test_matern_origin_limit(nu):
    # x^nu K_nu(x) -> 2^(nu-1) Gamma(nu): M_nu(x) -> 1 continuously at 0
    assert oracle.matern_unit(nu, 0.0) == 1.0
    assert abs(oracle.matern_unit(nu, 1e-14) - 1.0) < 1e-6
    vals = [oracle.matern_unit(nu, x) for x in np.logspace(-4, 1.5, 30)]
    assert all(a > b for a, b in zip(vals, vals[1:]))          # strictly decreasing


def test_besselk_against_library():
    special = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(7)
    for _ in range(60):
        nu = rng.uniform(0.3, 2.5)
        x = 10 ** rng.uniform(-4, 2)
        ref = special.kve(nu, x)
        assert abs(oracle.besselk_scaled(nu, x) - ref) <= 1e-12 * ref


# --- dense log-likelihood (Eq. 1) -------------------------------------------

LOG2PI = math.log(2.0 * math.pi)


def test_loglik_nugget_only_closed_form():
    # sigma^2 = 0: C = tau^2 I, L = -n/2 log 2pi - n/2 log tau^2 - Z.Z/(2 tau^2)
    n = 60
    locs = synth.locations_uniform(n, 2, seed=3)
    Z = synth.normal(4, n)
    t2 = 0.37
    ll, logdet, q = oracle.loglik_dense(locs, Z, (0.1, 0.7, 0.0, t2))
    ref = -0.5 * n * LOG2PI - 0.5 * n * math.log(t2) - float(Z @ Z) / (2 * t2)
    assert abs(ll - ref) <= 1e-12 * abs(ref)
    assert abs(logdet - n * math.log(t2)) <= 1e-12 * n


def _leibniz_det(A):
    n = A.shape[0]
    tot = 0.0
    for p in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        prod = 1.0
        for i in range(n):
            prod *= A[i, p[i]]
        tot += -prod if inv % 2 else prod
    return tot


@pytest.mark.parametrize("n,theta", [(3, (0.3, 0.9, 1.2, 0.05)), (8, (0.2, 1.7, 0.8, 0.01))])
def test_loglik_brute_force(n, theta):
    locs = synth.locations_uniform(n, 2, seed=10 + n)
    Z = synth.normal(20 + n, n)
    C = oracle.matern_matrix(locs, theta)
    det = _leibniz_det(C)
    # Cramer's rule: x_i = det(C with column i replaced by Z) / det(C)
    x = np.empty(n)
    for i in range(n):
        Ci = C.copy()
        Ci[:, i] = Z
        x[i] = _leibniz_det(Ci) / det
    ref = -0.5 * n * LOG2PI - 0.5 * math.log(det) - 0.5 * float(Z @ x)
    ll, logdet, q = oracle.loglik_dense(locs, Z, theta)
    assert abs(logdet - math.log(det)) <= 1e-10 * max(1.0, abs(logdet))
    assert abs(q - float(Z @ x)) <= 1e-9 * abs(q)
    assert abs(ll - ref) <= 1e-10 * abs(ref)


def test_loglik_scaling_invariant():
    # C(c sigma2, c tau2) = c C  =>  logdet += n log c, q /= c
    n = 300
    locs = synth.locations_uniform(n, 2, seed=5)
    Z = synth.normal(6, n)
    th = (0.15, 1.2, 1.3, 0.02)
    c = 3.7
    ll, ld, q = oracle.loglik_dense(locs, Z, th)
    ll2, ld2, q2 = oracle.loglik_dense(locs, Z, (th[0], th[1], c * th[2], c * th[3]))
    assert abs(ld2 - (ld + n * math.log(c))) <= 1e-11 * n
    assert abs(q2 - q / c) <= 1e-11 * q
    assert abs(ll2 - (ll - 0.5 * n * math.log(c) - 0.5 * q * (1 / c - 1))) <= 1e-10 * abs(ll)


def test_loglik_permutation_invariant():
    n = 400
    locs = synth.locations_uniform(n, 2, seed=8)
    Z = synth.normal(9, n)
    th = (0.1, 0.8, 1.0, 0.01)
    p = np.argsort(synth.uniform(11, n))
    a = oracle.loglik_dense(locs, Z, th)
    b = oracle.loglik_dense(locs[p], Z[p], th)
    for u, v in zip(a, b):
        assert abs(u - v) <= 1e-10 * max(1.0, abs(u))


@pytest.mark.parametrize("t2", [0.0, 1e-3, 0.05])
def test_loglik_exponential_on_a_line_matches_kalman(t2):
    n = 700
    locs = synth.locations_collinear(n, seed=12)
    Z = synth.normal(13, n)
    ell, s2 = 0.07, 1.4
    ll, _, _ = oracle.loglik_dense(locs, Z, (ell, 0.5, s2, t2))
    ref = oracle.kalman_exponential(locs[:, 0], Z, ell, s2, t2)
    assert abs(ll - ref) <= 1e-9 * abs(ref), (ll, ref)


def test_exponential_line_simulation_is_the_cholesky_factor():
    """The O(n) Ornstein-Uhlenbeck recursion without nugget is L xi with L
    the dense Cholesky factor of the exponential covariance on sorted points;
    the nugget then adds tau eta."""
    n = 300
    locs = synth.locations_collinear(n, seed=14)
    xi, eta = synth.normal(15, n), synth.normal(16, n)
    th = (0.05, 0.5, 1.7, 0.0)
    u = oracle.simulate_exponential_line(locs[:, 0], th, xi, eta)
    assert np.max(np.abs(u - oracle.simulate(locs, th, xi))) <= 1e-11
    th2 = (0.05, 0.5, 1.7, 0.02)
    z = oracle.simulate_exponential_line(locs[:, 0], th2, xi, eta)
    assert np.max(np.abs(z - u - math.sqrt(0.02) * eta)) <= 1e-14


def test_loglik_tiny_range_is_white_noise():
    # ell -> 0 with distinct points: C -> (sigma2 + tau2) I
    n = 200
    locs = synth.locations_uniform(n, 2, seed=14)
    Z = synth.normal(15, n)
    s2, t2 = 0.8, 0.2
    ll, _, _ = oracle.loglik_dense(locs, Z, (1e-9, 1.0, s2, t2))
    v = s2 + t2
    ref = -0.5 * n * LOG2PI - 0.5 * n * math.log(v) - float(Z @ Z) / (2 * v)
    assert abs(ll - ref) <= 1e-12 * abs(ref)


def test_loglik_rejects_non_spd():
    # two coincident points with tau2 = 0 make C singular
    locs = np.array([[0.2, 0.3], [0.2, 0.3], [0.7, 0.1]])
    with pytest.raises(np.linalg.LinAlgError):
        oracle.loglik_dense(locs, np.ones(3), (0.3, 0.5, 1.0, 0.0))


def test_simulated_field_quadratic_form_is_chi2():
    # Z = L xi  =>  Z^T C^{-1} Z = |xi|^2 ~ chi^2_n
    n = 1500
    locs = synth.locations_uniform(n, 2, seed=16)
    th = (0.1, 0.5, 1.0, 0.01)
    xi = synth.normal(17, n)
    Z = oracle.simulate(locs, th, xi)
    _, _, q = oracle.loglik_dense(locs, Z, th)
    assert abs(q - float(xi @ xi)) <= 1e-8 * q
    assert abs(q / n - 1.0) <= 5 * math.sqrt(2.0 / n)


# --- transform and Nelder-Mead ----------------------------------------------

def test_transform_golden_start_point():
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "transform_start.json")))
    ell, nu, s2, t2 = oracle.transform(g["x0"])
    assert abs(math.sqrt(s2) - g["sigma"]) <= 1e-15
    assert abs(ell - g["ell"]) <= 1e-15
    assert abs(nu - g["nu"]) <= 1e-15
    assert abs(math.sqrt(t2) - g["tau"]) <= 1e-20


def test_transform_roundtrip():
    for th in [(0.2, 1.0, 0.5, 0.05), (0.01, 2.4, 3.0, 1e-9), (0.5, 0.31, 0.1, 0.3)]:
        back = oracle.transform(oracle.untransform(th))
        for a, b in zip(th, back):
            assert abs(a - b) <= 1e-13 * a


def test_nelder_mead_quadratic():
    c = np.array([1.0, -2.0, 0.5, 3.0])
    w = np.array([1.0, 4.0, 0.5, 2.0])
    f = lambda x: float(np.sum(w * (x - c) ** 2))
    x, fx, it, nev = oracle.nelder_mead(f, np.zeros(4), 1.0, 1e-14, 1e-8, 5000)
    assert np.max(np.abs(x - c)) < 1e-6 and fx < 1e-12


def test_nelder_mead_rosenbrock():
    f = lambda x: 100.0 * (x[1] - x[0] ** 2) ** 2 + (1 - x[0]) ** 2
    x, fx, it, nev = oracle.nelder_mead(f, np.array([-1.2, 1.0]), 0.5, 1e-14, 1e-10, 5000)
    assert np.max(np.abs(x - 1.0)) < 1e-5


def test_nelder_mead_iteration_cap():
    f = lambda x: float(np.sum(x ** 2))
    _, _, it, _ = oracle.nelder_mead(f, np.full(3, 50.0), 1.0, 0.0, 0.0, 17)
    assert it == 17


@pytest.mark.slow
def test_fit_recovers_simulated_theta():
    n = 500
    locs = synth.locations_uniform(n, 2, seed=18)
    th = (0.1, 0.5, 1.0, 0.01)
    Z = oracle.simulate(locs, th, synth.normal(19, n))
    th_hat, ll_hat, it, nev = oracle.fit(locs, Z, (0.2, 1.0, 0.5, 0.05), max_iter=400)
    ll_true = oracle.loglik_dense(locs, Z, th)[0]
    assert ll_hat >= ll_true - 1e-3          # the MLE is at least as likely as the truth
    assert 0.03 < th_hat[0] < 0.3 and 0.2 < th_hat[1] < 1.2 and 0.3 < th_hat[2] < 3.0


def test_prediction_interpolates_without_nugget():
    # Eq. 4 with tau2 = 0: a training location's own row of C21 is its row of
    # C11, so the prediction there returns the observed value exactly
    rng = np.random.default_rng(3)
    locs = rng.uniform(size=(40, 2))
    Z = rng.normal(size=40)
    th = (0.3, 1.5, 1.2, 0.0)
    pred = oracle.predict(locs, Z, locs[[3, 17, 31]], th)
    assert np.allclose(pred, Z[[3, 17, 31]], rtol=0, atol=1e-8)


def test_prediction_single_point_closed_form():
    # one training point: Z2 = sigma2 M(h/ell) / (sigma2 + tau2) * Z1
    th = (0.5, 0.5, 2.0, 0.5)
    z = np.array([1.7])
    p = oracle.predict(np.array([[0.0, 0.0]]), z, np.array([[0.3, 0.4]]), th)[0]
    expect = 2.0 * math.exp(-0.5 / 0.5) / (2.0 + 0.5) * 1.7    # nu = 1/2: M(x) = exp(-x)
    assert abs(p - expect) <= 1e-12


def test_rmse_definition():
    assert oracle.rmse([1.0, 2.0, 3.0], [1.0, 0.0, 3.0]) == math.sqrt(4.0 / 3.0)


def test_profile_likelihood_is_the_maximum_over_sigma2():
    # L_p(ell, nu, rho) = L(ell, nu, s2_hat, rho s2_hat) and L at any other
    # sigma2 on the same ray is lower (the maximiser is the closed form)
    rng = np.random.default_rng(8)
    locs = rng.uniform(size=(60, 2))
    Z = rng.normal(size=60) * 1.3
    lp, s2 = oracle.loglik_profiled(locs, Z, 0.2, 0.7, 0.05)
    full = oracle.loglik_dense(locs, Z, (0.2, 0.7, s2, 0.05 * s2))[0]
    assert abs(lp - full) <= 1e-9 * abs(full)
    for f in (0.5, 0.9, 1.1, 2.0):
        assert oracle.loglik_dense(locs, Z, (0.2, 0.7, f * s2, 0.05 * f * s2))[0] < lp


def test_mloe_mmom_vanish_for_the_true_model_and_mloe_is_nonnegative():
    # Eq. 5-6: with the approximated model equal to the true one both
    # measures are 0; the true model's predictor has the smallest mean square
    # error under the true model, so MLOE >= 0 for any other model
    rng = np.random.default_rng(12)
    locs1 = rng.uniform(size=(120, 2))
    locs2 = rng.uniform(size=(15, 2))
    th = (0.15, 0.8, 1.0, 0.02)
    lo, mo = oracle.mloe_mmom(locs1, locs2, th, th)
    assert abs(lo) <= 1e-10 and abs(mo) <= 1e-10
    for tha in [(0.3, 0.8, 1.0, 0.02), (0.15, 1.6, 2.0, 0.1), (0.08, 0.5, 0.5, 0.01)]:
        lo, mo = oracle.mloe_mmom(locs1, locs2, th, tha)
        assert lo >= -1e-12


def test_prediction_errors_per_location_from_the_joint_covariance():
    # Per location, by another route than the oracle's solves: the kriging
    # variance is the conditional variance of Z(s_j) given Z_1, the inverse
    # of the last diagonal entry of the inverse joint covariance of
    # (Z_1, Z(s_j)); the error of predictor a under the true model is the
    # variance w^T J_t w of w = (l_a, -1), the coefficients of Z_a - Z; and
    # no predictor beats the true model's under the true model
    rng = np.random.default_rng(21)
    locs1 = rng.uniform(size=(80, 2))
    locs2 = rng.uniform(size=(9, 2))
    tht, tha = (0.15, 0.8, 1.0, 0.02), (0.25, 1.4, 1.5, 0.05)
    e_tt, e_aa, e_ta = oracle.prediction_errors(locs1, locs2, tht, tha)
    n = len(locs1)
    for j in range(len(locs2)):
        pts = np.vstack([locs1, locs2[j:j + 1]])
        Jt, Ja = oracle.matern_matrix(pts, tht), oracle.matern_matrix(pts, tha)
        assert abs(e_tt[j] - 1.0 / np.linalg.inv(Jt)[n, n]) <= 1e-10 * Jt[n, n]
        assert abs(e_aa[j] - 1.0 / np.linalg.inv(Ja)[n, n]) <= 1e-10 * Ja[n, n]
        w = np.append(np.linalg.solve(Ja[:n, :n], Ja[:n, n]), -1.0)
        assert abs(e_ta[j] - w @ Jt @ w) <= 1e-10 * Jt[n, n]
        assert e_ta[j] >= e_tt[j] - 1e-12


# --- LDL^T (Sec. 2: the factorisation without square roots) -------------------

def test_ldlt_hand_examples():
    # [[4, 2], [2, 3]]: d1 = 4, l21 = 2/4, d2 = 3 - (1/2)^2 4 = 2 (by hand)
    L, d = oracle.ldlt(np.array([[4.0, 2.0], [2.0, 3.0]]))
    assert L[1, 0] == 0.5 and list(d) == [4.0, 2.0] and L[0, 1] == 0.0 and L[1, 1] == 1.0
    # indefinite [[1, 2], [2, 1]]: the factorisation exists, d = (1, -3), l21 = 2
    L, d = oracle.ldlt(np.array([[1.0, 2.0], [2.0, 1.0]]))
    assert L[1, 0] == 2.0 and list(d) == [1.0, -3.0]
    # 3 x 3 by hand: [[2, -2, 0], [-2, 5, 3], [0, 3, 6]] -> d = (2, 3, 3),
    # l21 = -1, l31 = 0, l32 = 1
    L, d = oracle.ldlt(np.array([[2.0, -2.0, 0.0], [-2.0, 5.0, 3.0], [0.0, 3.0, 6.0]]))
    assert list(d) == [2.0, 3.0, 3.0]
    assert (L[1, 0], L[2, 0], L[2, 1]) == (-1.0, 0.0, 1.0)


def test_ldlt_is_the_cholesky_factor_without_square_roots():
    # L_chol = L D^(1/2) (Sec. 2), against LAPACK's Cholesky as a library routine
    locs = synth.locations_uniform(50, 2, seed=61)
    C = oracle.matern_matrix(locs, (0.2, 1.3, 1.5, 0.02))
    L, d = oracle.ldlt(C)
    Lc = np.linalg.cholesky(C)
    assert np.abs(L * np.sqrt(d) - Lc).max() <= 1e-12
    assert np.abs(L @ np.diag(d) @ L.T - C).max() <= 1e-13


def test_loglik_ldlt_matches_closed_forms_and_the_cholesky_route():
    # nugget only: L = I, d = tau2, the closed form of Eq. 1
    n, t2 = 30, 0.3
    Z = synth.normal(62, n)
    ll, ld, q = oracle.loglik_ldlt(t2 * np.eye(n), Z)
    assert abs(ld - n * math.log(t2)) <= 1e-12 * n
    assert abs(q - Z @ Z / t2) <= 1e-12 * (Z @ Z / t2)
    assert abs(ll - (-0.5 * n * math.log(2 * math.pi) - 0.5 * n * math.log(t2) - 0.5 * Z @ Z / t2)) <= 1e-10
    # a Matern C: the same (L, log|C|, q) as the Cholesky route, and log|C|
    # as numpy's slogdet (LU with pivoting, another library routine)
    locs = synth.locations_uniform(80, 2, seed=63)
    C = oracle.matern_matrix(locs, (0.15, 0.7, 1.0, 0.01))
    Z = synth.normal(64, 80)
    a = oracle.loglik_ldlt(C, Z)
    b = oracle.loglik_from_matrix(C, Z)
    sign, sld = np.linalg.slogdet(C)
    assert sign == 1.0 and abs(a[1] - sld) <= 1e-10 * abs(sld)
    for u, v in zip(a, b):
        assert abs(u - v) <= 1e-10 * max(1.0, abs(v))


def test_loglik_ldlt_rejects_an_indefinite_matrix():
    with pytest.raises(np.linalg.LinAlgError):
        oracle.loglik_ldlt(np.array([[1.0, 2.0], [2.0, 1.0]]), np.ones(2))


def test_mloe_mmom_one_training_point_by_hand():
    # One training point s1 and one test point s2 at distance h, nu = 1/2
    # (M(x) = e^{-x}).  Kriging weight of model m: lam_m = c_m / v_m with
    # c_m = sigma2_m e^{-h / ell_m} and v_m = sigma2_m + tau2_m.  Mean square
    # errors: e_tt = v_t - c_t^2 / v_t, e_aa = v_a - c_a^2 / v_a and
    # e_ta = v_t - 2 lam_a c_t + lam_a^2 v_t; MLOE = e_ta / e_tt - 1,
    # MMOM = e_aa / e_ta - 1 (Eq. 5-6).
    s1, s2 = np.array([[0.2, 0.3]]), np.array([[0.5, 0.7]])
    h = 0.5                                           # |(0.3, 0.4)|
    tt, ta = (0.3, 0.5, 1.2, 0.1), (0.15, 0.5, 0.8, 0.05)
    def parts(th):
        c = th[2] * math.exp(-h / th[0])
        v = th[2] + th[3]
        return c, v
    ct, vt = parts(tt)
    ca, va = parts(ta)
    lam = ca / va
    e_tt = vt - ct * ct / vt
    e_aa = va - ca * ca / va
    e_ta = vt - 2.0 * lam * ct + lam * lam * vt
    lo, mo = oracle.mloe_mmom(s1, s2, tt, ta)
    assert abs(lo - (e_ta / e_tt - 1.0)) <= 1e-13
    assert abs(mo - (e_aa / e_ta - 1.0)) <= 1e-13


def test_profile_likelihood_of_white_noise_in_closed_form():
    # ell -> 0 with distinct points: R = (1 + rho) I, so sigma2_hat =
    # Z^T Z / (n (1 + rho)) and L_p = -n/2 log 2 pi - n/2 log sigma2_hat
    # - n/2 log(1 + rho) - n/2
    rng = np.random.default_rng(9)
    locs = rng.uniform(size=(40, 2))
    Z = rng.normal(size=40) * 0.7
    n, rho = 40, 0.3
    lp, s2 = oracle.loglik_profiled(locs, Z, 1e-6, 0.5, rho)
    s2_ref = float(Z @ Z) / (n * (1 + rho))
    assert abs(s2 - s2_ref) <= 1e-12 * s2_ref
    ref = -0.5 * n * math.log(2 * math.pi) - 0.5 * n * math.log(s2_ref) \
        - 0.5 * n * math.log(1 + rho) - 0.5 * n
    assert abs(lp - ref) <= 1e-10 * abs(ref)


def test_plain_cholesky_is_the_library_factor():
    # the oracle's written-out row-by-row Cholesky against LAPACK's (the
    # factor of an SPD matrix is unique), and its refusal of an indefinite one
    n = 400
    locs = synth.locations_uniform(n, 2, seed=17)
    C = oracle.matern_matrix(locs, (0.1, 1.5, 1.0, 1e-4))
    L = oracle.cholesky_plain(C)
    assert np.allclose(L, np.tril(L), rtol=0, atol=0)
    assert np.max(np.abs(L - np.linalg.cholesky(C))) <= 1e-12
    assert np.max(np.abs(L @ L.T - C)) <= 1e-12
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky_plain(np.array([[1.0, 2.0], [2.0, 1.0]]))
