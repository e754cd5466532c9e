"""CPU FP64 oracle for the H-MLE log-likelihood -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU product path
(``paper_2104_07146_gb300``) never imports it and shares no code with it.

What it computes (the exact, dense definitions the H-matrix method
approximates):

* ``matern_matrix`` -- C(theta) of Eq. 2 (Sec. 1): C_ij = sigma^2 M_nu(h/ell)
  + tau^2 [i == j], M_nu(x) = x^nu K_nu(x) / (2^(nu-1) Gamma(nu)).
* ``loglik_dense`` -- Eq. 1 (Sec. 1):
  L = -n/2 log(2 pi) - 1/2 log|C| - 1/2 Z^T C^{-1} Z, with log|C| =
  2 sum log L_ii (Sec. 2, "Storage and complexity") and
  Z^T C^{-1} Z = |L^{-1} Z|^2.
* ``ldlt`` / ``loglik_ldlt`` -- the square-root-free factorisation
  C = L D L^T of Sec. 2 (L unit lower triangular, D diagonal, related to the
  Cholesky factor by L_chol = L D^(1/2)); log|C| = sum log d_i and
  Z^T C^{-1} Z = sum (L^{-1} Z)_i^2 / d_i.
* ``predict`` / ``rmse`` / ``mloe_mmom`` -- kriging prediction
  Z2 = C21 C11^{-1} Z1 (Eq. 4), the root mean square error of Eq. 7 and the
  MLOE / MMOM measures of Eq. 5-6.
* ``transform`` / ``untransform`` -- the positivity transform of Sec. 5
  (Test 1a): sigma = 2 / 1.1^s0, ell = 1 / 1.5^l0, nu = 1 / 1.2^n0,
  tau = 1 / 2^t0.
* ``nelder_mead`` -- the MLE driver (Sec. 2, "Maximization of the
  log-likelihood"; threshold 1e-4 and at most 400 iterations).
* ``kalman_exponential`` / ``simulate_exponential_line`` -- Eq. 1 and a
  draw from the model, in O(n), for nu = 1/2 (C_ij = sigma^2 exp(-h/ell) +
  tau^2 [i == j], Eq. 2) on sorted collinear points: the exponential kernel
  is then an Ornstein-Uhlenbeck process, a Markov chain in x, so the
  prediction-error decomposition of a scalar Kalman filter is exact.  This is
  the reference at sizes where the dense factorisation cannot run.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hmle_oracle.c")
_LIB = os.path.join(_HERE, "libhmle_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, -O2, OpenMP) in-tree."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i64, i32, p = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.oracle_besselk_scaled.argtypes = [d, d]
        lib.oracle_besselk_scaled.restype = d
        lib.oracle_matern_unit.argtypes = [d, d]
        lib.oracle_matern_unit.restype = d
        lib.oracle_matern_matrix.argtypes = [i64, i32, p, d, d, d, d, p]
        lib.oracle_matern_matrix.restype = i32
        lib.oracle_matern_cross.argtypes = [i64, i64, i32, p, p, d, d, d, p]
        lib.oracle_matern_cross.restype = i32
        lib.oracle_forward_solve.argtypes = [i64, p, p, p]
        lib.oracle_forward_solve.restype = i32
        lib.oracle_cholesky.argtypes = [i64, p]
        lib.oracle_cholesky.restype = i32
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def besselk(nu: float, x: float) -> float:
    """K_nu(x) for x > 0 (integral representation, trapezoid rule)."""
    return _load().oracle_besselk_scaled(float(nu), float(x)) * math.exp(-float(x))


def besselk_scaled(nu: float, x: float) -> float:
    """e^x K_nu(x) for x > 0."""
    return _load().oracle_besselk_scaled(float(nu), float(x))


def matern_unit(nu: float, x: float) -> float:
    """M_nu(x) = x^nu K_nu(x) / (2^(nu-1) Gamma(nu)), M_nu(0) = 1."""
    return _load().oracle_matern_unit(float(nu), float(x))


def matern_matrix(locs: np.ndarray, theta) -> np.ndarray:
    """Dense C(theta) of Eq. 2; theta = (ell, nu, sigma2, tau2)."""
    locs = np.ascontiguousarray(locs, dtype=np.float64)
    n, d = locs.shape
    ell, nu, s2, t2 = (float(v) for v in theta)
    C = np.empty((n, n), dtype=np.float64)
    rc = _load().oracle_matern_matrix(n, d, _ptr(locs), ell, nu, s2, t2, _ptr(C))
    if rc != 0:
        raise ValueError("oracle_matern_matrix: invalid arguments")
    return C


def matern_cross(A: np.ndarray, B: np.ndarray, theta) -> np.ndarray:
    """Cross-covariance sigma^2 M_nu(|a_i - b_j| / ell), no nugget."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    ell, nu, s2, _ = (float(v) for v in theta)
    out = np.empty((A.shape[0], B.shape[0]), dtype=np.float64)
    rc = _load().oracle_matern_cross(A.shape[0], B.shape[0], A.shape[1], _ptr(A),
                                     _ptr(B), ell, nu, s2, _ptr(out))
    if rc != 0:
        raise ValueError("oracle_matern_cross: invalid arguments")
    return out


def forward_solve(L: np.ndarray, z: np.ndarray) -> np.ndarray:
    L = np.ascontiguousarray(L, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    w = np.empty_like(z)
    if _load().oracle_forward_solve(L.shape[0], _ptr(L), _ptr(z), _ptr(w)) != 0:
        raise np.linalg.LinAlgError("non-positive pivot in forward solve")
    return w


PLAIN_CHOLESKY_MAX_N = 512


def cholesky_plain(C: np.ndarray) -> np.ndarray:
    """Dense Cholesky factor by the unblocked row-by-row algorithm written
    out in the oracle's C code; raises numpy.linalg.LinAlgError when C is not
    positive definite."""
    A = np.array(C, dtype=np.float64, order="C", copy=True)
    if _load().oracle_cholesky(A.shape[0], _ptr(A)) != 0:
        raise np.linalg.LinAlgError("non-positive pivot")
    return A


def cholesky(C: np.ndarray) -> np.ndarray:
    """Dense Cholesky factor: the plain algorithm (cholesky_plain) up to
    n = 512, LAPACK dpotrf through numpy above (the same factor to rounding:
    a pin checks the two against each other); raises
    numpy.linalg.LinAlgError when C is not positive definite."""
    if C.shape[0] <= PLAIN_CHOLESKY_MAX_N:
        return cholesky_plain(C)
    return np.linalg.cholesky(C)


def loglik_from_matrix(C: np.ndarray, Z: np.ndarray):
    """(L, log|C|, Z^T C^{-1} Z) of Eq. 1 for a given dense SPD C."""
    n = C.shape[0]
    L = cholesky(C)
    logdet = 0.0
    for v in np.diag(L):           # sequential sum in index order
        logdet += 2.0 * math.log(v)
    w = forward_solve(L, np.asarray(Z, dtype=np.float64))
    q = 0.0
    for v in w:
        q += v * v
    ll = -0.5 * n * math.log(2.0 * math.pi) - 0.5 * logdet - 0.5 * q
    return ll, logdet, q


def ldlt(C: np.ndarray):
    """C = L D L^T without pivoting (Sec. 2, the factorisation that extracts
    no square roots): column j gives d_j = C_jj - sum_{k<j} L_jk^2 d_k, then
    L_ij = (C_ij - sum_{k<j} L_ik L_jk d_k) / d_j for i > j.  Returns
    (L unit lower triangular, d).  It exists whenever every leading minor of
    C is non-zero, so it also runs on symmetric indefinite matrices; a zero
    pivot raises numpy.linalg.LinAlgError."""
    C = np.asarray(C, dtype=np.float64)
    n = C.shape[0]
    L = np.eye(n)
    d = np.zeros(n)
    for j in range(n):
        d[j] = C[j, j] - np.dot(L[j, :j] ** 2, d[:j])
        if d[j] == 0.0:
            raise np.linalg.LinAlgError("zero pivot in LDL^T")
        for i in range(j + 1, n):
            L[i, j] = (C[i, j] - np.dot(L[i, :j] * L[j, :j], d[:j])) / d[j]
    return L, d


def loglik_ldlt(C: np.ndarray, Z: np.ndarray):
    """(L, log|C|, Z^T C^{-1} Z) of Eq. 1 through C = L D L^T: w solves the
    unit lower triangular system L w = Z by forward substitution, log|C| =
    sum log d_i and q = sum w_i^2 / d_i (sequential sums in index order).
    The Gaussian density needs C positive definite, so a pivot d_i <= 0
    raises numpy.linalg.LinAlgError, as the Cholesky route does."""
    L, d = ldlt(C)
    if not np.all(d > 0.0):
        raise np.linalg.LinAlgError("non-positive pivot in LDL^T: C is not positive definite")
    n = len(d)
    Z = np.asarray(Z, dtype=np.float64)
    w = np.empty(n)
    for i in range(n):
        w[i] = Z[i] - np.dot(L[i, :i], w[:i])
    logdet = 0.0
    q = 0.0
    for i in range(n):
        logdet += math.log(d[i])
        q += w[i] * w[i] / d[i]
    return -0.5 * n * math.log(2.0 * math.pi) - 0.5 * logdet - 0.5 * q, logdet, q


def loglik_dense(locs: np.ndarray, Z: np.ndarray, theta):
    """Exact Eq. 1 with C from Eq. 2.  Returns (L, log|C|, q)."""
    return loglik_from_matrix(matern_matrix(locs, theta), Z)


def simulate(locs: np.ndarray, theta, xi: np.ndarray) -> np.ndarray:
    """Z = L xi with L the dense Cholesky factor of C(theta)."""
    return cholesky(matern_matrix(locs, theta)) @ np.asarray(xi, dtype=np.float64)


def kalman_exponential(x: np.ndarray, z: np.ndarray, ell: float, s2: float, t2: float) -> float:
    """Exact Eq. 1 for nu = 1/2 on sorted collinear points x (Eq. 2 with
    M_1/2(h) = exp(-h)): the latent state follows x_i = rho_i x_{i-1} + noise
    with rho_i = exp(-(x_i - x_{i-1}) / ell) and stationary variance s2, each
    observation adds t2; L is the sum over i of the Gaussian log-density of
    the one-step prediction error."""
    m, P = 0.0, s2                       # prior of the latent state at x_0
    ll = 0.0
    log2pi = math.log(2.0 * math.pi)
    for i in range(len(x)):
        if i > 0:
            rho = math.exp(-(x[i] - x[i - 1]) / ell)
            m, P = rho * m, rho * rho * P + s2 * (1.0 - rho * rho)
        S = P + t2
        e = z[i] - m
        ll += -0.5 * (log2pi + math.log(S) + e * e / S)
        K = P / S
        m, P = m + K * e, (1.0 - K) * P
    return ll


def simulate_exponential_line(x: np.ndarray, theta, xi: np.ndarray, eta: np.ndarray) -> np.ndarray:
    """A draw from the model of Eq. 2 with nu = 1/2 on sorted collinear
    points x: the latent Ornstein-Uhlenbeck state u_0 = sigma xi_0,
    u_i = rho_i u_{i-1} + sigma sqrt(1 - rho_i^2) xi_i (rho_i as above) is
    L xi with L the Cholesky factor of sigma^2 exp(-|x_i - x_j| / ell), and
    the observation adds the nugget, z = u + tau eta."""
    ell, nu, s2, t2 = theta
    assert nu == 0.5
    x = np.asarray(x, dtype=np.float64)
    xi = np.asarray(xi, dtype=np.float64)
    sig = math.sqrt(s2)
    rho = np.exp(-np.diff(x) / ell)
    gain = sig * np.sqrt(1.0 - rho * rho)
    u = np.empty_like(x)
    u[0] = sig * xi[0]
    for i in range(1, len(x)):
        u[i] = rho[i - 1] * u[i - 1] + gain[i - 1] * xi[i]
    return u + math.sqrt(t2) * np.asarray(eta, dtype=np.float64)


def loglik_profiled(locs: np.ndarray, Z: np.ndarray, ell: float, nu: float, rho: float):
    """The profile log-likelihood over sigma2 (Sec. 7: update instead of
    recompute): with C = sigma2 R, R = M_nu(h / ell) + rho I, maximising Eq. 1
    over sigma2 gives sigma2_hat = Z^T R^{-1} Z / n and
    L_p = -n/2 log(2 pi) - n/2 log(sigma2_hat) - 1/2 log|R| - n/2.
    Returns (L_p, sigma2_hat)."""
    n = len(Z)
    _, ld, q = loglik_dense(locs, Z, (ell, nu, 1.0, rho))
    s2 = q / n
    return -0.5 * n * math.log(2 * math.pi) - 0.5 * n * math.log(s2) - 0.5 * ld - 0.5 * n, s2


def predict(locs1: np.ndarray, Z1: np.ndarray, locs2: np.ndarray, theta) -> np.ndarray:
    """Kriging prediction of Eq. 4: Z2 = C21 C11^{-1} Z1, C11 from Eq. 2 at the
    n1 training locations (nugget on its diagonal), C21 the cross-covariance
    without nugget.  C11^{-1} Z1 by the dense Cholesky factor: L w = Z1
    (forward substitution), then L^T x = w (back substitution)."""
    L = cholesky(matern_matrix(locs1, theta))
    w = forward_solve(L, np.asarray(Z1, dtype=np.float64))
    x = np.linalg.solve(L.T, w)   # library triangular step (upper)
    return matern_cross(locs2, locs1, theta) @ x


def prediction_errors(locs1: np.ndarray, locs2: np.ndarray, theta_t, theta_a):
    """The per-location mean square errors behind Eq. 5-6, with dense FP64
    matrices.  For each test location s_j, the kriging predictors under the
    true (t) and approximated (a) models: with c = cross-covariance column,
    C = training covariance, v = sigma2 + tau2 (the variance of Z(s_j)),
    l_a = C_a^{-1} c_a:
      E_t[(Z_t - Z)^2] = v_t - c_t^T C_t^{-1} c_t
      E_a[(Z_a - Z)^2] = v_a - c_a^T l_a
      E_t[(Z_a - Z)^2] = v_t - 2 l_a^T c_t + l_a^T C_t l_a
    Returns the three arrays (M each) in that order."""
    Ct, Ca = matern_matrix(locs1, theta_t), matern_matrix(locs1, theta_a)
    ct = matern_cross(locs1, locs2, theta_t)          # n x M columns c_t(j)
    ca = matern_cross(locs1, locs2, theta_a)
    lt = np.linalg.solve(Ct, ct)
    la = np.linalg.solve(Ca, ca)
    vt = float(theta_t[2]) + float(theta_t[3])
    va = float(theta_a[2]) + float(theta_a[3])
    e_tt = vt - np.sum(ct * lt, axis=0)
    e_aa = va - np.sum(ca * la, axis=0)
    e_ta = vt - 2.0 * np.sum(la * ct, axis=0) + np.sum(la * (Ct @ la), axis=0)
    return e_tt, e_aa, e_ta


def mloe_mmom(locs1: np.ndarray, locs2: np.ndarray, theta_t, theta_a):
    """MLOE and MMOM of Eq. 5-6: MLOE = mean(E_t[a] / E_t[t] - 1),
    MMOM = mean(E_a[a] / E_t[a] - 1) over the per-location errors of
    prediction_errors."""
    e_tt, e_aa, e_ta = prediction_errors(locs1, locs2, theta_t, theta_a)
    return float(np.mean(e_ta / e_tt - 1.0)), float(np.mean(e_aa / e_ta - 1.0))


def rmse(pred: np.ndarray, truth: np.ndarray) -> float:
    """Eq. 7: sqrt(mean((Z_hat - Z)^2)) over the test locations."""
    d = np.asarray(pred, dtype=np.float64) - np.asarray(truth, dtype=np.float64)
    return float(np.sqrt(np.mean(d * d)))


# --- positivity transform of Sec. 5 (Test 1a) ---------------------------------

def transform(x):
    """Transformed coordinates (s0, l0, n0, t0) -> theta (ell, nu, sigma2, tau2).

    sigma = 2 / 1.1^s0, ell = 1 / 1.5^l0, nu = 1 / 1.2^n0, tau = 1 / 2^t0.
    """
    s0, l0, n0, t0 = (float(v) for v in x)
    sigma = 2.0 / 1.1 ** s0
    ell = 1.0 / 1.5 ** l0
    nu = 1.0 / 1.2 ** n0
    tau = 1.0 / 2.0 ** t0
    return (ell, nu, sigma * sigma, tau * tau)


def untransform(theta):
    """theta (ell, nu, sigma2, tau2) -> (s0, l0, n0, t0), the exact inverse."""
    ell, nu, s2, t2 = (float(v) for v in theta)
    s0 = -math.log(math.sqrt(s2) / 2.0) / math.log(1.1)
    l0 = -math.log(ell) / math.log(1.5)
    n0 = -math.log(nu) / math.log(1.2)
    t0 = -math.log(math.sqrt(t2)) / math.log(2.0)
    return (s0, l0, n0, t0)


# --- Nelder-Mead ---------------------------------------------------------------

def nelder_mead(f, x0, step=1.0, ftol=1e-4, xtol=1e-4, max_iter=400):
    """Minimise f by the Nelder-Mead simplex method (reflection 1, expansion 2,
    contraction 1/2, shrink 1/2; Lagarias et al. 1998 ordering rules).

    The initial simplex is x0 plus ``step`` (scalar or per-coordinate) along
    each axis.  Stops when max_i |f_i - f_best| <= ftol and
    max_i |x_i - x_best|_inf <= xtol, or after ``max_iter`` iterations.
    Equal f values keep their previous order (stable sort), so the run is
    deterministic.  Returns (x_best, f_best, iterations, evaluations).
    """
    x0 = np.asarray(x0, dtype=np.float64)
    m = x0.size
    steps = np.broadcast_to(np.asarray(step, dtype=np.float64), (m,))
    simplex = [x0.copy()]
    for i in range(m):
        v = x0.copy()
        v[i] += steps[i]
        simplex.append(v)
    fvals = [f(v) for v in simplex]
    nev = m + 1
    it = 0
    while True:
        order = sorted(range(m + 1), key=lambda i: fvals[i])
        simplex = [simplex[i] for i in order]
        fvals = [fvals[i] for i in order]
        fspread = max(abs(fv - fvals[0]) for fv in fvals[1:])
        xspread = max(float(np.max(np.abs(v - simplex[0]))) for v in simplex[1:])
        if (fspread <= ftol and xspread <= xtol) or it >= max_iter:
            break
        it += 1
        centroid = sum(simplex[:-1]) / m
        worst = simplex[-1]
        xr = centroid + (centroid - worst)
        fr = f(xr); nev += 1
        if fvals[0] <= fr < fvals[-2]:
            simplex[-1], fvals[-1] = xr, fr
            continue
        if fr < fvals[0]:
            xe = centroid + 2.0 * (centroid - worst)
            fe = f(xe); nev += 1
            if fe < fr:
                simplex[-1], fvals[-1] = xe, fe
            else:
                simplex[-1], fvals[-1] = xr, fr
            continue
        if fr < fvals[-1]:          # outside contraction
            xc = centroid + 0.5 * (xr - centroid)
            fc = f(xc); nev += 1
            if fc <= fr:
                simplex[-1], fvals[-1] = xc, fc
                continue
        else:                       # inside contraction
            xc = centroid + 0.5 * (worst - centroid)
            fc = f(xc); nev += 1
            if fc < fvals[-1]:
                simplex[-1], fvals[-1] = xc, fc
                continue
        best = simplex[0]           # shrink towards the best vertex
        for i in range(1, m + 1):
            simplex[i] = best + 0.5 * (simplex[i] - best)
            fvals[i] = f(simplex[i]); nev += 1
    return simplex[0], fvals[0], it, nev


def fit(locs, Z, theta0, step=1.0, ftol=1e-4, xtol=1e-4, max_iter=400):
    """MLE: maximise Eq. 1 over theta by Nelder-Mead in the transformed
    coordinates of Sec. 5.  Non-SPD trial points score -inf.
    Returns (theta_hat, L_hat, iterations, evaluations)."""

    def negll(x):
        try:
            return -loglik_dense(locs, Z, transform(x))[0]
        except np.linalg.LinAlgError:
            return math.inf

    xb, fb, it, nev = nelder_mead(negll, untransform(theta0), step, ftol, xtol, max_iter)
    return transform(xb), -fb, it, nev
