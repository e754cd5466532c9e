"""Prediction errors of the kriging predictor (Eq. 5-7).

Thin driver over the C ABI: the solves (hmle_solve: forward and backward
sweeps), the cross-covariance products (hmle_cross_matvec) and the H-matvec
(hmle_hmatrix_matvec) all run in the library's kernels; this module only
combines their outputs.

For test locations s_1..s_M, a true model theta_t and an approximated
(estimated) model theta_a, with c_x(j) = C_x(train, s_j), C_x the covariance
of the training points and v_x = sigma2_x + tau2_x the variance of Z(s_j):
  E_t[(Z_t - Z)^2] = v_t - c_t(j)^T C_t^{-1} c_t(j)          (kriging variance)
  E_a[(Z_a - Z)^2] = v_a - c_a(j)^T C_a^{-1} c_a(j)
  E_t[(Z_a - Z)^2] = v_t - 2 l_a^T c_t(j) + l_a^T C_t l_a,   l_a = C_a^{-1} c_a(j)
  MLOE = mean_j (E_t[(Z_a - Z)^2] / E_t[(Z_t - Z)^2] - 1)   (Eq. 5)
  MMOM = mean_j (E_a[(Z_a - Z)^2] / E_t[(Z_a - Z)^2] - 1)   (Eq. 6)
  RMSE = sqrt(mean((Z_hat - Z)^2))                           (Eq. 7)
"""
from __future__ import annotations

import numpy as np


def rmse(pred, truth) -> float:
    d = np.asarray(pred, dtype=np.float64) - np.asarray(truth, dtype=np.float64)
    return float(np.sqrt(np.mean(d * d)))


def mloe_mmom(tree, locs2, theta_t, theta_a):
    """(MLOE, MMOM) of Eq. 5-6 at the M x d test locations locs2: 2 solves,
    2 cross-covariance products and one H-matvec per test location."""
    locs2 = np.ascontiguousarray(locs2, dtype=np.float64)
    M = locs2.shape[0]
    ht, ha = tree.assemble(theta_t), tree.assemble(theta_a)
    ft, fa = ht.factor(None), ha.factor(None)
    vt = theta_t[2] + theta_t[3]
    va = theta_a[2] + theta_a[3]
    loe, mom = [], []
    for j in range(M):
        e = np.zeros(M)
        e[j] = 1.0
        ct = tree.cross_matvec(theta_t, locs2, e, trans=True)
        ca = tree.cross_matvec(theta_a, locs2, e, trans=True)
        lt = ft.solve(ct)
        la = fa.solve(ca)
        e_tt = vt - ct @ lt
        e_aa = va - ca @ la
        e_ta = vt - 2.0 * (la @ ct) + la @ ht.matvec(la)
        loe.append(e_ta / e_tt - 1.0)
        mom.append(e_aa / e_ta - 1.0)
    for x in (ft, fa, ht, ha):
        x.close()
    return float(np.mean(loe)), float(np.mean(mom))
