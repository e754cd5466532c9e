"""Prediction errors of the kriging predictor (Eq. 5-7).

Thin driver over the C ABI.  MLOE and MMOM come from hmle_prediction_errors.
The per-location columns of the cross-covariance, the solves (cooperative
sweeps over up to 256 columns at once), the H-matvecs and the dot products
all run on the device; this module passes the factors and reads back the
means and the per-location errors.

For test locations s_1..s_M, a true model theta_t and an approximated
(estimated) model theta_a, with c_x(j) = C_x(train, s_j), C_x the covariance
of the training points and v_x = sigma2_x + tau2_x the variance of Z(s_j):
  E_t[(Z_t - Z)^2] = v_t - c_t(j)^T C_t^{-1} c_t(j)          (kriging variance)
  E_a[(Z_a - Z)^2] = v_a - c_a(j)^T C_a^{-1} c_a(j)
  E_t[(Z_a - Z)^2] = v_t - 2 l_a^T c_t(j) + l_a^T C_t l_a,   l_a = C_a^{-1} c_a(j)
  MLOE = mean_j (E_t[(Z_a - Z)^2] / E_t[(Z_t - Z)^2] - 1)   (Eq. 5)
  MMOM = mean_j (E_a[(Z_a - Z)^2] / E_t[(Z_a - Z)^2] - 1)   (Eq. 6)
  RMSE = sqrt(mean((Z_hat - Z)^2))                           (Eq. 7)

    python -m paper_2104_07146_gb300.prediction [--n 65536] [--m 1000]

times MLOE / MMOM at m test locations on the medium workload's point set
(true model: the workload's theta; approximated: ell and nu 10% off) and
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def rmse(pred, truth) -> float:
    d = np.asarray(pred, dtype=np.float64) - np.asarray(truth, dtype=np.float64)
    return float(np.sqrt(np.mean(d * d)))


def mloe_mmom(tree, locs2, theta_t, theta_a, per_point=False):
    """(MLOE, MMOM) of Eq. 5-6 at the M x d test locations locs2 (and the
    M x 3 per-location errors with per_point=True)."""
    ht, ha = tree.assemble(theta_t), tree.assemble(theta_a)
    ft, fa = ht.factor(None), ha.factor(None)
    try:
        loe, mom, per = ft.prediction_errors(fa, locs2)
    finally:
        for x in (ft, fa, ht, ha):
            x.close()
    return (loe, mom, per) if per_point else (loe, mom)


def main():
    from . import hmle, synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=65536)
    ap.add_argument("--m", type=int, default=1000)
    a = ap.parse_args()
    w = synth.MEDIUM
    locs = synth.locations_blobs(a.n, 2, w["frac_blob"], w["nblobs"], w["sd"], w["seed"])
    locs2 = synth.uniform(w["seed"] + 17, 2 * a.m).reshape(a.m, 2)
    th_t = tuple(w["theta"])
    th_a = (th_t[0] * 1.1, th_t[1] * 0.9, th_t[2], th_t[3])
    ctx = hmle.Context()
    tree = hmle.Tree(ctx, locs, leaf_size=w["leaf"], eta=w["eta"], aca_eps=w["aca_eps"])
    ht, ha = tree.assemble(th_t), tree.assemble(th_a)
    ft, fa = ht.factor(None), ha.factor(None)
    ft.prediction_errors(fa, locs2[:8])          # first use: tables, sweeps' grid size
    t0 = time.time()
    loe, mom, per = ft.prediction_errors(fa, locs2)
    dt = time.time() - t0
    print(json.dumps({"config": "medium point set n=%d, m=%d uniform test locations, theta_t=%s, "
                                "theta_a=%s, leaf %d, eps %g" % (a.n, a.m, th_t, th_a, w["leaf"], w["aca_eps"]),
                      "mloe": loe, "mmom": mom, "seconds": dt, "locations_per_s": a.m / dt,
                      "min_kriging_variance": float(per[:, 0].min())}))
    for x in (ft, fa, ht, ha, tree):
        x.close()


if __name__ == "__main__":
    main()
