"""a16: the learned start of the MLE (Sec. 7 suggests precomputing the
optimiser's initial guess).

Thin driver over the C ABI (every numerical step runs in the library's
kernels): field statistics (``hmle_features``), the perceptron
(``hmle_mlp_*``), training data simulated by the H-Cholesky factor itself
(``hmle_simulate``, Sec. 2 factorisation used as Z = L~ xi), and the
comparison against the default start.

The perceptron predicts the transformed coordinates of Sec. 5 (mu) and log
initial simplex steps (s).  ``LearnedStart.start`` turns them into a theta
and steps for ``hmle_fit``; if the prediction is not finite or leaves the
admissible range it falls back to the default start (theta0 =
(0.2, 1.0, 0.5, 0.05), unit steps).
"""
from __future__ import annotations

import ctypes as C
import math
import time

import numpy as np

from . import hmle, synth
from .hmle import P, lib

NF = 35
DEFAULT_THETA0 = (0.2, 1.0, 0.5, 0.05)

# prior box of the simulated training fields (theta order ell, nu, sigma2,
# tau2): ell and tau2 log-uniform, nu and sigma2 uniform
PRIOR = {"ell": (0.02, 0.3), "nu": (0.3, 2.5), "sigma2": (0.5, 2.0), "tau2": (1e-4, 0.1)}


def theta_to_x(theta):
    x = (C.c_double * 4)()
    st = lib().hmle_theta_to_x(C.byref(hmle._theta(theta)), x)
    if st != 0:
        raise hmle.HmleError(st, "hmle_theta_to_x")
    return np.array(list(x))


def x_to_theta(x):
    xa = (C.c_double * 4)(*[float(v) for v in x])
    th = hmle.Theta()
    st = lib().hmle_x_to_theta(xa, C.byref(th))
    if st != 0:
        return None
    return (th.ell, th.nu, th.sigma2, th.tau2)


def features(ctx: hmle.Context, locs, Z) -> np.ndarray:
    locs = np.ascontiguousarray(locs, dtype=np.float64)
    n, d = locs.shape
    f = np.zeros(NF, dtype=np.float32)
    pz, keep = hmle._ptr(np.ascontiguousarray(Z, dtype=np.float64))
    ctx.check(lib().hmle_features(ctx._h, P(locs.ctypes.data), n, d, pz, P(f.ctypes.data)),
              "hmle_features")
    return f


class LearnedStart:
    """The perceptron of the learned start (owns an hmle_mlp)."""

    def __init__(self, ctx: hmle.Context, seed: int = 1):
        self.ctx = ctx
        self._h = P()
        ctx.check(lib().hmle_mlp_create(ctx._h, C.c_uint64(seed), C.byref(self._h)),
                  "hmle_mlp_create")
        self.nparams = lib().hmle_mlp_nparams()

    def close(self):
        if self._h:
            lib().hmle_mlp_destroy(self._h)
            self._h = P()

    def __del__(self):
        import sys
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def get(self):
        p = np.zeros(self.nparams, dtype=np.float32)
        mu = np.zeros(NF, dtype=np.float32)
        sd = np.zeros(NF, dtype=np.float32)
        self.ctx.check(lib().hmle_mlp_get(self.ctx._h, self._h, P(p.ctypes.data), P(mu.ctypes.data),
                                          P(sd.ctypes.data)), "hmle_mlp_get")
        return p, mu, sd

    def set(self, params=None, mu=None, sd=None):
        def ptr(a):
            if a is None:
                return None, None
            a = np.ascontiguousarray(a, dtype=np.float32)
            return P(a.ctypes.data), a
        (pp, k1), (pm, k2), (ps, k3) = ptr(params), ptr(mu), ptr(sd)
        self.ctx.check(lib().hmle_mlp_set(self.ctx._h, self._h, pp, pm, ps), "hmle_mlp_set")

    def forward(self, feats) -> np.ndarray:
        F = np.ascontiguousarray(np.atleast_2d(feats), dtype=np.float32)
        out = np.zeros((F.shape[0], 8), dtype=np.float32)
        self.ctx.check(lib().hmle_mlp_forward(self.ctx._h, self._h, P(F.ctypes.data), F.shape[0],
                                              P(out.ctypes.data)), "hmle_mlp_forward")
        return out

    def grad(self, feats, targets):
        F = np.ascontiguousarray(feats, dtype=np.float32)
        T = np.ascontiguousarray(targets, dtype=np.float32)
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = C.c_float()
        self.ctx.check(lib().hmle_mlp_grad(self.ctx._h, self._h, P(F.ctypes.data), P(T.ctypes.data),
                                           F.shape[0], P(g.ctypes.data), C.byref(loss)),
                       "hmle_mlp_grad")
        return g, loss.value

    def adam_step(self, grad, lr):
        g = np.ascontiguousarray(grad, dtype=np.float32)
        self.ctx.check(lib().hmle_mlp_adam_step(self.ctx._h, self._h, P(g.ctypes.data),
                                                C.c_float(lr)), "hmle_mlp_adam_step")

    def train(self, feats, targets, epochs=200, batch=64, lr=3e-3, seed=7):
        F = np.ascontiguousarray(feats, dtype=np.float32)
        T = np.ascontiguousarray(targets, dtype=np.float32)
        l0, l1 = C.c_float(), C.c_float()
        self.ctx.check(lib().hmle_mlp_train(self.ctx._h, self._h, P(F.ctypes.data), P(T.ctypes.data),
                                            F.shape[0], epochs, batch, C.c_float(lr),
                                            C.c_uint64(seed), C.byref(l0), C.byref(l1)),
                       "hmle_mlp_train")
        return l0.value, l1.value

    def start(self, locs, Z):
        """(theta0, steps, used_fallback) for hmle_fit on this field."""
        y = self.forward(features(self.ctx, locs, Z))[0].astype(np.float64)
        mu, s = y[:4], y[4:]
        th = x_to_theta(mu) if np.all(np.isfinite(y)) else None
        if th is None or not (1e-4 <= th[0] <= 1e3 and 0.05 <= th[1] <= 20.0):
            return DEFAULT_THETA0, [1.0, 1.0, 1.0, 1.0], True
        steps = [float(min(2.0, max(0.05, math.exp(v)))) for v in s]
        return th, steps, False


def draw_theta(seed: int, i: int):
    """theta of training field i: log-uniform ell and tau2, uniform nu and
    sigma2, over the prior box."""
    u = synth.uniform(seed * 1_000_003 + i, 4)
    lo, hi = PRIOR["ell"]
    ell = lo * (hi / lo) ** u[0]
    nu = PRIOR["nu"][0] + (PRIOR["nu"][1] - PRIOR["nu"][0]) * u[1]
    s2 = PRIOR["sigma2"][0] + (PRIOR["sigma2"][1] - PRIOR["sigma2"][0]) * u[2]
    lo, hi = PRIOR["tau2"]
    t2 = lo * (hi / lo) ** u[3]
    return (float(ell), float(nu), float(s2), float(t2))


def field(ctx, seed: int, i: int, n: int, three_d: bool = False):
    """Field i of a seeded family: point set (2-D uniform or blob mixture,
    alternating, or uniform in the unit cube with three_d), theta from the
    prior, Z = L~ xi simulated by the H-Cholesky factor at eps 1e-8 (1e-6
    when the smoothest fields need more rank than the blocks hold at 1e-8)."""
    th = draw_theta(seed, i)
    if three_d:
        locs = synth.uniform(seed * 7919 + i, 3 * n).reshape(n, 3)
    elif i % 2 == 0:
        locs = synth.locations_uniform(n, 2, seed=seed * 7919 + i)
    else:
        locs = synth.locations_blobs(n, 2, 0.3, 8, 0.03, seed=seed * 7919 + i)
    xi = synth.normal(seed * 104729 + i, n)
    leaf = 32 if n <= 3000 else 64
    for eps in (1e-8, 1e-6):
        tree = hmle.Tree(ctx, locs, leaf_size=leaf, aca_eps=eps, max_rank=48, oversample=16)
        try:
            Z = tree.simulate(th, xi)
            return locs, Z, th
        except hmle.HmleError as e:
            if e.status != 5:   # only a rank overflow is retried
                raise
        finally:
            tree.close()
    raise hmle.HmleError(5, "simulate: rank overflow at eps 1e-6")


def training_set(ctx, count: int, seed: int = 11, n_range=(4096, 16384), three_d_every: int = 0,
                 time_limit_s: float = 0.0):
    """Up to count simulated fields -> (features k x 35, targets k x 4): n
    log-uniform in n_range; every three_d_every-th field 3-D (0: none).
    With time_limit_s > 0 the generation stops after that many seconds and
    returns the fields made so far (k <= count)."""
    F = np.zeros((count, NF), dtype=np.float32)
    T = np.zeros((count, 4), dtype=np.float32)
    t0 = time.time()
    k = 0
    for i in range(count):
        if time_limit_s > 0 and time.time() - t0 > time_limit_s:
            break
        u = synth.uniform(seed * 31337 + i, 1)[0]
        n = int(n_range[0] * (n_range[1] / n_range[0]) ** u)
        three = three_d_every > 0 and i % three_d_every == three_d_every - 1
        try:
            locs, Z, th = field(ctx, seed, i, n, three)
        except hmle.HmleError as e:
            if e.status != 5:
                raise
            continue            # a field whose ranks overflow even at 1e-6: skipped
        F[k] = features(ctx, locs, Z)
        T[k] = theta_to_x(th)
        k += 1
    return F[:k], T[:k]


def compare_starts(ctx, model: LearnedStart, fields, **fit_kw):
    """Fit every (locs, Z, theta) field from the default start and from the
    learned start.  Returns per-field records and totals."""
    rows = []
    for locs, Z, th in fields:
        tree = hmle.Tree(ctx, locs, leaf_size=32, aca_eps=1e-8, max_rank=48, oversample=16)
        t0 = time.time()
        th_d, ll_d, it_d, ev_d, st_d = tree.fit(Z, DEFAULT_THETA0, **fit_kw)
        t_d = time.time() - t0
        th0, steps, fb = model.start(locs, Z)
        t0 = time.time()
        th_l, ll_l, it_l, ev_l, st_l = tree.fit(Z, th0, step=steps, **fit_kw)
        t_l = time.time() - t0
        tree.close()
        rows.append({"n": int(locs.shape[0]), "theta": th, "fallback": fb,
                     "default": {"theta": th_d, "L": ll_d, "iters": it_d, "evals": ev_d,
                                 "status": st_d, "s": t_d},
                     "learned": {"theta0": th0, "theta": th_l, "L": ll_l, "iters": it_l,
                                 "evals": ev_l, "status": st_l, "s": t_l}})
    tot = {k: {f: sum(r[k][f] for r in rows) for f in ("iters", "evals", "s")}
           for k in ("default", "learned")}
    return rows, tot


def main():
    """Train on simulated fields, then fit held-out fields from the default
    and from the learned start; prints one JSON summary.

        python -m paper_2104_07146_gb300.learned_start [--train 200000] [--time 600]
                                                       [--test 6] [--n 2000]

    Training fields: n log-uniform in [4096, 16384], every fourth one 3-D,
    as many of --train as --time seconds of simulation allow.
    """
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=200_000)
    ap.add_argument("--time", type=float, default=600.0)
    ap.add_argument("--test", type=int, default=6)
    ap.add_argument("--n", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=200)
    a = ap.parse_args()
    ctx = hmle.Context()
    t0 = time.time()
    F, T = training_set(ctx, a.train, seed=11, n_range=(4096, 16384), three_d_every=4,
                        time_limit_s=a.time)
    t_data = time.time() - t0
    model = LearnedStart(ctx, seed=1)
    t0 = time.time()
    l0, l1 = model.train(F, T, epochs=a.epochs, batch=64, lr=1e-3, seed=3)
    t_train = time.time() - t0
    fields = [field(ctx, 977, i, a.n) for i in range(a.test)]
    rows, tot = compare_starts(ctx, model, fields)
    err = lambda th, ref: [abs(u - v) for u, v in zip(theta_to_x(th), theta_to_x(ref))]
    out = {"train_fields": int(F.shape[0]), "train_requested": a.train, "data_s": t_data, "train_s": t_train, "loss_first": l0,
           "loss_last": l1, "test_fields": a.test, "n": a.n, "totals": tot,
           "fields": [{"theta_true": r["theta"], "fallback": r["fallback"],
                       "x_err_learned_start": err(r["learned"]["theta0"], r["theta"]),
                       "x_err_default_start": err(DEFAULT_THETA0, r["theta"]),
                       "L_default": r["default"]["L"], "L_learned": r["learned"]["L"],
                       "evals_default": r["default"]["evals"], "evals_learned": r["learned"]["evals"],
                       "s_default": r["default"]["s"], "s_learned": r["learned"]["s"]}
                      for r in rows]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
