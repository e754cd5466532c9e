"""The batched configuration: many independent fields of uneven size, many
theta trial points per field, evaluated in one call (hmle_loglik_multi).

    python -m paper_2104_07146_gb300.batched_fields [--fields 256] [--trials 16]
                                                    [--precision 1] [--concurrency 16]

Fields: n log-uniform in [2,048, 32,768]; half 2-D (uniform in [0,1]^2), half
3-D (uniform in [0,1]^3); a theta per field with ell and tau2 log-uniform in
[0.02, 0.3] and [1e-4, 1e-1], nu and sigma2 uniform in [0.3, 2.5] and
[0.5, 2]; Z seeded white noise (the time of an evaluation does not depend on
Z).  Trial points: the field's theta and its neighbours at +-0.25 along the
transformed coordinates of Sec. 5, as a simplex or a line search asks for.
Trees: leaf 64, eta 2, ACA eps 1e-6, rank capacity 48, oversampling 16; the
products in the requested precision (default: three BF16 slices on the
tensor cores, PCG for the quadratic form).

The call is hmle_loglik_multi_retry: a task that fails (rank overflow, or
a mixed-form PCG that does not converge) is evaluated again on a tree derived
from its own, one rung of the retry ladder further each time.

Prints a JSON line after the trees are built and one after the call, then
the summary line: the tree-build time, the one call's time and tasks/s,
the per-status counts after the retries and the rungs the retried tasks
ended on, and the tasks of the first fields run again in one call and one
call each (looped, after one warm-up evaluation per tree) for comparison,
with the number of first-attempt results bit-equal to the single
evaluation's.
"""
from __future__ import annotations

import argparse
import json
import math
import time

from . import hmle, synth
from .learned_start import theta_to_x, x_to_theta


def field_theta(seed: int, i: int):
    u = synth.uniform(seed * 1_000_003 + i, 4)
    ell = 0.02 * (0.3 / 0.02) ** u[0]
    nu = 0.3 + 2.2 * u[1]
    s2 = 0.5 + 1.5 * u[2]
    t2 = 1e-4 * (1e-1 / 1e-4) ** u[3]
    return (float(ell), float(nu), float(s2), float(t2))


def trial_points(theta, k: int):
    """theta and k - 1 neighbours: +-0.25 along each transformed coordinate,
    cycling; neighbours outside the admissible range are skipped."""
    x = theta_to_x(theta)
    out, j = [tuple(theta)], 0
    while len(out) < k and j < 64:
        y = list(x)
        y[j % 4] += 0.25 * (1 if (j // 4) % 2 == 0 else -1) * (1 + j // 8)
        th = x_to_theta(y)
        if th is not None:
            out.append(th)
        j += 1
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--fields", type=int, default=256)
    ap.add_argument("--trials", type=int, default=16)
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--concurrency", type=int, default=16)
    ap.add_argument("--looped-fields", type=int, default=4)
    ap.add_argument("--seed", type=int, default=31)
    ap.add_argument("--retries", type=int, default=3)
    a = ap.parse_args()
    ctx = hmle.Context()
    fields = []
    t0 = time.time()
    for i in range(a.fields):
        u = synth.uniform(a.seed * 7919 + i, 1)[0]
        n = int(2048 * 16 ** u)                    # log-uniform in [2048, 32768]
        d = 2 if i % 2 == 0 else 3
        locs = synth.uniform(a.seed * 104729 + i, d * n).reshape(n, d)
        tree = hmle.Tree(ctx, locs, leaf_size=64, eta=2.0, aca_eps=1e-6, max_rank=48, oversample=16,
                         precision=a.precision)
        fields.append((tree, synth.normal(a.seed * 15485863 + i, n), n, d, field_theta(a.seed, i)))
    t_tree = time.time() - t0
    tasks = [(tree, th, Z) for (tree, Z, n, d, th0) in fields for th in trial_points(th0, a.trials)]
    print(json.dumps({"phase": "trees", "fields": a.fields, "tasks": len(tasks), "tree_build_s": t_tree}),
          flush=True)
    t0 = time.time()
    ll, st, retry = ctx.loglik_multi_retry(tasks, concurrency=a.concurrency, max_retries=a.retries)
    dt = time.time() - t0
    counts = {}
    for s in st:
        counts[int(s)] = counts.get(int(s), 0) + 1
    rungs = {}
    for r in retry:
        if r["retries"]:
            key = "max_rank %d, %s, eps %g" % (r["max_rank"], "FP64" if r["precision"] == 0 else
                                               "mixed %d" % r["precision"], r["aca_eps"])
            rungs[key] = rungs.get(key, 0) + 1
    print(json.dumps({"phase": "call", "call_s": dt, "tasks_per_s": len(tasks) / dt, "status_counts": counts,
                      "retry_rungs": rungs}), flush=True)
    # the first fields' tasks once more: in one call, then one call each
    sub = [k for k, t in enumerate(tasks) if any(t[0] is f[0] for f in fields[:a.looped_fields])]
    t0 = time.time()
    ctx.loglik_multi([tasks[k] for k in sub], concurrency=a.concurrency)
    dt_sub = time.time() - t0
    for f in fields[:a.looped_fields]:           # buffers and graph of the single path
        try:
            f[0].loglik(f[4], f[1])
        except hmle.HmleError:
            pass
    single = {}
    t0 = time.time()
    for k in sub:
        try:
            single[k] = tasks[k][0].loglik(tasks[k][1], tasks[k][2])[0]
        except hmle.HmleError:
            pass
    dt_loop = time.time() - t0
    # a task that succeeded at its first attempt in the one call gives the
    # same bits as the single evaluation (same kernels, same order of sums)
    cmp = [k for k in sub if k in single and st[k] == 0 and retry[k]["retries"] == 0]
    bits_equal = sum(1 for k in cmp if single[k] == ll[k])
    ns = [f[2] for f in fields]
    print(json.dumps({
        "config": "batched: %d fields, n log-uniform in [2048, 32768] (%d..%d), half 2-D / half 3-D, "
                  "%d theta per field, leaf 64, eps 1e-6, rank capacity 48, precision %d, concurrency %d, "
                  "up to %d retries" % (a.fields, min(ns), max(ns), a.trials, a.precision, a.concurrency,
                                        a.retries),
        "tasks": len(tasks), "tree_build_s": t_tree, "call_s": dt, "tasks_per_s": len(tasks) / dt,
        "points_evals_per_s": sum(f[2] for f in fields) * a.trials / dt,
        "status_counts": counts, "retried": sum(1 for r in retry if r["retries"]),
        "retry_rungs": rungs,
        "subset": {"fields": a.looped_fields, "tasks": len(sub),
                   "one_call_tasks_per_s": len(sub) / dt_sub if dt_sub > 0 else None,
                   "looped_tasks_per_s": len(sub) / dt_loop if dt_loop > 0 else None,
                   "bits_equal_to_single": "%d of %d" % (bits_equal, len(cmp))},
        "ll_finite": int(sum(1 for v in ll if math.isfinite(v)))}))
    for f in fields:
        f[0].close()


if __name__ == "__main__":
    main()
