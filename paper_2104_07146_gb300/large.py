"""The large configuration: one H-matrix log-likelihood evaluation at
n = 2,000,000 (80 % uniform + 20 % in 8 Gaussian blobs, Matern ell = 0.02,
nu = 0.5, sigma2 = 1, tau2 = 1e-3, leaf 128, eta 2, ACA eps 1e-5).

    python -m paper_2104_07146_gb300.large [--n 2000000] [--nu 0.5] [--precision 0|1]

Prints one JSON line: tree build time, the times of two evaluations (the
first includes buffer allocation and graph capture), log|C~|, Z^T C~^-1 Z,
ranks, the algorithmic flops of the sweep and the device memory in use.  Z is
seeded white noise: the time of an evaluation does not depend on Z, and a
field simulated at this size would need a second, tighter factorisation.
"""
from __future__ import annotations

import argparse
import json
import time

from . import hmle, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=synth.LARGE["n"])
    ap.add_argument("--nu", type=float, default=0.5)
    ap.add_argument("--precision", type=int, default=0)
    a = ap.parse_args()
    import torch
    c = synth.LARGE
    locs = synth.locations_blobs(a.n, 2, c["frac_blob"], c["nblobs"], c["sd"], c["seed"])
    Z = synth.normal(c["seed"] + 1, a.n)
    th = (c["theta"][0], a.nu, c["theta"][2], c["theta"][3])
    ctx = hmle.Context()
    t0 = time.time()
    tree = hmle.Tree(ctx, locs, leaf_size=c["leaf"], eta=c["eta"], aca_eps=c["aca_eps"],
                     max_rank=48, oversample=16, precision=a.precision)
    t_tree = time.time() - t0
    ti = tree.info()
    times = []
    for _ in range(2):
        t0 = time.time()
        ll, info = tree.loglik(th, Z)
        times.append(time.time() - t0)
    free, total = torch.cuda.mem_get_info()
    print(json.dumps({
        "config": "large: n=%d, 80%% uniform + 20%% in 8 blobs (sd 0.03), Matern ell=%g nu=%g "
                  "sigma2=1 tau2=1e-3, leaf %d, eta %g, ACA eps %g, rank capacity 48, "
                  "oversampling 16, %s; Z white noise"
                  % (a.n, th[0], a.nu, c["leaf"], c["eta"], c["aca_eps"],
                     "mixed FP32 + PCG" if a.precision else "FP64"),
        "tree_build_s": t_tree, "leaves": ti.n_leaves, "dense_blocks": ti.n_dense,
        "lowrank_blocks": ti.n_lowrank, "eval_s": times, "loglik": ll, "logdet": info.logdet,
        "quad": info.quad, "max_rank_c": info.max_rank_c, "max_rank_l": info.max_rank_l,
        "mean_rank_l": info.mean_rank_l, "pcg_iters": info.pcg_iters,
        "sweep_gflop": info.flops / 1e9, "kernel_launches": info.kernel_launches,
        "device_gb_in_use": (total - free) / 1e9, "device_gb_total": total / 1e9}))


if __name__ == "__main__":
    main()
