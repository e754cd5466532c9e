"""Per-kernel time and algorithmic FP64 throughput of one evaluation.

    python -m paper_2104_07146_gb300.profile_kernels [--n 65536] [--leaf 64] [--eps 1e-6] [--nu 0.5]
                                                     [--precision 0|1] [--single]

For every kernel kind of the factorisation sweep, one evaluation is run with
that kernel's launches bracketed by CUDA events on their own stream
(hmle_profile_select); the summed launch time is reported with the kernel's
algorithmic FP64 flops (tallied from the schedule and the evaluation's
ranks) and the fraction of the FP64 peak (152 SMs x 2 FMA/clk x 2.07 GHz).
Workload: the medium configuration's point set (uniform + Gaussian blobs).
"""
from __future__ import annotations

import argparse
import time

from paper_2104_07146_gb300 import hmle, synth

KERNELS = ["k_gram", "k_side_t", "k_side_s", "k_rows", "k_tsqr_part", "k_tsqr_final",
           "k_tall_apply", "k_cholqr_part", "k_cholqr_final", "k_dense_pair", "k_dense_reduce",
           "k_potrf", "k_trsm", "k_wsolve", "k_htask", "k_updrow"]
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=65536)
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--eps", type=float, default=1e-6)
    ap.add_argument("--nu", type=float, default=0.5)
    ap.add_argument("--leaf-lowrank", type=int, default=0)
    ap.add_argument("--precision", type=int, default=0, help="0 FP64, 1 mixed FP32 + PCG")
    ap.add_argument("--single", action="store_true",
                    help="one warm-up and one timed evaluation only (for an external profiler)")
    a = ap.parse_args()
    ctx = hmle.Context()
    locs = synth.medium_locations(a.n)
    tree = hmle.Tree(ctx, locs, leaf_size=a.leaf, aca_eps=a.eps, leaf_lowrank=a.leaf_lowrank,
                     precision=a.precision)
    Z = synth.normal(7, a.n)
    th = (0.05, a.nu, 1.0, 1e-3)
    tree.loglik(th, Z)
    t0 = time.time()
    ll, info = tree.loglik(th, Z)
    wall = time.time() - t0
    print("n %d  one evaluation %.3f s  %d kernel launches  L = %.6f" % (a.n, wall, info.kernel_launches, ll))
    if a.single:
        return
    rows, tot = [], 0.0
    for name in KERNELS:
        p = hmle.Profiler(ctx, name)
        p.enable(True)
        tree.loglik(th, Z)
        r = p.read()
        p.enable(False)
        rows.append(r)
        tot += r["ms"]
    print("| kernel | launches | ms | share | GFLOP | GFLOP/s | % FP64 peak |")
    print("|---|---:|---:|---:|---:|---:|---:|")
    for r in sorted(rows, key=lambda x: -x["ms"]):
        gf = r["flops"] / (r["ms"] / 1e3) / 1e9 if r["ms"] > 0 else 0.0
        print("| %s | %d | %.1f | %.1f%% | %.3g | %.1f | %.1f |" % (
            r["name"], r["launches"], r["ms"], 100 * r["ms"] / tot, r["flops"] / 1e9, gf,
            100 * gf / FP64_PEAK_GFLOPS))
    print("sum of kernel time %.1f ms" % tot)


if __name__ == "__main__":
    main()
