"""Per-kernel time and algorithmic FP64 throughput of one evaluation.

    python -m paper_2104_07146_gb300.profile_kernels [--n 65536] [--leaf 64] [--eps 1e-6] [--nu 0.5]
                                                     [--precision 0|1] [--single] [--phases]

For every kernel kind of the factorisation sweep, one evaluation is run with
that kernel's launches bracketed by CUDA events on their own stream
(hmle_profile_select); the summed launch time is reported with the kernel's
algorithmic FP64 flops (tallied from the schedule and the evaluation's
ranks) and the fraction of the FP64 peak (152 SMs x 2 FMA/clk x 2.07 GHz).
Workload: the medium configuration's point set (uniform + Gaussian blobs).

--phases prints a per-phase table instead: the assembly of C~ (a3 + a4), the
factorisation sweep with its fused forward solve (a5-a10) and one solve
through a stored factor (a10 + a11, the persistent sweeps), each with its
wall time (synchronised library calls, median of three) and algorithmic work
(hmle_phase_work, hmle_eval_info.flops) against the FP64 peak or the
measured HBM copy bandwidth.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import time

from paper_2104_07146_gb300 import hmle, synth

KERNELS = ["k_gram", "k_side_t", "k_side_s", "k_rows", "k_tsqr_part", "k_tsqr_final",
           "k_tall_apply", "k_cholqr_part", "k_cholqr_final", "k_dense_pair", "k_dense_reduce",
           "k_potrf", "k_trsm", "k_wsolve", "k_htask", "k_updrow"]
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07


def hbm_peak_gbs():
    """Measured copy bandwidth of this GPU type (MEASURED_PEAKS.json at the
    repository root), else the recipe's fallback figure."""
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def phases(tree, th, Z, eval_s, info, reps=3):
    hm = tree.assemble(th)
    f = hm.factor(Z)
    f.solve(Z)                                   # warm-up of the persistent sweeps
    fa, sb = f.phase_work()
    ta, ts = [], []
    for _ in range(reps):
        t0 = time.perf_counter()
        h2 = tree.assemble(th)
        ta.append(time.perf_counter() - t0)
        h2.close()
    for _ in range(reps):
        t0 = time.perf_counter()
        f.solve(Z)
        ts.append(time.perf_counter() - t0)
    t_asm, t_sol = statistics.median(ta), statistics.median(ts)
    t_sweep = eval_s - t_asm
    hbm, kind = hbm_peak_gbs()
    print("| phase | s | algorithmic work | rate | % of peak |")
    print("|---|---:|---:|---:|---:|")
    for name, t, work, unit, peak in [
            ("assembly of C~ (a3 + a4)", t_asm, fa / 1e9, "GFLOP", FP64_PEAK_GFLOPS),
            ("factorisation sweep + fused forward solve (a5-a10)", t_sweep, info.flops / 1e9, "GFLOP",
             FP64_PEAK_GFLOPS),
            ("solve through the stored factor (a10 + a11)", t_sol, sb / 1e9, "GB", hbm)]:
        rate = work / t if t > 0 else 0.0
        print("| %s | %.4f | %.4g %s | %.4g %s/s | %.2f%% |" % (name, t, work, unit, rate, unit,
                                                           100 * rate / peak))
    print("peaks: FP64 %.1f GFLOP/s (unit counts x max clock); HBM %.1f GB/s (%s copy)" % (
        FP64_PEAK_GFLOPS, hbm, kind))
    print("sweep time = one evaluation (%.3f s) - assembly" % eval_s)


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
    ap.add_argument("--phases", action="store_true",
                    help="the per-phase table (assembly, sweep, solve) instead of the kernel table")
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
    if a.phases:
        phases(tree, th, Z, wall, info)
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
