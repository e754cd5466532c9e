"""Benchmark of the H-MLE hot path: H-matrix log-likelihood evaluations per
second (Eq. 1 with the Matern covariance of Eq. 2) on one GB300.

One evaluation = Matern tables + ACA assembly of the admissible blocks + the
H-Cholesky leaf sweep with the fused forward solve + log-det / quadratic
form.  One step = one batch of B = 32 evaluations at B distinct theta (the
workload theta and its neighbours in the transformed coordinates of Sec. 5,
as an optimiser's simplex would ask for), run concurrently through
hmle_loglik_batch, for the medium workload: n = 65,536 points in
[0,1]^2 (70 % uniform, 30 % in 8 Gaussian blobs of sd 0.03), Matern
(ell, nu, sigma2, tau2) = (0.05, 0.5, 1, 1e-3), leaf 64, eta 2, eps 1e-6.
The cluster/block trees and the schedule are built once (θ-independent).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  --impl reference times the CPU oracle (dense FP64
Cholesky of the same likelihood) on a bounded subset of the same workload.
Under torchrun (N > 1) every rank evaluates its own replica (the single-field
factorisation does not shard); value is the total over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The batched form runs one stream pair per concurrent evaluation; give the
# context enough hardware work queues that the streams do not share queues
# (must be set before the CUDA context is created).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "H-loglik evals/sec and MLE fit time at n=64k and 2M on 1 GB300 at |ΔL|/n≤1e-6"
WORKLOAD = dict(workload="medium: n=65536 2-D, 70% uniform + 30% in 8 blobs (sd 0.03), Matern "
                "ell=0.05 nu=0.5 sigma2=1 tau2=1e-3, leaf 64, eta 2, ACA eps 1e-6, FP64",
                n=65536, d=2, theta=[0.05, 0.5, 1.0, 1e-3], leaf=64, eta=2.0, eps=1e-6)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07  # SMs x FP64 FMA/clk x 2 flops x GHz (max clock)
# DRAM bytes per launch of the FP64 k_rows in this bench's batched step:
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of five
# launches, mean (8,458,496 + 6,790,656 + 5,495,040 + 3,072,512 + 24,783,872
# read, nothing written)
K_ROWS_DRAM_BYTES = 9_720_115


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, name in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(name)
            except Exception:
                pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist(backend="nccl"):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch.distributed as dist
    dist.init_process_group(backend)
    return dist, dist.get_rank(), ws


def reduce_max(dist, values, device="cpu"):
    """The per-rank timings combined as their maximum over ranks (the slowest
    replica sets the whole job's time); no-op on one process."""
    if not dist:
        return list(values)
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def job_rate(ws, units_per_rank, ms_max):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return ws * units_per_rank / (ms_max / 1e3)


def shard(n_tasks, rank, ws):
    """The contiguous range of tasks (fields / theta points) of one rank when
    a batched workload is split over ranks: no data exchange is needed."""
    per, extra = divmod(n_tasks, ws)
    lo = rank * per + min(rank, extra)
    return lo, lo + per + (1 if rank < extra else 0)


def _workload_inputs(n):
    from paper_2104_07146_gb300 import synth
    locs = synth.locations_blobs(n, 2, 0.3, 8, 0.03, seed=1001)
    Z = synth.normal(1002, n)
    return locs, Z


def run_gpu(args):
    import torch
    from paper_2104_07146_gb300 import hmle
    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    w = WORKLOAD
    n = w["n"]
    locs, Z = _workload_inputs(n)
    stream = torch.cuda.current_stream()
    ctx = hmle.Context(stream)
    tree = hmle.Tree(ctx, locs, leaf_size=w["leaf"], eta=w["eta"], aca_eps=w["eps"],
                     precision=args.precision, **({"batch_size": args.batch_size} if args.batch_size else {}))
    Zd = torch.from_numpy(Z).to(f"cuda:{local}")           # resident input
    Zh = torch.from_numpy(Z).pin_memory()                   # host input for e2e
    theta = tuple(w["theta"])
    thetas = batch_thetas(theta, args.batch)
    prof = hmle.Profiler(ctx, args.roofline_kernel)

    def step(z):
        ll, st = tree.loglik_batch(thetas, z, concurrency=args.batch)
        assert all(s == 0 for s in st), st
        return ll

    for _ in range(args.warmup):
        step(Zd)
    # one single evaluation: its latency, and the launches of one evaluation
    ll1, info = tree.loglik(theta, Zd)
    t0 = time.time()
    ll1, info = tree.loglik(theta, Zd)
    single_ms = (time.time() - t0) * 1e3
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        ll = step(Zd)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # kernels of one step: the sweeps of the ceil(B / batch_size) sub-batches
    # (each launch serves batch_size evaluations, gridDim.z) plus, per
    # evaluation, the three assembly launches, the permutation of Z and the
    # final reduction (a single evaluation's count holds those five)
    nsub = -(-args.batch // tree.opts.batch_size)
    launches = args.steps * (nsub * (info.kernel_launches - 5) + 5 * args.batch)
    # roofline kernel: every launch of it in one batched step (B evaluations
    # per launch, the bench's launch configuration), bracketed by CUDA events
    # on its launching stream; the step's sweep is then launched directly,
    # since events inside a captured graph cannot be read back
    prof.enable(True)
    step(Zd)
    dom = prof.read()
    prof.enable(False)
    dom["mode"] = ("one batched step of %d evaluations (%d per launch), direct launches"
                   % (args.batch, tree.opts.batch_size))
    # e2e: host Z (pinned) through the C ABI; the copy in and the result out
    # are inside the timed region
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        ll_e2e = step(Zh.numpy())
    e3.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e2.elapsed_time(e3)
    clk = clocks.stop()
    ms, ms_e2e = reduce_max(dist, [ms, ms_e2e], device=f"cuda:{local}")
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    phases = phase_rooflines(tree, theta, Z, single_ms, info.flops)
    value = job_rate(ws, args.steps * args.batch, ms)
    e2e = job_rate(ws, args.steps * args.batch, ms_e2e)
    achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e9 if dom["ms"] > 0 else None
    peaks = _peaks()
    out = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "f64", 1: "f64 + tensor-core products (3 BF16 slices, f32 accumulation)",
                  2: "f64 + tensor-core products (2 BF16 slices, f32 accumulation)"}[args.precision],
        "data": "synthetic",
        "config": {**{k: v for k, v in WORKLOAD.items()},
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2": "working set %.1f GB > 129 MB L2 (no flush needed)"
                         % (tree.info().lowrank_words * 8 / 1e9)},
        "batch": args.batch, "single_eval_ms": single_ms,
        "loglik": ll1, "logdet": info.logdet, "quad": info.quad,
        "ranks": {"max_c": info.max_rank_c, "max_l": info.max_rank_l, "mean_l": info.mean_rank_l},
        "e2e": {"value": e2e, "unit": "evals/s", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 24 * args.batch},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": dom["name"], "achieved": achieved,
                     "launches": dom["launches"], "kernel_ms": dom["ms"],
                     "flops_per_launch": dom["flops"] / max(dom["launches"], 1),
                     "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                     "frac": (achieved / FP64_PEAK_GFLOPS) if achieved else None,
                     "traffic": K_ROWS_DRAM_BYTES if args.precision == 0 else None,
                     "traffic_source": (
                         "dram__bytes_read.sum + dram__bytes_write.sum of 5 launches of the FP64 "
                         "k_rows in this command's first step, mean per launch (3.1-24.8 MB read, "
                         "0 written; profiles/k_rows_dram_bench_medium_n65536.md)"
                         if args.precision == 0 else "not captured for this form"),
                     "note": "FP64 ALU peak from 152 SMs x 2 FMA/clk x 2070 MHz "
                             "(measured FMA loop: 1254.6 GFLOP/s); algorithmic FP64 flops of "
                             "the kernel's launches (plan x ranks of every evaluation) over "
                             "their summed CUDA-event durations: " + dom["mode"]},
        "step_roofline": {
            "bound": "alu", "flops_per_eval": info.flops,
            "achieved": info.flops * value / ws / 1e9 if info.flops else None,
            "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
            "frac": (info.flops * value / ws / 1e9 / FP64_PEAK_GFLOPS) if info.flops else None,
            "note": "whole batched step on one GPU: algorithmic flops of one evaluation (plan "
                    "x ranks) x evaluations/s, against the FP64 ALU peak"},
        "phases": phases,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_sample_n)
    if not args.no_fit:
        out["fit"] = fit_small(ctx, not args.no_cpu_baseline)
    if args.forms:
        out["forms"] = other_forms(ctx, locs, Z, Zd, thetas, args.batch, value)
    print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


SMALL = dict(n=2000, theta=(0.1, 0.5, 1.0, 0.01), theta0=(0.2, 1.0, 0.5, 0.05), leaf=32, eps=1e-8)
# (default rank capacity 32 and oversampling 8, as the small-configuration parity tests use)


def fit_small(ctx, with_oracle):
    """The MLE of the small configuration: n = 2000 uniform points, Z = L xi
    (dense factor of C at theta), Nelder-Mead of all 4 parameters from theta0
    (Sec. 2; tolerance 1e-4, at most 400 iterations); the oracle's own fit of
    the same field timed beside it on the host cores."""
    from paper_2104_07146_gb300 import hmle, synth
    import oracle
    c = SMALL
    locs = synth.locations_uniform(c["n"], 2, seed=1000)
    Z = oracle.simulate(locs, c["theta"], synth.normal(1001, c["n"]))
    tree = hmle.Tree(ctx, locs, leaf_size=c["leaf"], aca_eps=c["eps"])
    t0 = time.time()
    th, ll, it, nev, st = tree.fit(Z, c["theta0"])
    dt = time.time() - t0
    out = {"config": "small: n=2000 uniform, theta=(0.1, 0.5, 1, 0.01), Z = L xi, leaf 32, "
                     "eps 1e-8, Nelder-Mead from (0.2, 1, 0.5, 0.05)",
           "gpu_s": dt, "iterations": it, "evaluations": nev, "status": st,
           "theta_hat": th, "loglik_hat": ll,
           "loglik_hat_oracle": oracle.loglik_dense(locs, Z, th)[0]}
    t0 = time.time()
    th_p, ll_p, it_p, nev_p, st_p = tree.fit(Z, c["theta0"], profiled=True)
    out["profiled"] = {"gpu_s": time.time() - t0, "iterations": it_p, "evaluations": nev_p,
                       "status": st_p, "theta_hat": th_p, "loglik_hat": ll_p,
                       "note": "sigma2 profiled out: Nelder-Mead over (ell, nu, tau2/sigma2)"}
    if with_oracle:
        t0 = time.time()
        th_c, ll_c, it_c, nev_c = oracle.fit(locs, Z, c["theta0"])
        out["cpu_oracle"] = {"s": time.time() - t0, "iterations": it_c, "evaluations": nev_c,
                             "theta_hat": th_c, "loglik_hat": ll_c, "cores": os.cpu_count()}
    tree.close()
    return out


def other_forms(ctx, locs, Z, Zd, thetas, B, fp64_value):
    """The mixed-precision and multi-instance batched forms on the same GPU,
    reported against the plain FP64 batched form of this run."""
    import torch
    from paper_2104_07146_gb300 import hmle, synth
    w = WORKLOAD
    res = {"fp64_batched_evals_per_s": fp64_value}
    for prec, key in ((1, "mixed_fp32_pcg"), (2, "mixed_bf16_pcg")):
        # the products on the tensor cores with three (24-bit) or two (16-bit)
        # BF16 slices per operand; the quadratic form by PCG
        tm = hmle.Tree(ctx, locs, leaf_size=w["leaf"], eta=w["eta"], aca_eps=w["eps"], precision=prec)
        ll_m, st = tm.loglik_batch(thetas, Zd, concurrency=B)          # buffers, graphs
        torch.cuda.synchronize()
        t0 = time.time()
        ll_m, st = tm.loglik_batch(thetas, Zd, concurrency=B)
        dt = time.time() - t0
        ll1, info = tm.loglik(thetas[0], Zd)
        t0 = time.time()
        ll1, info = tm.loglik(thetas[0], Zd)
        single = time.time() - t0
        res[key] = {"evals_per_s": B / dt, "single_eval_ms": single * 1e3, "pcg_iters": info.pcg_iters,
                    "pcg_relres": info.pcg_relres, "loglik": ll1, "logdet": info.logdet,
                    "status": [int(x) for x in st]}
        tm.close()
    # multi-instance: 8 fields of uneven n (2-D and 3-D), 4 theta each, one call
    fields = []
    for i in range(8):
        n = int(2048 * 2 ** (4 * synth.uniform(500 + i, 1)[0]))      # log-uniform in [2048, 32768]
        d = 2 if i % 2 == 0 else 3
        pts = (synth.locations_uniform(n, 2, seed=600 + i) if d == 2
               else synth.uniform(700 + i, 3 * n).reshape(n, 3))
        fields.append((hmle.Tree(ctx, pts, leaf_size=64, aca_eps=1e-6, max_rank=48, oversample=16),
                       synth.normal(800 + i, n), n, d))
    tasks = [(t, (0.05 + 0.01 * k, 0.5 + 0.1 * k, 1.0, 1e-3), z) for (t, z, n, d) in fields
             for k in range(4)]
    ctx.loglik_multi(tasks, concurrency=16)
    t0 = time.time()
    ll, st = ctx.loglik_multi(tasks, concurrency=16)
    dt = time.time() - t0
    ok = [k for k, x in enumerate(st) if x == 0]
    for k in ok:                                                  # graphs of the single path
        tasks[k][0].loglik(tasks[k][1], tasks[k][2])
    t0 = time.time()
    for k in ok:                                                  # the same tasks one call each
        tasks[k][0].loglik(tasks[k][1], tasks[k][2])
    dt_loop = time.time() - t0
    # the same call with failed tasks retried on derived trees (larger rank
    # capacity, then a looser accuracy), reported per task
    t0 = time.time()
    ll_r, st_r, retry = ctx.loglik_multi_retry(tasks, concurrency=16, max_retries=3)
    dt_r = time.time() - t0
    res["multi_instance"] = {"fields": [(n, d) for (_, _, n, d) in fields], "tasks": len(tasks),
                             "evals_per_s": len(tasks) / dt,
                             "looped_evals_per_s": len(ok) / dt_loop if ok else None,
                             "points_evals_per_s": sum(n for (_, _, n, _) in fields) * 4 / dt,
                             "status": [int(x) for x in st],
                             "with_retries": {
                                 "call_s": dt_r, "status": [int(x) for x in st_r],
                                 "ok": int(sum(1 for x in st_r if x == 0)),
                                 "first_try_bits_equal": bool(all(
                                     ll_r[k] == ll[k] for k in ok)),
                                 "retried": [dict(task=k, **r) for k, r in enumerate(retry) if r["retries"]]}}
    for t, _, _, _ in fields:
        t.close()
    return res


def phase_rooflines(tree, theta, Z, single_ms, sweep_flops):
    """Time and algorithmic work of the phases of one evaluation: the
    assembly of C~ (a3 + a4) and one solve through a stored factor (a10 +
    a11, the persistent sweeps), each the median of three synchronised
    library calls, with the work from hmle_phase_work; the factorisation
    sweep with its fused forward solve (a5-a10) is the single evaluation
    minus the assembly.  A failure here is reported in the line, not raised."""
    import statistics
    try:
        hm = tree.assemble(theta)
        f = hm.factor(Z)
        f.solve(Z)                                   # warm-up of the persistent sweeps
        fa, sb = f.phase_work()
        ta, ts = [], []
        for _ in range(3):
            t0 = time.perf_counter()
            h2 = tree.assemble(theta)
            ta.append(time.perf_counter() - t0)
            h2.close()
        for _ in range(3):
            t0 = time.perf_counter()
            f.solve(Z)
            ts.append(time.perf_counter() - t0)
        f.close()
        hm.close()
        t_a, t_s = statistics.median(ta), statistics.median(ts)
        t_sw = single_ms / 1e3 - t_a
        hbm = _peaks().get("hbm_gbs")

        def row(sec, work, unit, peak, bound, **kw):
            rate = work / sec / 1e9 if sec > 0 else None
            return {"s": sec, "work": work, "achieved": rate, "unit": unit, "peak": peak,
                    "frac": rate / peak if (rate and peak) else None, "bound": bound, **kw}
        return {
            "assembly": row(t_a, fa, "GFLOP/s", FP64_PEAK_GFLOPS, "alu",
                            work_unit="FP64 flops (3d + 68 per Matern entry, ACA updates)"),
            "sweep": row(t_sw, sweep_flops, "GFLOP/s", FP64_PEAK_GFLOPS, "alu",
                         work_unit="FP64 flops (plan x ranks)"),
            "solve": row(t_s, sb, "GB/s", hbm, "hbm",
                         work_unit="bytes of the factor read by the forward and backward sweeps",
                         note="limited by the grid barriers of the leaf chain, not by HBM"),
            "note": "wall times of synchronised library calls (median of 3); sweep = single "
                    "evaluation - assembly; solve peak = measured HBM copy (MEASURED_PEAKS.json)"}
    except Exception as e:                           # keep the bench line
        return {"error": repr(e)}


def batch_thetas(theta, B):
    """The workload theta and B - 1 neighbours: +-0.25 along each transformed
    coordinate of Sec. 5 (sigma0, ell0, nu0, tau0), cycling."""
    ell, nu, s2, t2 = theta
    x = [-math.log(math.sqrt(s2) / 2.0) / math.log(1.1), -math.log(ell) / math.log(1.5),
         -math.log(nu) / math.log(1.2), -math.log(math.sqrt(t2)) / math.log(2.0)]
    out = [tuple(theta)]
    k = 0
    while len(out) < B:
        y = list(x)
        y[k % 4] += 0.25 * (1 if (k // 4) % 2 == 0 else -1) * (1 + k // 8)
        sig = 2.0 / 1.1 ** y[0]
        tau = 1.0 / 2.0 ** y[3]
        out.append((1.0 / 1.5 ** y[1], 1.0 / 1.2 ** y[2], sig * sig, tau * tau))
        k += 1
    return out


def _oracle_seconds(n_sub):
    """Seconds of one dense oracle evaluation (Eq. 1) on the first n_sub points
    of the workload, and on the first n_sub / 2."""
    import oracle
    locs, Z = _workload_inputs(WORKLOAD["n"])
    theta = tuple(WORKLOAD["theta"])
    out = []
    for m in (n_sub // 2, n_sub):
        t0 = time.time()
        oracle.loglik_dense(locs[:m], Z[:m], theta)
        out.append(time.time() - t0)
    return out


def extrapolate_seconds(t_half, t_full, n_sub, n):
    """The dense oracle's time at n from its times at n_sub / 2 and n_sub:
    t(m) = a m^2 + b m^3 (the matrix generation and the forward substitution
    grow with m^2, the Cholesky with m^3) through the two points.  When the
    two times do not fit that form (b <= 0 or a < 0, timing noise), the
    n_sub time alone scaled by (n / n_sub)^3.  Returns (seconds, how)."""
    b3 = (t_full - 4.0 * t_half) / 4.0      # b (n_sub / 2)^3
    a2 = t_half - b3                        # a (n_sub / 2)^2
    r = n / (n_sub / 2.0)
    if b3 > 0.0 and a2 >= 0.0:
        return a2 * r ** 2 + b3 * r ** 3, "a m^2 + b m^3 through both sizes"
    return t_full * (n / n_sub) ** 3, "m^3 from the larger size"


def cpu_baseline(n_sub):
    """The oracle as it stands (dense FP64) on two subsets of the workload,
    extrapolated to n = 65,536 (extrapolate_seconds)."""
    t_half, t_full = _oracle_seconds(n_sub)
    est, how = extrapolate_seconds(t_half, t_full, n_sub, WORKLOAD["n"])
    return {"value": 1.0 / est, "unit": "evals/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": "one dense evaluation on the first %d and %d points of the workload (%.1f s, %.1f s), "
                      "extrapolated to n=%d by %s (%.0f s)" % (n_sub // 2, n_sub, t_half, t_full,
                                                              WORKLOAD["n"], how, est)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_sub = args.cpu_sample_n
    for _ in range(args.warmup):
        _oracle_seconds(n_sub)
    halves, fulls = [], []
    for _ in range(max(args.steps, 1)):
        th, tf = _oracle_seconds(n_sub)
        halves.append(th)
        fulls.append(tf)
    t_half, t_full = sum(halves) / len(halves), sum(fulls) / len(fulls)
    est, how = extrapolate_seconds(t_half, t_full, n_sub, WORKLOAD["n"])
    v = 1.0 / est
    sample = ("dense FP64 oracle on the first %d and %d points per step (%.2f s, %.2f s), extrapolated "
              "to n=%d by %s" % (n_sub // 2, n_sub, t_half, t_full, WORKLOAD["n"], how))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": est * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": WORKLOAD,
        "cpu_baseline": {"value": v, "unit": "evals/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-sample-n", type=int, default=16384)
    ap.add_argument("--batch", type=int, default=32,
                    help="concurrent theta evaluations per step (hmle_loglik_batch)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fit", action="store_true", help="skip the small-configuration MLE fit")
    ap.add_argument("--forms", action="store_true",
                    help="also report the mixed-precision and multi-instance batched forms")
    ap.add_argument("--batch-size", type=int, default=0,
                    help="evaluations per launch of each sweep kernel (0: the library default)")
    ap.add_argument("--precision", type=int, default=0,
                    help="0 FP64 (the headline form); 1, 2: the mixed forms (tensor-core products, PCG)")
    ap.add_argument("--roofline-kernel", default="k_rows",
                    help="sweep kernel whose launches are timed for the roofline line")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
