#!/usr/bin/env python
"""Benchmark: Acc-Sinkhorn time to marginal L1 1e-6 on one GB300.

Workload (stored cost): n = m = 16384, X and Y from 8-component Gaussian
mixtures in R^3 (sigma 0.05, means uniform in [0,1]^3), dense FP32 squared-
Euclidean cost scaled to max 1 (1 GiB), Dirichlet(1) marginals, eps = 1e-3,
tol = 1e-6 (seeded, synthetic; the paper's images and word vectors are not
available, these inputs stand in for them).

One step = one complete solve to tol through the C-ABI (accsink_solve) with
the inputs resident in HBM. The cost (1 GiB) is larger than L2 (129 MB), so
every pass streams it from HBM; no L2 flush is needed between steps.

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
on the same workload instead: one full Acc solve to tol (the value) and
single S evaluations (the steps).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 16384
EPS = 1e-3
TOL = 1e-6
SEED = 0
METRIC = "time to marginal L1 1e-6, Acc vs plain Sinkhorn on 1 GB300; HBM GB/s; p50/p99 latency"
WORKLOAD = ("gmm8-r3 stored sqeuclid cost n=m=16384 (1 GiB FP32, max 1), Dirichlet(1) "
            "marginals, eps=1e-3, tol=1e-6")


def bench_config(n):
    """The workload description both arms print (identical dicts)."""
    return {"workload": WORKLOAD, "n": n, "m": n, "eps": EPS, "tol": TOL,
            "method": "acc (Algorithm 1+2, mu0=0.25, m0=4, y carried across stages; the "
                      "literal hand-over of Algorithm 2 is reported as acc_carry_w)",
            "l2": "inputs larger than L2 (1 GiB cost vs 129 MB L2); no flush",
            "parallelism": "none (one problem per device; replicas across ranks)"}


# Peaks that MEASURED_PEAKS.json does not hold, measured on this GB300 (152
# SMs, SM clock 2070 MHz) with a CUDA-event throughput probe (1216 CTAs x 256
# threads, 8 independent dependency chains per thread, best of 5): MUFU
# ex2.approx.ftz.f32 and FP32 FFMA lane operations per second.
MEASURED_EX2_PER_S = 9.983e12
MEASURED_FFMA_PER_S = 3.906e13


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def measured_bf16_tflops():
    """Dense bf16 tensor peak (cuBLAS burst) from MEASURED_PEAKS.json, else the
    fallback figure."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["bf16_tflops"])
    except Exception:
        return 1900.0


def profile_traffic(kernel_file: str, profile_name: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (its sha256 is recorded in the summary)."""
    src = os.path.join(ROOT, "paper_2605_30267_gb300", "csrc", kernel_file)
    prof = os.path.join(ROOT, "profiles", profile_name)
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        fields = {}
        for line in open(prof):
            if ":" in line:
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        if fields.get("source_sha256") != sha:
            return None
        return float(fields["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running."""

    def __init__(self):
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", "0", f"--query-gpu={q}",
                                           "--format=csv,noheader,nounits", "-lms", "200"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                          text=True)
        except Exception:
            self._proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
        time.sleep(0.05)
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if s[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def percentile(v, q):
    v = sorted(v)
    if not v:
        return None
    k = (len(v) - 1) * q
    lo, hi = int(k), min(int(k) + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


def dist_setup():
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if os.environ.get("ACCSINK_BENCH_GLOO") is None else "gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Max of a host scalar over the ranks (time of the slowest replica)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Replicas only: every rank solves its own independent problem."""
    return SEED + rank


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2605_30267_gb300 import binding as B
    from paper_2605_30267_gb300 import workloads as W

    rank, world = dist_setup()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pr = W.gmm_stored_cost_problem(seed=replica_seed(rank), n=args.n, m=args.n, eps=EPS, tol=TOL)
    C = torch.from_numpy(pr["C"]).to(dev)
    a = torch.from_numpy(pr["a"]).to(dev)
    b = torch.from_numpy(pr["b"]).to(dev)
    ctx = B.Context(local)
    stream = torch.cuda.Stream(dev)
    prob = B.problem_dense(C, a, b)
    f = torch.empty(args.n, dtype=torch.float64, device=dev)
    g = torch.empty(args.n, dtype=torch.float64, device=dev)

    def solve(method, eps, **kw):
        p = B.default_params(eps=eps, tol=TOL, method=method,
                             use_graph=0 if args.host_loop else 1, **kw)
        return ctx.accsink_solve(prob, p, f, g, stream=stream)

    # warm-up (untimed)
    for _ in range(args.warmup):
        solve(B.ACC, EPS)
    torch.cuda.synchronize()

    # ---- timed region: K Acc solves at eps = 1e-3 ----------------------
    clocks = ClockSampler()
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    lat = []
    steps = []
    launches = 0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    ev0.record(stream)
    for k in range(args.steps):
        evs[k][0].record(stream)
        res = solve(B.ACC, EPS)
        evs[k][1].record(stream)
        steps.append(res.sinkhorn_steps)
        # set-up (state, stage table, cost statistics, init, transpose), the
        # loop's three kernels per S evaluation, launched four evaluations per
        # trip of the graph's WHILE node (eight per host round trip in the
        # host loop; the kernels after the stopping step return at once), the
        # final cost pass and two output scalings
        k = res.sinkhorn_steps
        per = 8 if args.host_loop else 4
        launches += 5 + 3 * per * ((k + per - 1) // per) + 1 + 2
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    total_ms = ev0.elapsed_time(ev1)
    lat = [e0.elapsed_time(e1) for e0, e1 in evs]
    clk = clocks.stop()
    total_ms = max_over_ranks(total_ms, world)
    ms_per_step = total_ms / args.steps
    acc_res = B.result_dict(res)

    out = None
    if rank == 0:
        # ---- roofline of the streaming passes (CUDA events on this stream)
        row_ms, col_ms = ctx.accsink_time_passes(prob, EPS, g, args.pass_reps, stream=stream)
        nm = args.n * args.n
        row_bytes = 4 * nm + 8 * args.n + 24 * args.n          # C, G/Gk, loga/a/u/F
        # column pass over the transposed copy: C^T once, F pair (8 B/row),
        # ell out (8 B/column)
        col_bytes = 4 * nm + 8 * args.n + 8 * args.n
        peak, peak_kind = measured_peaks()
        row_gbs = row_bytes / (row_ms * 1e-3) / 1e9
        col_gbs = col_bytes / (col_ms * 1e-3) / 1e9
        dominant = ("row_pass", row_ms, row_bytes, row_gbs) if row_ms >= col_ms else \
            ("col_pass", col_ms, col_bytes, col_gbs)
        # the committed DRAM counters are for the 16384^2 workload only
        traffic = (profile_traffic("row_warp.cu", f"ncu_{dominant[0]}_gmm16384.txt")
                   if args.n == N else None)

        # ---- Acc vs plain at each eps (one solve each, after the timed region)
        # acc: the default hand-over between homotopy stages (y = w / alpha
        # kept, the state Theorem 1 follows); acc_carry_w: Algorithm 2 as
        # printed, w handed over unchanged.
        versus = {}
        if not args.quick:
            for eps in (1e-1, 1e-2, 1e-3):
                row = {}
                for name, meth, kw in (("acc", B.ACC, {}), ("plain", B.PLAIN, {}),
                                       ("acc_carry_w", B.ACC, {"carry": B.CARRY_W})):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    r = solve(meth, eps, **kw)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    row[name + "_s"] = round(e0.elapsed_time(e1) / 1e3, 6)
                    row[name + "_steps"] = r.sinkhorn_steps
                    row[name + "_status"] = B.STATUS_NAMES[r.status]
                row["speedup"] = round(row["plain_s"] / row["acc_s"], 3)
                row["speedup_carry_w"] = round(row["plain_s"] / row["acc_carry_w_s"], 3)
                versus[f"{eps:g}"] = row

        # ---- end to end through the host-buffer C-ABI call
        Ch = torch.from_numpy(pr["C"]).pin_memory().numpy()
        ah = torch.from_numpy(pr["a"]).pin_memory().numpy()
        bh = torch.from_numpy(pr["b"]).pin_memory().numpy()
        fh = torch.empty(args.n, dtype=torch.float64).pin_memory().numpy()
        gh = torch.empty(args.n, dtype=torch.float64).pin_memory().numpy()
        pe = B.default_params(eps=EPS, tol=TOL)
        ctx.accsink_solve_host(Ch, ah, bh, pe, fh, gh, stream=stream)     # warm-up
        e2e = []
        for _ in range(max(1, min(args.steps, 3))):
            t0 = time.perf_counter()
            ctx.accsink_solve_host(Ch, ah, bh, pe, fh, gh, stream=stream)
            e2e.append(time.perf_counter() - t0)
        h2d = Ch.nbytes + ah.nbytes + bh.nbytes
        d2h = fh.nbytes + gh.nbytes

        value = ms_per_step / 1e3
        out = {
            "metric": METRIC,
            "value": round(value, 6),
            "unit": "s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": False,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 bulk, f64 reductions",
            "data": "synthetic (seeded)",
            "config": bench_config(args.n),
            "loop": "CUDA graph, conditional WHILE node" if acc_res["loop_mode"] else "host loop",
            "latency_s": {"p50": round(percentile(lat, 0.5) / 1e3, 6),
                          "p99": round(percentile(lat, 0.99) / 1e3, 6)},
            "acc_steps": steps[-1],
            "ms_per_sinkhorn_step": round(ms_per_step / steps[-1], 5),
            "final_marginal_l1_gpu": acc_res["marginal_l1"],
            "acc_vs_plain": versus,
            "roofline": {"bound": "hbm", "kernel": dominant[0],
                         "achieved": round(dominant[3], 1), "peak": peak, "unit": "GB/s",
                         "frac": round(dominant[3] / peak, 4), "traffic": traffic,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, burst)",
                         "bytes_per_launch": dominant[2],
                         "ms_per_launch": round(dominant[1], 5),
                         "other_pass": {"row_pass_gbs": round(row_gbs, 1),
                                        "col_pass_gbs": round(col_gbs, 1)}},
            "e2e": {"value": round(statistics.median(e2e), 6), "unit": "s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": launches,
            "clocks": clk,
        }
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(pr, steps[-1], args.cpu_evals)
        if not args.no_points:
            out["points_workload"] = measure_points(ctx, dev, stream, args.points_n,
                                                    not args.quick, args.pass_reps,
                                                    clk.get("sm_max_mhz"), args.host_loop)
        if not args.no_batch:
            out["batch_workload"] = measure_batch(ctx, dev, stream, args.batch_count, 3,
                                                  not args.quick, not args.quick)
            out["batch_workload"]["large_problem"] = measure_batch_large(
                ctx, stream, prob, args.n, steps[-1], ms_per_step)
        if not args.no_serve:
            out["serving_workload"] = measure_serving(
                args.serve_rates, args.serve_window, args.serve_max, 64, 16,
                args.serve_long_rates, args.serve_long_window, args.serve_group_cap)
    ctx.close()
    return out


def run_batch_only(args):
    """Only the batched workload (used for profiling the persistent solver)."""
    import torch

    from paper_2605_30267_gb300 import binding as B
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = B.Context(0)
    stream = torch.cuda.Stream(dev)
    out = measure_batch(ctx, dev, stream, args.batch_count, max(1, args.steps), not args.quick,
                        not args.quick)
    ctx.close()
    return {"metric": METRIC, "batch_workload": out}


def run_batch_large_only(args):
    """Only the stored-cost workload (size --n) as a batch of one (profiling
    the batched solver on a large problem)."""
    import torch

    from paper_2605_30267_gb300 import binding as B
    from paper_2605_30267_gb300 import workloads as W
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    pr = W.gmm_stored_cost_problem(seed=SEED, n=args.n, m=args.n, eps=EPS, tol=TOL)
    C = torch.from_numpy(pr["C"]).to(dev)
    a = torch.from_numpy(pr["a"]).to(dev)
    b = torch.from_numpy(pr["b"]).to(dev)
    ctx = B.Context(0)
    stream = torch.cuda.Stream(dev)
    prob = B.problem_dense(C, a, b)
    f = torch.empty(args.n, dtype=torch.float64, device=dev)
    g = torch.empty(args.n, dtype=torch.float64, device=dev)
    r = ctx.accsink_solve(prob, B.default_params(eps=EPS, tol=TOL), f, g, stream=stream)
    out = measure_batch_large(ctx, stream, prob, args.n, r.sinkhorn_steps, r.gpu_ms)
    ctx.close()
    return {"metric": METRIC, "batch_large_problem": out}


def run_serve_only(args):
    """Only the serving workload."""
    import torch
    torch.cuda.set_device(0)
    return {"metric": METRIC,
            "serving_workload": measure_serving(args.serve_rates, args.serve_window,
                                                args.serve_max, 64, 16, args.serve_long_rates,
                                                args.serve_long_window, args.serve_group_cap)}


def run_points_only(args):
    """Only the point-cloud workload (used for profiling the point passes)."""
    import torch

    from paper_2605_30267_gb300 import binding as B
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = B.Context(0)
    stream = torch.cuda.Stream(dev)
    out = measure_points(ctx, dev, stream, args.points_n, not args.quick, args.pass_reps, None,
                         args.host_loop)
    ctx.close()
    return {"metric": METRIC, "points_workload": out}


POINTS_N = 65536
POINTS_WORKLOAD = ("colour-transfer-shaped point clouds n=m=65536 in [0,1]^3 (source uniform, "
                   "target 16-cluster mixture sigma 0.03), squared Euclidean cost formed on the "
                   "fly and scaled to max 1, uniform marginals, eps=1e-3, tol=1e-6")


def measure_points(ctx, dev, stream, n, with_plain, pass_reps, sm_max_mhz, host_loop=False):
    """Colour-transfer-shaped solve with the cost formed on the fly from the
    point clouds (no n x m matrix): Acc (and plain) time to tol, and the
    arithmetic roofline of the two point passes."""
    import torch

    from paper_2605_30267_gb300 import binding as B
    from paper_2605_30267_gb300 import workloads as W
    pr = W.color_transfer_problem(seed=SEED, n=n, eps=EPS, tol=TOL)
    X = torch.from_numpy(pr["X"]).to(dev)
    Y = torch.from_numpy(pr["Y"]).to(dev)
    a = torch.from_numpy(pr["a"]).to(dev)
    b = torch.from_numpy(pr["b"]).to(dev)
    prob = B.problem_points(X, Y, "sqeuclid", a, b, True)
    f = torch.empty(n, dtype=torch.float64, device=dev)
    g = torch.empty(n, dtype=torch.float64, device=dev)
    out = {"workload": POINTS_WORKLOAD.replace("65536", str(n)), "n": n, "m": n, "d": 3,
           "eps": EPS, "tol": TOL}
    methods = ((("acc", B.ACC, {}), ("plain", B.PLAIN, {}),
                ("acc_carry_w", B.ACC, {"carry": B.CARRY_W}))
               if with_plain else (("acc", B.ACC, {}),))
    for name, meth, kw in methods:
        p = B.default_params(eps=EPS, tol=TOL, method=meth, use_graph=0 if host_loop else 1,
                             **kw)
        if name == "acc":
            ctx.accsink_solve(prob, p, f, g, stream=stream)          # warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = ctx.accsink_solve(prob, p, f, g, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name + "_s"] = round(e0.elapsed_time(e1) / 1e3, 6)
        out[name + "_steps"] = r.sinkhorn_steps
        out[name + "_status"] = B.STATUS_NAMES[r.status]
        out[name + "_marginal_l1"] = r.marginal_l1
        if name == "acc":
            gsol = g.clone()
    if with_plain:
        out["speedup"] = round(out["plain_s"] / out["acc_s"], 3)
        out["speedup_carry_w"] = round(out["plain_s"] / out["acc_carry_w_s"], 3)
    row_ms, col_ms = ctx.accsink_time_passes(prob, EPS, gsol, pass_reps, stream=stream)
    # FP32 work per cost entry of the exact expansion (8 per coordinate:
    # FMUL, 2 FFMA, 5 FADD) plus the exponent (2 FADD), the accumulation
    # (1 FADD), the running max and the Kahan fold (~2); ex2 runs on the XU.
    d = 3
    ops = 8 * d + 5
    peak = MEASURED_FFMA_PER_S / 1e9              # FP32 lane operations, G/s
    ms = max(row_ms, col_ms)
    achieved = ops * n * n / (ms * 1e-3) / 1e9
    entries_per_s = n * n / (ms * 1e-3)
    out["pass_ms"] = {"row": round(row_ms, 4), "col": round(col_ms, 4)}
    # The solve runs on the clouds in Hilbert-curve order and skips the slots whose
    # terms are all below 2^-80 of their rows' sums; the single passes timed
    # above run every slot. Per S evaluation of the timed Acc solve:
    ms_step = out["acc_s"] * 1e3 / max(1, out["acc_steps"])
    out["solve_per_step"] = {"ms": round(ms_step, 4),
                             "unpruned_pass_pair_ms": round(row_ms + col_ms, 4),
                             "cost_entries_per_s": round(2 * n * n / (ms_step * 1e-3), 1),
                             "note": "sorted clouds, pruned slots; the roofline below is the "
                                     "unpruned pass kernel, every slot evaluated"}
    out["roofline"] = {"bound": "alu", "kernel": "row_pass" if row_ms >= col_ms else "col_pass",
                       "achieved": round(achieved, 1), "peak": round(peak, 1),
                       "unit": "G FP32 ops/s", "frac": round(achieved / peak, 4),
                       "ops_per_element": ops, "elements_per_launch": n * n,
                       "ops_counted": "the exact double-float expansion the pass executes",
                       "peak_source": "measured FFMA lane operations/s (throughput probe)",
                       "cost_entries_per_s": round(entries_per_s, 1),
                       # the method's own work per entry: d multiply-adds of
                       # x.y and one exponential (no double-float expansion)
                       "method_work": {
                           "fma_per_element": d, "exp_per_element": 1,
                           "fma_frac": round(d * entries_per_s / MEASURED_FFMA_PER_S, 4),
                           "exp_frac": round(entries_per_s / MEASURED_EX2_PER_S, 4),
                           "exp_peak_per_s": MEASURED_EX2_PER_S,
                           "peak_source": "measured ex2.approx and FFMA rates (probe)"}}
    return out


BATCH_COUNT = 512
BATCH_WORKLOAD = ("word-alignment-shaped batch: 512 problems, n, m log-uniform in [16, 2048], "
                  "unit-norm Gaussian points in R^300, cosine cost 1 - x.y, Dirichlet(1) "
                  "marginals, eps ~ U[0.005, 0.05], tol=1e-6")


def measure_batch(ctx, dev, stream, count, reps, one_at_a_time=True, autotune=True):
    """Many independent problems in one persistent launch (accsink_solve_batch):
    time to solve the whole batch, the cost formation and the solve phase,
    after the project's autotuner picked the work split; beside it the same
    problems solved one at a time through the same engine."""
    import numpy as np
    import torch

    from paper_2605_30267_gb300 import binding as B
    from paper_2605_30267_gb300 import workloads as W
    batch = W.word_alignment_batch(seed=SEED, count=count)
    structs, params, fs, gs = [], [], [], []
    nm = 0
    for pr in batch:
        X = torch.from_numpy(pr["X"]).to(dev)
        Y = torch.from_numpy(pr["Y"]).to(dev)
        a = torch.from_numpy(pr["a"]).to(dev)
        b = torch.from_numpy(pr["b"]).to(dev)
        structs.append(B.problem_points(X, Y, "cosine", a, b, False))
        params.append(B.default_params(eps=pr["eps"], tol=TOL))
        fs.append(torch.empty(X.shape[0], dtype=torch.float64, device=dev))
        gs.append(torch.empty(Y.shape[0], dtype=torch.float64, device=dev))
        nm += X.shape[0] * Y.shape[0]
    out = {"workload": BATCH_WORKLOAD.replace("512 problems", f"{count} problems"),
           "count": count, "d": 300, "sum_nm": nm}
    if autotune:
        best, times = ctx.accsink_batch_autotune(structs, params, fs, gs, stream=stream)
        out["autotune"] = {"best": best, "candidates": len(times),
                           "best_ms": round(min(times), 3), "worst_ms": round(max(times), 3)}
    res = ctx.accsink_solve_batch(structs, params, fs, gs, stream=stream)   # warm-up
    tms = []
    for _ in range(max(1, reps)):
        res = ctx.accsink_solve_batch(structs, params, fs, gs, stream=stream)
        tms.append(ctx.accsink_batch_last_timing())
    steps = [r.sinkhorn_steps for r in res]
    evals = sum(st * 2 * structs[k].n * structs[k].m for k, st in enumerate(steps))
    # cost bytes the solve reads: every S evaluation passes over the stored
    # double-float K (hi + lo, 8 bytes per entry) twice (row pass, column pass
    # over K or K^T), the final evaluation pass once more
    kbytes = sum((16 * st + 8) * structs[k].n * structs[k].m for k, st in enumerate(steps))
    med = sorted(tms, key=lambda t: t["total_ms"])[len(tms) // 2]
    out.update({
        "batch_s": round(med["total_ms"] / 1e3, 6),
        "form_s": round(med["form_ms"] / 1e3, 6),
        "solve_s": round(med["solve_ms"] / 1e3, 6),
        "solves_per_s": round(count / (med["total_ms"] / 1e3), 1),
        "converged": sum(1 for r in res if r.status == 0),
        "steps": {"min": min(steps), "median": int(np.median(steps)), "max": max(steps)},
        "cost_entry_evaluations": evals,
        "solve_entries_per_s": round(evals / (med["solve_ms"] / 1e3), 1),
    })
    peak, peak_kind = measured_peaks()
    kgbs = kbytes / (med["solve_ms"] / 1e3) / 1e9
    out["roofline"] = {
        "bound": "hbm", "kernel": "k_batch_solve", "achieved": round(kgbs, 1), "peak": peak,
        "unit": "GB/s", "frac": round(kgbs / peak, 4), "traffic": None,
        "bytes_per_launch": kbytes,
        "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, burst)",
        "note": "cost bytes read by the solve phase (K hi + lo, 16 B per entry per S "
                "evaluation, 8 B for the final pass) over its time; problems with n m <= 65536 "
                "are solved whole by one CTA and read their 512 KB or less of K mostly from "
                "L2, so this is a read bandwidth against the HBM peak, not DRAM traffic"}
    # the method's own contraction x.y (d multiply-adds per entry), against
    # the slice-pair products the exact formation issues
    method_macs = sum(s_.n * s_.m * 300 for s_ in structs)
    # the cosine costs are formed on the tensor cores: 21 FP16 slice-pair
    # products per 128 x 64 tile and 16-element contraction step
    dpad = (300 + 31) // 32 * 32
    tiles = sum(-(-s.n // 128) * -(-s.m // 64) for s in structs)
    macs = tiles * 128 * 64 * dpad * 21
    form_tf = 2 * macs / (med["form_ms"] / 1e3) / 1e12
    method_tf = 2 * method_macs / (med["form_ms"] / 1e3) / 1e12
    out["form_tensor_cores"] = {
        "kernel": "k_batch_form_tc (tcgen05 kind::f16, FP32 accumulators in TMEM)",
        "tiles": tiles, "slice_pair_macs": macs,
        "achieved_tflops": round(form_tf, 1), "peak_tflops": measured_bf16_tflops(),
        "frac": round(form_tf / measured_bf16_tflops(), 4),
        "method_macs": method_macs,
        "method_tflops": round(method_tf, 2),
        "method_frac": round(method_tf / measured_bf16_tflops(), 4),
        "note": "over the whole formation phase (slicing, tiles, statistics); peak: measured "
                "dense bf16 cuBLAS burst (FP16 runs at the same tensor rate). method_*: the "
                "cosine costs' own d = 300 multiply-adds per entry; the exact integer-slice "
                "formation issues 21 slice-pair products for each (the cost of K exact to "
                "2^-39, which FP32 or 3xTF32 products cannot give)"}
    if one_at_a_time:
        tot = 0.0
        for k in range(count):
            ctx.accsink_solve_batch([structs[k]], [params[k]], [fs[k]], [gs[k]], stream=stream)
            tot += ctx.accsink_batch_last_timing()["total_ms"]
        out["one_at_a_time_s"] = round(tot / 1e3, 6)
        out["batched_speedup"] = round(tot / med["total_ms"], 2)
    return out


def measure_batch_large(ctx, stream, prob, n, steps_single, ms_single):
    """The benchmark's own 16384 x 16384 stored-cost problem through the batch
    API (a batch of one). By default a lone dense problem is handed to the
    single-solve path (loop_mode 1); with dense_solo_min_nm = -1 it runs in
    the batched launch, whose time per S evaluation and cost-read bandwidth
    are reported beside it (the batched launch stores K = k C as a
    double-float pair: 16 bytes per entry per S evaluation, against the
    single solve's 8)."""
    import torch

    from paper_2605_30267_gb300 import binding as B
    dev = torch.device("cuda", torch.cuda.current_device())
    f = torch.empty(n, dtype=torch.float64, device=dev)
    g = torch.empty(n, dtype=torch.float64, device=dev)
    p = B.default_params(eps=EPS, tol=TOL)
    ctx.accsink_solve_batch([prob], [p], [f], [g], stream=stream)        # warm-up
    res = ctx.accsink_solve_batch([prob], [p], [f], [g], stream=stream)
    t = ctx.accsink_batch_last_timing()
    routed = {"loop_mode": res[0].loop_mode, "steps": res[0].sinkhorn_steps,
              "total_ms": round(t["total_ms"], 3),
              "ms_per_s_evaluation": round(t["total_ms"] / max(1, res[0].sinkhorn_steps), 4)}
    cfg = ctx.accsink_batch_get_config()
    ctx.accsink_batch_set_config(cfg["small_max_nm"], cfg["row_tile_elems"], cfg["ctas_per_sm"],
                                 dense_solo_min_nm=-1)
    try:
        ctx.accsink_solve_batch([prob], [p], [f], [g], stream=stream)    # warm-up
        res = ctx.accsink_solve_batch([prob], [p], [f], [g], stream=stream)
        t = ctx.accsink_batch_last_timing()
    finally:
        ctx.accsink_batch_set_config(cfg["small_max_nm"], cfg["row_tile_elems"],
                                     cfg["ctas_per_sm"], cfg["dense_solo_min_nm"])
    st = res[0].sinkhorn_steps
    per = t["solve_ms"] / max(1, st)
    peak, _ = measured_peaks()
    gbs = 16 * n * n / (per * 1e-3) / 1e9
    return {"problem": f"the stored-cost workload (dense {n} x {n}, eps=1e-3) as a batch of one",
            "batch_api": routed,
            "single_solve_ms_per_s_evaluation": round(ms_single / max(1, steps_single), 4),
            "batched_launch": {"loop_mode": res[0].loop_mode, "steps": st,
                               "form_ms": round(t["form_ms"], 3),
                               "solve_ms": round(t["solve_ms"], 3),
                               "ms_per_s_evaluation": round(per, 4),
                               "cost_read_gbs": round(gbs, 1),
                               "frac_of_hbm_peak": round(gbs / peak, 4),
                               "note": "dense_solo_min_nm = -1 keeps the problem in the "
                                       "batched launch"}}


SERVE_WORKLOAD = ("serving: Poisson arrivals; requests are squared-Euclidean problems, points "
                  "uniform in [0,1]^d, d in {2..64}, n, m log-uniform in [64, 16384], Dirichlet(1) "
                  "marginals, eps log-uniform in [1e-3, 1e-1], tol=1e-6, cost scaled to max 1; "
                  "64 GB admission budget")


def serve_window(probs, params, rate, window_s, group_cap, seed):
    """The request server under Poisson arrivals at `rate` for `window_s`
    seconds (a fresh server, 64 GB budget). Requests are submitted as they
    arrive; what the server completes inside the window counts. Reports the
    offered and completed counts, the sustained rate (completed / window),
    the submit-to-done latency of the completed requests, and the backlog at
    the window's end (queued or running, with the age of the oldest); the
    server is then closed, which drops the queued requests."""
    import threading

    from paper_2605_30267_gb300 import binding as B
    from paper_2605_30267_gb300 import workloads as W
    pool_size = len(probs)
    arrivals = W.poisson_arrivals(seed, rate, int(rate * window_s * 1.3) + 16)
    arrivals = arrivals[arrivals < window_s]
    count = len(arrivals)
    srv = B.Server(0, 64 << 30)
    if group_cap is not None:
        srv.set_limits(group_cap)
    tickets = [None] * count
    submitted = [0]
    lats = []
    done_t = []
    stop = threading.Event()
    try:
        start = time.perf_counter()
        end = start + window_s

        def collect():
            i = 0
            while i < count:
                while tickets[i] is None and not stop.is_set():
                    time.sleep(0.0002)
                if tickets[i] is None:
                    return
                left_ms = int((end - time.perf_counter()) * 1e3)
                if left_ms <= 0:
                    return
                rc, res, lat = srv.wait(tickets[i], left_ms)
                if rc == B.ERR_TIMEOUT:
                    return
                lats.append(lat)
                done_t.append(time.perf_counter() - start)
                srv.release(tickets[i])
                i += 1

        th = threading.Thread(target=collect)
        th.start()
        for i in range(count):
            delay = start + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            if time.perf_counter() >= end:
                break
            k = i % pool_size
            tickets[i] = srv.submit(probs[k], params[k])
            submitted[0] = i + 1
        stop.set()
        th.join()
        now = time.perf_counter() - start
        done = len(lats)
        st = srv.stats()
        oldest = (now - arrivals[done]) if done < submitted[0] else 0.0
        out = {"offered_per_s": rate, "window_s": window_s, "offered": submitted[0],
               "completed": done, "sustained_per_s": round(done / window_s, 2),
               "latency_ms": {"p50": round(percentile(lats, 0.5), 3) if lats else None,
                              "p99": round(percentile(lats, 0.99), 3) if lats else None},
               "backlog_at_end": {"queued": st["queued"],
                                  "queued_or_running": submitted[0] - done,
                                  "oldest_age_s": round(oldest, 3)},
               "server": {"batches": st["batches"], "peak_gb": round(st["peak_bytes"] / 1e9, 3),
                          "busy_s": round(st["busy_ms"] / 1e3, 3),
                          "device_busy_frac": round(st["busy_ms"] / 1e3 / window_s, 3)}}
        if group_cap is not None:
            out["group_entry_limit"] = group_cap
        return out
    finally:
        srv.close()


def measure_serving(rates, window_s, max_requests, pool_size, solo_count, long_rates=(),
                    long_window_s=60.0, group_cap=None):
    """The request server at offered Poisson rates: sustained solves/s and the
    submit-to-done latency (p50/p99, queueing included), beside the same
    requests served one at a time (each submitted after the previous one
    completed); then `long_window_s` windows at `long_rates` (serve_window)."""
    import threading

    import numpy as np

    from paper_2605_30267_gb300 import binding as B
    from paper_2605_30267_gb300 import workloads as W
    pool = W.serving_requests(seed=SEED, count=pool_size)
    probs = [B.problem_host(r["a"], r["b"], X=r["X"], Y=r["Y"], kind="sqeuclid",
                            scale_to_max=True) for r in pool]
    params = [B.default_params(eps=r["eps"], tol=r["tol"]) for r in pool]
    srv = B.Server(0, 64 << 30)
    if group_cap is not None:
        srv.set_limits(group_cap)
    out = {"workload": SERVE_WORKLOAD, "pool": pool_size,
           "mean_nm": float(np.mean([r["X"].shape[0] * r["Y"].shape[0] for r in pool]))}
    try:
        # warm-up: every pool request once, all at once
        ts = [srv.submit(probs[k], params[k]) for k in range(pool_size)]
        steps = []
        for t in ts:
            rc, res, _ = srv.wait(t, 600000)
            steps.append(res.sinkhorn_steps)
            srv.release(t)
        out["steps"] = {"median": int(np.median(steps)), "max": int(max(steps))}
        # one at a time
        t0 = time.perf_counter()
        solo = []
        for k in range(solo_count):
            t = srv.submit(probs[k % pool_size], params[k % pool_size])
            rc, res, lat = srv.wait(t, 600000)
            solo.append(lat)
            srv.release(t)
        solo_s = time.perf_counter() - t0
        out["one_at_a_time"] = {"requests": solo_count,
                                "solves_per_s": round(solo_count / solo_s, 2),
                                "latency_ms": {"p50": round(percentile(solo, 0.5), 3),
                                               "p99": round(percentile(solo, 0.99), 3)}}
        # offered rates
        sweep = []
        for rate in rates:
            count = int(min(max_requests, max(8, rate * window_s)))
            arrivals = W.poisson_arrivals(SEED + int(rate), rate, count)
            tickets = [None] * count
            lats = [None] * count
            done_at = [0.0] * count
            ready = threading.Event()

            def collect():
                ready.wait()
                for i in range(count):
                    while tickets[i] is None:
                        time.sleep(0.0002)
                    rc, res, lat = srv.wait(tickets[i], 600000)
                    lats[i] = lat
                    done_at[i] = time.perf_counter()
                    srv.release(tickets[i])

            th = threading.Thread(target=collect)
            th.start()
            start = time.perf_counter()
            ready.set()
            for i in range(count):
                delay = start + arrivals[i] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                k = i % pool_size
                tickets[i] = srv.submit(probs[k], params[k])
            th.join()
            elapsed = max(done_at) - start
            sweep.append({"offered_per_s": rate, "requests": count,
                          "sustained_per_s": round(count / elapsed, 2),
                          "latency_ms": {"p50": round(percentile(lats, 0.5), 3),
                                         "p99": round(percentile(lats, 0.99), 3)}})
        out["sweep"] = sweep
        st = srv.stats()
        out["server"] = {"batches": st["batches"], "solved": st["solved"], "failed": st["failed"],
                         "peak_gb": round(st["peak_bytes"] / 1e9, 3),
                         "busy_s": round(st["busy_ms"] / 1e3, 3)}
    finally:
        srv.close()
    # long windows (the serving configuration: Poisson arrivals for 60 s)
    out["windows"] = [serve_window(probs, params, r, long_window_s, group_cap, SEED + 7 * int(r))
                      for r in long_rates]
    return out


def cpu_baseline(pr, acc_steps, evals):
    """The FP64 oracle on the host cores: `evals` S evaluations at full size,
    extrapolated to the Acc step count of the GPU solve."""
    import numpy as np

    import oracle as O
    cores = O.set_threads(0)
    cost = O.Cost(C=pr["C"])
    a = O.normalise(pr["a"])
    b = O.normalise(pr["b"])
    x = np.zeros(pr["C"].shape[1])
    t0 = time.perf_counter()
    for _ in range(evals):
        err, u, c, s = O.sinkhorn_map(cost, EPS, a, b, x)
        x = s
    per = (time.perf_counter() - t0) / evals
    return {"value": round(per * acc_steps, 3), "unit": "s", "cores": cores, "kind": "oracle",
            "sample": f"{evals} full-size S evaluations (row + column pass, FP64, OpenMP) "
                      f"at {per:.3f} s each, extrapolated to the {acc_steps} S evaluations "
                      f"of the Acc solve"}


def _oracle_solve_time(O, cost, a, b, eps, method):
    t0 = time.perf_counter()
    r = O.solve(cost, a, b, eps, TOL, method=method)
    return time.perf_counter() - t0, r


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle (plain C, OpenMP over rows and
    columns) on this machine's host cores, on the GPU arm's workload.

    value: one full Acc solve to tol at the benchmark size, measured (not
    extrapolated). steps: `--steps` S evaluations (row pass + column pass)
    at the benchmark size after `--warmup` untimed ones; ms_per_step is their
    median. Beside it: the same S evaluation on one thread, full solves to
    tol of the 256 x 256 point-cloud problem on one thread and on all cores,
    and of the benchmark cost at eps = 1e-1 (plain and Acc)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import numpy as np

    import oracle as O
    from paper_2605_30267_gb300 import workloads as W
    pr = W.gmm_stored_cost_problem(seed=SEED, n=args.n, m=args.n, eps=EPS, tol=TOL)
    cores = O.set_threads(0)
    cost = O.Cost(C=pr["C"])
    a, b = O.normalise(pr["a"]), O.normalise(pr["b"])

    # per S evaluation, all cores
    x = np.zeros(args.n)
    for _ in range(args.warmup):
        O.sinkhorn_map(cost, EPS, a, b, x)
    per = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        err, u, c, s = O.sinkhorn_map(cost, EPS, a, b, x)
        per.append(time.perf_counter() - t0)
        x = s
    per_s = statistics.median(per)

    # the full Acc solve to tol (the metric)
    solve_s, r = _oracle_solve_time(O, cost, a, b, EPS, O.ACC)
    acc_steps = r["sinkhorn_steps"]

    extra = {"acc_steps": acc_steps, "acc_status": "converged" if r["status"] == O.CONVERGED
             else "not converged", "acc_marginal_l1": r["marginal_l1"],
             "per_s_evaluation_s": round(per_s, 4),
             "extrapolated_s": round(per_s * acc_steps, 3)}
    # one thread: one S evaluation at full size
    O.set_threads(1)
    t0 = time.perf_counter()
    O.sinkhorn_map(cost, EPS, a, b, np.zeros(args.n))
    extra["single_thread_per_s_evaluation_s"] = round(time.perf_counter() - t0, 3)
    # the 256 x 256 point-cloud problem to tol, one thread and all cores
    sp = W.small_pointcloud_problem(SEED)
    scost = O.Cost(C=sp["C"])
    small = {}
    for label, th in (("1_thread", 1), (f"{cores}_threads", cores)):
        O.set_threads(th)
        for name, meth in (("acc", O.ACC), ("plain", O.PLAIN)):
            t, rr = _oracle_solve_time(O, scost, sp["a"], sp["b"], sp["eps"], meth)
            small[f"{name}_{label}_s"] = round(t, 4)
            small[f"{name}_steps"] = rr["sinkhorn_steps"]
    extra["small_pointcloud_256"] = dict(small, eps=sp["eps"], tol=TOL)
    # the benchmark cost at eps = 1e-1, all cores
    O.set_threads(cores)
    big01 = {}
    for name, meth in (("acc", O.ACC), ("plain", O.PLAIN)):
        t, rr = _oracle_solve_time(O, cost, a, b, 1e-1, meth)
        big01[f"{name}_s"] = round(t, 3)
        big01[f"{name}_steps"] = rr["sinkhorn_steps"]
    extra["eps_0.1"] = big01

    sample = (f"one full FP64 oracle Acc solve to tol on {cores} threads ({acc_steps} S "
              f"evaluations, measured); steps: single S evaluations at full size, median "
              f"{per_s:.3f} s")
    return {"impl": "reference", "metric": METRIC, "value": round(solve_s, 3), "unit": "s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(per_s * 1e3, 3), "step": "one S evaluation (row + column pass)",
            "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": bench_config(args.n),
            "cpu_baseline": {"value": round(solve_s, 3), "unit": "s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(solve_s, 3), "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "oracle": extra}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--pass-reps", type=int, default=20)
    ap.add_argument("--cpu-evals", type=int, default=30)
    ap.add_argument("--quick", action="store_true", help="skip the Acc-vs-plain table")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive iterations from the host instead of the graph loop")
    ap.add_argument("--points-n", type=int, default=POINTS_N,
                    help="size of the colour-transfer point-cloud workload")
    ap.add_argument("--no-points", action="store_true",
                    help="skip the point-cloud workload")
    ap.add_argument("--points-only", action="store_true",
                    help="run only the point-cloud workload (profiling)")
    ap.add_argument("--batch-count", type=int, default=BATCH_COUNT,
                    help="problems in the word-alignment-shaped batch")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched workload (profiling)")
    ap.add_argument("--batch-large-only", action="store_true",
                    help="run only the stored-cost workload of size --n as a batch of one")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving workload")
    ap.add_argument("--serve-only", action="store_true", help="run only the serving workload")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[25, 50, 100, 200, 2000],
                    help="offered Poisson rates (requests/s)")
    ap.add_argument("--serve-window", type=float, default=3.0,
                    help="seconds of arrivals per offered rate")
    ap.add_argument("--serve-max", type=int, default=400,
                    help="cap on requests per offered rate")
    ap.add_argument("--serve-long-rates", type=float, nargs="*", default=[200, 2000],
                    help="offered rates of the long serving windows")
    ap.add_argument("--serve-long-window", type=float, default=60.0,
                    help="seconds of Poisson arrivals per long window")
    ap.add_argument("--serve-group-cap", type=int, default=None,
                    help="server admission limit in cost entries per group (default: the "
                         "library's)")
    args = ap.parse_args()
    if args.impl == "reference":
        out = run_reference(args)
    elif args.points_only:
        out = run_points_only(args)
    elif args.batch_only:
        out = run_batch_only(args)
    elif args.batch_large_only:
        out = run_batch_large_only(args)
    elif args.serve_only:
        out = run_serve_only(args)
    else:
        out = run_gpu(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
