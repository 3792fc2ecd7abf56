#!/usr/bin/env python
"""Benchmark: time to 1e-4 relative KKT error of restarted PDHG on one GB300.

Workload: the synthetic 1,000,000 x 2,000,000 LP with power-law row lengths
(alpha = 2.1 on 4..5000 nonzeros, nnz ~ 20.07M, N(0,1) values, half >= rows,
half = rows, planted optimum), solved to 1e-4 relative KKT error.  One step is
one full lp_solve: Ruiz scaling, power iteration, and the restarted adaptive
PDHG loop with its KKT checks, in the mixed path (FP32 matrix, iterates and SpMV
accumulation; FP64 reductions).  The plain FP64 path is solved once beside it.

Prints one JSON line (rank 0).  With torchrun and N GPUs each rank solves its
own instance (seed + rank): replicas, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "time to 1e-4 rel KKT (s), PDHG iters/s, SpMV HBM GB/s vs FP64 plain"
FALLBACK_HBM_GBS = 6800.0
CACHE = os.environ.get("PDHG_BENCH_CACHE", "/tmp/pdhg_bench_cache")

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# step kernels from one ncu capture of the current kernel source (absent when
# the kernel changed after the capture).  Summary: profiles/spmv_powerlaw_1Mx2M_fp32.md
NCU_TRAFFIC = {"spmv_K_dual": 198_677_504, "spmv_KT_primal": 230_124_032}

# kernel classes of lp_profile_step: a PDHG attempt is the K-side SpMV with the
# dual step and the Algorithm 5 decision, then the K^T-side SpMV with the fused
# primal step (no separate primal launch); a Halpern iteration has three
STEP_NAMES = ["primal_update", "spmv_K_dual", "spmv_KT_primal", "step_control"]


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="powerlaw",
                   choices=["powerlaw", "small", "dispatch", "batch", "adjoint"],
                   help="powerlaw: the 1M x 2M LP (default bench line); small: 200 x 400; "
                        "dispatch: the 615,001 x 5,000 dispatch-shaped LP; batch: 512 LPs "
                        "solved by one lp_batch_solve; adjoint: lp_grad of 500 unrolled "
                        "iterations on the 100k x 200k LP (extra lines)")
    p.add_argument("--tol", type=float, default=1e-4)
    p.add_argument("--method", default="pdhg", choices=["pdhg", "halpern"],
                   help="pdhg: the paper's restarted adaptive PDHG (the bench line); halpern: "
                        "restarted reflected Halpern PDHG in the timed loop")
    p.add_argument("--no-halpern", action="store_true",
                   help="skip the restarted Halpern PDHG measurement (extra key)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-samples", type=int, default=7,
                   help="oracle samples of 32 iterations for the CPU baseline")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extra", action="store_true",
                   help="skip the other workloads of the default line (the dispatch-shaped "
                        "LP, the 512-LP batch with its FP64 comparisons, lp_grad)")
    p.add_argument("--no-fishnet", action="store_true",
                   help="skip the Algorithm 7 warm-start measurement (extra key)")
    p.add_argument("--fp64-profile", action="store_true",
                   help="with --kernel-profile: also time the FP64 step kernels")
    p.add_argument("--fishnet-profile", action="store_true",
                   help="one lp_fishnet call on the workload (32 points, 2 steps per round), "
                        "for kernel profilers; prints its time")
    p.add_argument("--host-loop", action="store_true",
                   help="host-driven loop graph (lp_opts.loop_mode = 1), for ncu launch lists")
    p.add_argument("--gather-ceiling", action="store_true",
                   help="time the minimal gather loop (lp_profile_gather) over K and K^T of "
                        "the workload beside the step kernels (no bench line)")
    p.add_argument("--kernel-profile", action="store_true",
                   help="short run for ncu: one 64-iteration mixed solve, then 3 timed step "
                        "attempts of each kernel class (no bench line)")
    return p.parse_args()


def kernel_profile(args):
    import torch
    from paper_2508_16806_gb300 import lp as L
    L.load()
    lp, desc = workload(args.workload)
    stream = torch.cuda.Stream()
    prob = L.Problem(lp, device_copy=True, stream=stream)
    halp = int(args.method == "halpern")
    prob.solve(tol=args.tol, precision=L.LP_PREC_MIXED, max_iters=64, halpern=halp)
    ms, by = prob.profile_step(L.LP_PREC_MIXED, reps=3)
    line = {"kernel_profile": desc, "method": args.method, "ms": ms, "bytes": by}
    if args.fp64_profile:
        prob.solve(tol=args.tol, precision=L.LP_PREC_FP64, max_iters=64, halpern=halp)
        line["ms_fp64"], line["bytes_fp64"] = prob.profile_step(L.LP_PREC_FP64, reps=3)
    print(json.dumps(line), flush=True)
    prob.close()


def gather_ceiling(prob, prec, lp, reps=20):
    """lp_profile_gather: the minimal gather loop over the nonzeros of K and of
    K^T (milliseconds per launch, CUDA events on the solver's stream) and the
    rate of gathers it reaches, for 4 and 8 resident blocks per SM."""
    out = {"by_blocks_per_sm": {}}
    for bps in (2, 4, 6, 8):
        ms = prob.profile_gather(prec, reps=reps, blocks_per_sm=bps)
        out["by_blocks_per_sm"][bps] = ms
        for side, t in zip(("K", "KT"), ms):
            cur = out.get(side)
            if cur is None or t < cur["ms"]:
                out[side] = {"ms": t, "gathers_per_s": lp.nnz / (t * 1e-3),
                             "blocks_per_sm": bps}
    return out


def kernel_profile_gather(args):
    """--gather-ceiling: one mixed solve of 64 iterations (the vectors), then the
    gather ceiling and the step kernels of both precisions (no bench line)."""
    import torch
    from paper_2508_16806_gb300 import lp as L
    L.load()
    lp, desc = workload(args.workload)
    stream = torch.cuda.Stream()
    prob = L.Problem(lp, device_copy=True, stream=stream)
    line = {"gather_ceiling": desc}
    for prec, tag in ((L.LP_PREC_MIXED, "fp32"), (L.LP_PREC_FP64, "fp64")):
        prob.solve(tol=args.tol, precision=prec, max_iters=64)
        line[tag] = gather_ceiling(prob, prec, lp)
        ms, by = prob.profile_step(prec, reps=20)
        line[tag]["step_ms"] = dict(zip(STEP_NAMES, ms))
    print(json.dumps(line), flush=True)
    prob.close()


def halpern_leg(L, prob, stream, opts):
    """Restarted reflected Halpern PDHG (fixed eta = 0.9 / ||K~||) on the same LP,
    tolerance and precision: one warm-up solve (its loop graph), one timed with
    CUDA events on the solver's stream (outside the bench line's timed region)."""
    import torch
    o = dict(opts, halpern=1, time_limit_s=300.0)
    prob.solve(**dict(o, max_iters=64))
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    _, _, info, _ = prob.solve(**o)
    ev1.record(stream)
    torch.cuda.synchronize()
    out = {"time_to_tol_s": ev0.elapsed_time(ev1) / 1e3, "iters": int(info["iters"]),
           "fp64_iters": int(info["fp64_iters"]), "restarts": int(info["restarts"]),
           "status": L.STATUS[info["status"]], "reflect": 1.0, "reflect_fp32": 0.5,
           "setup_s": info["setup_s"]}
    # its step kernels (FP32), CUDA events on the solver's stream
    prob.solve(**dict(o, max_iters=256))
    ms_k, by_k = prob.profile_step(L.LP_PREC_MIXED, reps=30)
    names = ["primal_halpern", "spmv_K_halpern_dual", "spmv_KT_halpern"]
    out["kernels"] = {nm: {"ms": a, "bytes": b, "gbs": b / (a * 1e-3) / 1e9 if a > 0 else None}
                      for nm, a, b in zip(names, ms_k, by_k)}
    return out


def max_over_ranks(value, world):
    """The slowest rank's time (the whole job finishes with it)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_batch(args):
    """512 planted LPs (m log-uniform 500..50,000, n = 2m, 5-20 nonzeros per row)
    solved together to 1e-4 (mixed path) by one lp_batch_solve per step; LPs/s,
    per-LP device time to tolerance (p50 / p99), and a loop of single lp_solve
    calls on the first 64 LPs scaled to 512 for comparison."""
    import torch
    import torch.distributed as dist
    from paper_2508_16806_gb300 import lp as L
    from paper_2508_16806_gb300 import synth
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    L.load()
    # independent LPs: one list of 512 x world LPs shared among the ranks by
    # nonzeros (weak scaling: about 512 LPs per rank); each rank builds only its
    # own LPs
    from paper_2508_16806_gb300 import dist as D
    share = D.partition_by_nnz(synth.batch_nnz(512 * world), world)[rank]
    lps = synth.batch_lps(indices=share)
    batch = L.Batch(lps)
    opts = dict(tol=args.tol, precision=L.LP_PREC_MIXED, max_iters=2_000_000, autotune=1)
    for _ in range(args.warmup):
        batch.solve(**opts)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(batch.stream)
    outs = []
    for _ in range(args.steps):
        outs.append(batch.solve(**opts))
    ev1.record(batch.stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
    last = outs[-1]
    per_lp = sorted(info["solve_s"] for _, _, info in last)
    launches = int(sum(info["kernel_launches"] for o in outs for _, _, info in o))
    statuses = sorted({L.STATUS[info["status"]] for _, _, info in last})
    # loop of single solves on a sample (rank 0 reports it)
    sample = 64 if rank == 0 else 0
    t0 = time.perf_counter()
    for lp in lps[:sample]:
        p = L.Problem(lp)
        p.solve(**opts)
        p.close()
    torch.cuda.synchronize()
    loop_s = (time.perf_counter() - t0) * len(lps) / max(sample, 1)
    batch.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {"metric": "LPs/s (512-LP batch, time to 1e-4 rel KKT)",
            "value": 512 * world / (ms / 1e3), "unit": "LP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "512 planted LPs per GPU, m log-uniform 500..50,000, n = 2m, "
                                   "5-20 nnz/row (one list of 512 x N shared by nonzeros)",
                       "nnz": int(sum(lp.nnz for lp in lps)), "lps_rank0": len(lps), "tol": args.tol,
                       "step": "one lp_batch_solve of all 512 LPs"},
            "statuses": statuses,
            "per_lp_time_to_tol_s": {"p50": per_lp[len(per_lp) // 2],
                                     "p99": per_lp[min(len(per_lp) - 1, int(0.99 * len(per_lp)))],
                                     "max": per_lp[-1]},
            "iters": {"p50": sorted(i["iters"] for _, _, i in last)[len(last) // 2],
                      "max": max(i["iters"] for _, _, i in last)},
            "single_solve_loop_s": loop_s,
            "single_solve_loop_sample": f"first {sample} LPs, scaled to {len(lps)}",
            "clocks": clk, "gpu_launches": launches}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def workload(name, seed_offset=0):
    from paper_2508_16806_gb300 import synth
    if name == "small":
        lp = synth.small_dense_lp(20250816 + seed_offset)
        return lp, "lp200x400 (100 >= / 100 = rows, 2% N(0,1) sparsity, planted optimum)"
    if name == "dispatch":
        lp = synth.dispatch_lp(seed=20250818 + seed_offset)
        return lp, ("dispatch-shaped LP 615,001 x 5,000 (1 balance row, 15,000 flow rows x 41 "
                    "contingency blocks, 10-200 coefficients per row, costs U[10,100])")
    os.makedirs(CACHE, exist_ok=True)
    path = os.path.join(CACHE, f"powerlaw_{20250817 + seed_offset}.npz")
    desc = ("powerlaw LP 1,000,000 x 2,000,000 (row lengths alpha 2.1 on 4..5000, "
            "N(0,1) values, half >= / half = rows, planted optimum)")
    if os.path.exists(path):
        z = np.load(path)
        lp = synth.LP(int(z["m"]), int(z["n"]), z["row_ptr"], z["col_idx"], z["vals"], z["sense"],
                      z["c"], z["q"], z["l"], z["u"], z["x_star"], None, "powerlaw")
        return lp, desc
    lp = synth.power_law_lp(seed=20250817 + seed_offset)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, m=lp.m, n=lp.n, row_ptr=lp.row_ptr, col_idx=lp.col_idx, vals=lp.vals,
             sense=lp.sense, c=lp.c, q=lp.q, l=lp.l, u=lp.u, x_star=lp.x_star)
    os.replace(tmp, path)
    return lp, desc


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, burst copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.lines = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [t.strip() for t in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


ORACLE_SAMPLE_ITERS = 32


class OracleTimer:
    """Times the FP64 CPU oracle (one host core) on the workload, piece by piece.

    setup(): Ruiz (10 passes of Algorithm 3), one power iteration (Algorithm 2)
    and a run that stops at its start check (one power iteration + one KKT
    check), each timed once.
    sample(): one oracle run of ORACLE_SAMPLE_ITERS accepted iterations of the
    restarted adaptive loop (no Ruiz, one power iteration, a check at the start
    and at the end); the per-iteration time follows from it and the setup runs:
    t_iter = (T_sample - 2 T_start + t_pow) / ORACLE_SAMPLE_ITERS, where
    T_start = t_pow + t_check.
    estimate(N): Ruiz + 100 power iterations + N iterations + one check per 64
    iterations: the oracle's time to tolerance for a run of N iterations,
    estimated from the measured pieces (the run itself takes hours)."""

    def __init__(self, lp):
        import oracle
        oracle.build()
        self.oracle = oracle
        self.lp = lp
        self.t_iter = []

    def setup(self):
        o, lp = self.oracle, self.lp
        t = time.perf_counter()
        o.ruiz(lp, 10, 1e-4)
        self.t_ruiz = time.perf_counter() - t
        t = time.perf_counter()
        o.power_norm(lp, 1)
        self.t_pow = time.perf_counter() - t
        t = time.perf_counter()
        o.solve(lp, tol=0.0, max_iters=0, check_every=64, ruiz_iters=0, power_iters=1)
        self.t_start = time.perf_counter() - t
        self.t_check = max(self.t_start - self.t_pow, 0.0)

    def sample(self):
        k = ORACLE_SAMPLE_ITERS
        t = time.perf_counter()
        self.oracle.solve(self.lp, tol=0.0, max_iters=k, check_every=k, ruiz_iters=0,
                          power_iters=1)
        ts = time.perf_counter() - t
        self.t_iter.append(max(ts - 2 * self.t_start + self.t_pow, 1e-9) / k)
        return ts

    def iter_s(self):
        return statistics.mean(self.t_iter)

    def estimate(self, iters):
        return (self.t_ruiz + 100 * self.t_pow + iters * self.iter_s() +
                (iters / 64 + 1) * self.t_check)

    def describe(self, iters, src):
        return (f"measured on {len(self.t_iter)} oracle runs of {ORACLE_SAMPLE_ITERS} accepted "
                f"iterations of the restarted adaptive loop ({len(self.t_iter) * ORACLE_SAMPLE_ITERS} "
                f"iterations: {1.0 / self.iter_s():.4g} iterations/s, {self.iter_s():.4g} s each), "
                f"one KKT check {self.t_check:.4g} s, Ruiz {self.t_ruiz:.4g} s, one power iteration "
                f"{self.t_pow:.4g} s; the time to tolerance is estimated from these measured "
                f"pieces x the {iters} iterations of the {src} (+ one check per 64 iterations, "
                f"Ruiz, 100 power iterations)")


def cpu_info():
    out = {"nproc": os.cpu_count()}
    try:
        keys = {}
        for ln in open("/proc/cpuinfo"):
            k, _, v = ln.partition(":")
            k = k.strip().lower()
            if k in ("model name", "cpu implementer", "cpu part") and k not in keys:
                keys[k] = v.strip()
        out["cpu"] = keys.get("model name") or (
            f"implementer {keys.get('cpu implementer')} part {keys.get('cpu part')}")
        out["machine"] = os.uname().machine
    except Exception:
        pass
    return out


def reference_iterations(tol, lp):
    """Iterations the FP64 oracle takes to tol on this LP: a stored run of the
    oracle to tolerance (oracle/reference_runs.json, matched by nnz), or, for a
    small LP, a run made here."""
    path = os.path.join(ROOT, "oracle", "reference_runs.json")
    try:
        for r in json.load(open(path)):
            if abs(r["tol"] - tol) < 1e-15 and r["status"] == 1 and r.get("nnz") == lp.nnz:
                return int(r["iters"]), "oracle run to tolerance (oracle/reference_runs.json)"
    except Exception:
        pass
    if lp.nnz < 1_000_000:
        import oracle
        oracle.build()
        _, _, info, _ = oracle.solve(lp, tol=tol, max_iters=2_000_000)
        if info["status"] == 1:
            return int(info["iters"]), "oracle run to tolerance in this process"
    return None, None


def run_reference(args):
    """The oracle arm: each step is one measured oracle sample of the workload
    (OracleTimer.sample, about 7 s on the 1M x 2M LP); ms_per_step is that
    measured time; value is the oracle's estimated time to tolerance from the
    measured pieces (the same metric and unit as the GPU arm)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    lp, desc = workload(args.workload)
    iters, src = reference_iterations(args.tol, lp)
    if iters is None:
        iters, src = 5000, "assumed 5000 iterations (no stored oracle run)"
    ot = OracleTimer(lp)
    ot.setup()
    steps = []
    for s in range(args.warmup + args.steps):
        ts = ot.sample()
        if s >= args.warmup:
            steps.append(ts)
        else:
            ot.t_iter.pop()
    v = float(ot.estimate(iters))
    sample = ot.describe(iters, src)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(steps) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "tol": args.tol, "iterations_to_tol": iters,
                       "iterations_source": src,
                       "step": f"one oracle run of {ORACLE_SAMPLE_ITERS} accepted iterations "
                               "(measured); value = estimated time to tolerance"},
            "oracle_iters_per_s": 1.0 / ot.iter_s(),
            "value_is_estimate": True,
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": sample, **cpu_info()},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """lp_grad (hand-written adjoint) of 500 unrolled fixed-step iterations with a
    checkpoint every 50 on the 100,000 x 200,000 LP (20 nonzeros per row), FP32
    with FP64 accumulation of the gradients, device buffers, CUDA events; then
    64 instances at m = 5,000 one after another."""
    import torch
    from paper_2508_16806_gb300 import lp as L
    from paper_2508_16806_gb300 import synth
    from paper_2508_16806_gb300 import autograd as AG
    L.load()
    K, ckpt = 500, 50
    lp, xt = synth.adjoint_lp()
    prob = L.Problem(lp, device_copy=True)
    o = L.lp_opts_default(precision=L.LP_PREC_MIXED)
    dev = dict(device="cuda", dtype=torch.float64)
    xK = torch.empty(lp.n, **dev)
    yK = torch.empty(lp.m, **dev)
    assert L.lp_unroll(prob.handle, o, K, xK.data_ptr(), yK.data_ptr(), L.LP_MEM_DEVICE) == 0
    g = 2.0 * (xK - torch.tensor(xt, **dev))
    dc = torch.empty(lp.n, **dev)
    dq = torch.empty(lp.m, **dev)
    dv = torch.empty(lp.nnz, **dev)

    def one():
        s = L.lp_grad(prob.handle, o, K, ckpt, g.data_ptr(), dc.data_ptr(), dq.data_ptr(),
                      dv.data_ptr(), xK.data_ptr(), L.LP_MEM_DEVICE)
        assert s == 0, s

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        one()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    s_ = 4
    pair = 2 * lp.nnz * (s_ + 4)
    # per unrolled step: forward, its recompute in the reverse sweep, the reverse
    # K^T / K products (one SpMV pair each), the SDDMM for dA (row, column, FP64
    # accumulator read and write, four gathered values) and about 20 vector
    # values per row and column
    per_step = 3 * pair + lp.nnz * (4 + 4 + 16 + 4 * s_) + 20 * s_ * (lp.n + lp.m)
    t_batch = time.perf_counter()
    for k in range(64):
        lpk, xk = synth.adjoint_lp(5000, 10000, 20, seed=20250820 + k)
        pk = L.Problem(lpk, device_copy=True)
        xs, _, _ = AG.unroll(pk, K, precision=L.LP_PREC_MIXED)
        AG.grad(pk, K, ckpt, 2.0 * (xs - xk), precision=L.LP_PREC_MIXED)
        pk.close()
    torch.cuda.synchronize()
    batch_s = time.perf_counter() - t_batch
    line = {"metric": "lp_grad time, 500 unrolled iterations (s)", "value": ms / 1e3,
            "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "planted LP 100,000 x 200,000, 20 nonzeros per row, "
                                   "x_target ~ U[0,1]", "K": K, "checkpoint_every": ckpt,
                       "nnz": lp.nnz},
            "unrolled_steps_per_s": K / (ms / 1e3),
            "effective_gbs": per_step * K / (ms / 1e3) / 1e9,
            "bytes_model": "per step 3 SpMV pairs (forward, recompute, reverse) + SDDMM "
                           "nnz*(4+4+16+4s) + 20 s (n + m); working set largely L2-resident",
            "batch_64_at_m5000_s": batch_s,
            "batch_64_note": "64 instances one after another: generate, create, unroll, "
                             "grad (host buffers), destroy",
            "clocks": clk}
    print(json.dumps(line), flush=True)
    prob.close()


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def fp64_error(lp, x, y, info=None):
    """The oracle's FP64 termination quantities (Section 2.3.2) of a returned
    point, its objective against the planted optimum, and the solver's own
    figures beside them."""
    import oracle
    oracle.build()
    k = oracle.kkt(lp, x, y)
    out = {f: k[f] for f in ("rel_gap", "rel_pres", "rel_dres")}
    out["max"] = max(out.values())
    if lp.x_star is not None:
        f = lp.f_star
        out["objective_rel_err_vs_planted"] = abs(float(lp.c @ x) - f) / (1 + abs(f))
    if info is not None:
        out["reported"] = {f: info[f] for f in ("rel_gap", "rel_pres", "rel_dres")}
    return out


def timed_solve(prob, stream, **opts):
    """One lp_solve timed with CUDA events on the solver's stream."""
    import torch
    e0, e1 = _events()
    torch.cuda.synchronize()
    e0.record(stream)
    x, y, info, _ = prob.solve(**opts)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, x, y, info


def dispatch_leg(L, tol):
    """The 615,001 x 5,000 dispatch-shaped LP to tol: the mixed path and the
    plain FP64 path (one warm-up solve each builds the loop graphs), with the
    oracle's FP64 error of each result and the step kernels' times
    (lp_profile_step, CUDA events)."""
    import torch
    from paper_2508_16806_gb300 import synth
    lp = synth.dispatch_lp()
    stream = torch.cuda.Stream()
    prob = L.Problem(lp, device_copy=True, stream=stream)
    out = {"workload": "dispatch-shaped LP 615,001 x 5,000 (nnz %d)" % lp.nnz}
    for prec, tag in ((L.LP_PREC_MIXED, "mixed"), (L.LP_PREC_FP64, "fp64")):
        prob.solve(tol=tol, precision=prec, max_iters=64)
        t, x, y, info = timed_solve(prob, stream, tol=tol, precision=prec, max_iters=2_000_000)
        ms, _ = prob.profile_step(prec, reps=20)
        out[tag] = {"time_to_tol_s": t, "iters": int(info["iters"]),
                    "fp64_iters": int(info["fp64_iters"]), "status": L.STATUS[info["status"]],
                    "fp64_error": fp64_error(lp, x, y, info),
                    "step_kernels_ms": dict(zip(STEP_NAMES, ms))}
    out["mixed_speedup_vs_fp64"] = out["fp64"]["time_to_tol_s"] / out["mixed"]["time_to_tol_s"]
    prob.close()
    return out


def batch_leg(L, tol):
    """The 512 planted LPs: one lp_batch_solve (mixed, autotuned schedules) after
    a warm-up, CUDA events; per-LP device time to tol; the same 512 LPs by the
    batched FP64 path and by a loop of plain FP64 single solves (the FP64 GPU
    path the batched form is compared with: each lp_solve timed with CUDA
    events, creation apart);
    the oracle's FP64 error on a sample of 16 batch results."""
    import torch
    from paper_2508_16806_gb300 import synth
    lps = synth.batch_lps()
    batch = L.Batch(lps)
    out = {"workload": "512 planted LPs, m log-uniform 500..50,000, n = 2m, 5-20 nnz/row",
           "nnz": int(sum(lp.nnz for lp in lps))}
    for prec, tag in ((L.LP_PREC_MIXED, "mixed"), (L.LP_PREC_FP64, "fp64")):
        opts = dict(tol=tol, precision=prec, max_iters=2_000_000, autotune=1)
        batch.solve(**opts)
        e0, e1 = _events()
        torch.cuda.synchronize()
        e0.record(batch.stream)
        res = batch.solve(**opts)
        e1.record(batch.stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        per = sorted(info["solve_s"] for _, _, info in res)
        out["batched_" + tag] = {
            "time_s": t, "lps_per_s": len(lps) / t,
            "per_lp_time_to_tol_s": {"p50": per[len(per) // 2],
                                     "p99": per[min(len(per) - 1, int(0.99 * len(per)))]},
            "statuses": sorted({L.STATUS[i["status"]] for _, _, i in res})}
        if tag == "mixed":
            rng = np.random.default_rng(0)
            errs = [fp64_error(lps[k], res[k][0], res[k][1])["max"]
                    for k in rng.choice(len(lps), 16, replace=False)]
            out["batched_mixed"]["fp64_error_max_of_16"] = max(errs)
    batch.close()
    # plain FP64 single solves of the same LPs
    stream = torch.cuda.Stream()
    solve_s, wall0, statuses = [], time.perf_counter(), set()
    for lp in lps:
        p = L.Problem(lp, device_copy=True, stream=stream)
        t, _, _, info = timed_solve(p, stream, tol=tol, precision=L.LP_PREC_FP64,
                                    max_iters=2_000_000)
        solve_s.append(t)
        statuses.add(L.STATUS[info["status"]])
        p.close()
    loop = sum(solve_s)
    out["fp64_single_solves"] = {"time_s": loop, "wall_s_with_create": time.perf_counter() - wall0,
                                 "lps_per_s": len(lps) / loop,
                                 "per_lp_p50_s": sorted(solve_s)[len(solve_s) // 2],
                                 "statuses": sorted(statuses)}
    out["batched_mixed_speedup_vs_fp64_single"] = loop / out["batched_mixed"]["time_s"]
    return out


def adjoint_leg(L, reps=3):
    """lp_grad of 500 unrolled FP32 iterations (checkpoint every 50) on the
    100,000 x 200,000 LP, device buffers, CUDA events (mean of reps after one
    warm-up)."""
    import torch
    from paper_2508_16806_gb300 import synth
    K, ckpt = 500, 50
    lp, xt = synth.adjoint_lp()
    prob = L.Problem(lp, device_copy=True)
    o = L.lp_opts_default(precision=L.LP_PREC_MIXED)
    dev = dict(device="cuda", dtype=torch.float64)
    xK = torch.empty(lp.n, **dev)
    yK = torch.empty(lp.m, **dev)
    assert L.lp_unroll(prob.handle, o, K, xK.data_ptr(), yK.data_ptr(), L.LP_MEM_DEVICE) == 0
    g = 2.0 * (xK - torch.tensor(xt, **dev))
    dc = torch.empty(lp.n, **dev)
    dq = torch.empty(lp.m, **dev)
    dv = torch.empty(lp.nnz, **dev)

    def one():
        s = L.lp_grad(prob.handle, o, K, ckpt, g.data_ptr(), dc.data_ptr(), dq.data_ptr(),
                      dv.data_ptr(), xK.data_ptr(), L.LP_MEM_DEVICE)
        assert s == 0, s

    one()
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    for _ in range(reps):
        one()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    prob.close()
    # the batch of 64 instances at m = 5,000 (one after another, host buffers)
    from paper_2508_16806_gb300 import autograd as AG
    t_batch = time.perf_counter()
    for k in range(64):
        lpk, xk = synth.adjoint_lp(5000, 10000, 20, seed=20250820 + k)
        pk = L.Problem(lpk, device_copy=True)
        xs, _, _ = AG.unroll(pk, K, precision=L.LP_PREC_MIXED)
        AG.grad(pk, K, ckpt, 2.0 * (xs - xk), precision=L.LP_PREC_MIXED)
        pk.close()
    torch.cuda.synchronize()
    batch_s = time.perf_counter() - t_batch
    return {"workload": "planted LP 100,000 x 200,000, 20 nonzeros per row, K = 500, "
                        "checkpoint every 50, FP32", "lp_grad_s": ms / 1e3,
            "unrolled_steps_per_s": K / (ms / 1e3), "nnz": lp.nnz,
            "batch_64_at_m5000_s": batch_s,
            "batch_64_note": "64 instances 5,000 x 10,000 one after another: generate, create, "
                             "unroll, grad (host buffers), destroy; host wall clock"}


def fishnet_schedule(P):
    """Point counts of the rounds of Algorithm 7 (cull to half; repopulate back
    at odd rounds while more than two points entered the round)."""
    out, cols, i = [], P, 0
    while cols > 1:
        out.append(cols)
        keep = cols // 2
        cols = 2 * keep if (i % 2 == 1 and cols > 2) else keep
        i += 1
    return out


def spmm_bytes(lp, P, s=4):
    """Algorithmic bytes of one fixed PDHG step on P points with s-byte values:
    K^T-side block product with the primal update, then K-side with the dual
    update.  Matrix (s-byte value + 4-byte index per nonzero, row pointers), one
    gathered row of P values per nonzero, point blocks read / written by the
    epilogues, c, l, u, q and sense."""
    t_side = lp.nnz * (s + 4) + (lp.n + 1) * 8 + lp.nnz * P * s + lp.n * P * s * 2 + lp.n * 3 * s
    k_side = lp.nnz * (s + 4) + (lp.m + 1) * 8 + lp.nnz * P * s + lp.m * P * s * 4 + lp.m * (s + 1)
    return t_side + k_side


def fishnet_leg(L, lp, prob, stream, opts, cold_iters, cold_s, rank, P=32, k_steps=20):
    """Algorithm 7 on the bench LP (device-resident draws, CUDA events on the
    solver's stream), then the mixed solve from its point."""
    import torch
    rng = np.random.default_rng(20250821 + rank)
    G = torch.from_numpy(rng.standard_normal((lp.n, P))).to("cuda")
    nz = L.lp_fishnet_draws(P)
    Z = torch.from_numpy(rng.standard_normal(nz)).to("cuda")
    x0 = torch.empty(lp.n, dtype=torch.float64, device="cuda")
    y0 = torch.empty(lp.m, dtype=torch.float64, device="cuda")
    o = L.lp_opts_default(**{k: v for k, v in opts.items() if k != "loop_mode"})
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s = L.lp_fishnet(prob.handle, o, P, k_steps, G.data_ptr(), Z.data_ptr(), nz, x0.data_ptr(),
                     y0.data_ptr(), None, None, L.LP_MEM_DEVICE)
    e1.record(stream)
    torch.cuda.synchronize()
    if s != 0:
        return {"error": L.lp_status_string(s)}
    fish_s = e0.elapsed_time(e1) / 1e3
    e0.record(stream)
    _, _, info, _ = prob.solve(x0=x0.cpu().numpy(), y0=y0.cpu().numpy(), **opts)
    e1.record(stream)
    torch.cuda.synchronize()
    warm_s = e0.elapsed_time(e1) / 1e3
    sched = fishnet_schedule(P)
    s = 4 if o.precision == L.LP_PREC_MIXED else 8
    steps_bytes = sum(k_steps * spmm_bytes(lp, c, s) for c in sched)
    return {"points": P, "k_steps": k_steps, "rounds": len(sched), "points_per_round": sched,
            "fishnet_s": fish_s,
            "precision": "f32 point blocks, f64 gap reductions" if s == 4 else "f64",
            "block_spmm_bytes": steps_bytes,
            "block_spmm_gbs_lower_bound": steps_bytes / fish_s / 1e9,
            "warm_solve_s": warm_s, "warm_iters": int(info["iters"]),
            "warm_status": L.STATUS[info["status"]],
            "cold_solve_s": cold_s, "cold_iters": cold_iters,
            "note": "fishnet_s includes Ruiz, the power iteration, gap reductions, culls and "
                    "host round trips; the bandwidth is therefore a lower bound for the block "
                    "products"}


def fishnet_profile(args):
    import torch
    from paper_2508_16806_gb300 import lp as L
    L.load()
    lp, desc = workload(args.workload)
    stream = torch.cuda.Stream()
    prob = L.Problem(lp, device_copy=True, stream=stream)
    out = fishnet_leg(L, lp, prob, stream, dict(tol=args.tol, precision=L.LP_PREC_MIXED,
                                                max_iters=1), 0, 0.0, 0, P=32, k_steps=2)
    print(json.dumps({"fishnet_profile": desc, "fishnet_s": out.get("fishnet_s")}), flush=True)
    prob.close()


def main():
    args = parse()
    if args.fishnet_profile:
        fishnet_profile(args)
        return
    if args.kernel_profile:
        kernel_profile(args)
        return
    if args.gather_ceiling:
        kernel_profile_gather(args)
        return
    if args.workload == "batch" and args.impl == "ours":
        run_batch(args)
        return
    if args.workload == "adjoint" and args.impl == "ours":
        run_adjoint(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    from paper_2508_16806_gb300 import lp as L

    L.load()
    lp, desc = workload(args.workload, seed_offset=rank)
    stream = torch.cuda.Stream()
    prob = L.Problem(lp, device_copy=True, stream=stream)
    opts = dict(tol=args.tol, precision=L.LP_PREC_MIXED, max_iters=2_000_000,
                loop_mode=1 if args.host_loop else 0, halpern=int(args.method == "halpern"))

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        prob.solve(**opts)
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    infos = []
    ev0.record(stream)
    for _ in range(args.steps):
        x_last, y_last, info, _ = prob.solve(**opts)
        infos.append(info)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
    iters = statistics.mean(i["iters"] for i in infos)
    launches = int(sum(i["kernel_launches"] for i in infos))
    statuses = sorted({L.STATUS[i["status"]] for i in infos})

    # plain FP64 path on the same LP (outside the timed region; one warm-up
    # solve of 64 iterations builds its loop graph)
    prob.solve(tol=args.tol, precision=L.LP_PREC_FP64, max_iters=64)
    fp64_s, x64, y64, i64 = timed_solve(prob, stream, tol=args.tol, precision=L.LP_PREC_FP64,
                                        max_iters=2_000_000)
    # the oracle's FP64 evaluation of both returned points (rank 0)
    err_mixed = err_fp64 = None
    if rank == 0:
        err_mixed = fp64_error(lp, x_last, y_last, infos[-1])
        err_fp64 = fp64_error(lp, x64, y64, i64)

    # per-kernel timing of one step attempt (CUDA events on the solver's stream)
    peak, peak_src = measured_peak()
    rows = {}
    gather = {}
    for prec, tag in ((L.LP_PREC_MIXED, "fp32"), (L.LP_PREC_FP64, "fp64")):
        prob.solve(tol=args.tol, precision=prec, max_iters=256)
        ms_k, by_k = prob.profile_step(prec, reps=30)
        rows[tag] = {n: {"ms": a, "bytes": b, "gbs": (b / (a * 1e-3) / 1e9) if a > 0 else None}
                     for n, a, b in zip(STEP_NAMES, ms_k, by_k) if a > 0}
        if args.workload == "powerlaw":
            gather[tag] = gather_ceiling(prob, prec, lp)
    dom_name = max(("spmv_K_dual", "spmv_KT_primal"), key=lambda n: rows["fp32"][n]["ms"])
    dom = rows["fp32"][dom_name]
    iter_ms = sum(r["ms"] for r in rows["fp32"].values())
    iter_bytes = sum(r["bytes"] for r in rows["fp32"].values())
    # the ncu counters were taken on the power-law LP only
    traffic = NCU_TRAFFIC.get(dom_name) if args.workload == "powerlaw" else None
    roofline = {"bound": "hbm", "achieved": dom["gbs"], "peak": peak, "unit": "GB/s",
                "frac": dom["gbs"] / peak, "traffic": traffic, "kernel": dom_name,
                "peak_source": peak_src,
                "bytes_per_launch": dom["bytes"], "ms_per_launch": dom["ms"]}
    if gather:
        # the same kernel against the gather ceiling of its side (the minimal
        # coalesced-load / gather / multiply-add loop over the same nonzeros)
        side = "K" if dom_name == "spmv_K_dual" else "KT"
        g = gather["fp32"][side]
        roofline["gather_ceiling_ms"] = g["ms"]
        roofline["frac_of_gather_ceiling"] = g["ms"] / dom["ms"]
        roofline["gathers_per_s"] = lp.nnz / (dom["ms"] * 1e-3)

    # end to end through the C ABI with host buffers (H2D of the LP, D2H of x, y)
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        h2d = (lp.row_ptr.nbytes + lp.col_idx.nbytes + lp.vals.nbytes + lp.sense.nbytes +
               lp.c.nbytes + lp.q.nbytes + lp.l.nbytes + lp.u.nbytes)
        d2h = 8 * (lp.n + lp.m)
        times = []
        for _ in range(2):
            t0 = time.perf_counter()
            ph = L.Problem(lp, device_copy=False, stream=stream)
            ph.solve(**opts)
            ph.close()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        e2e = {"value": min(times), "unit": "s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    halp = None
    if not args.no_halpern and args.method == "pdhg":
        halp = halpern_leg(L, prob, stream, opts)

    fish = None
    if not args.no_fishnet:
        fish = fishnet_leg(L, lp, prob, stream, opts, iters, ms / 1e3, rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ref_iters, src = reference_iterations(args.tol, lp)
        if ref_iters is None:
            ref_iters, src = int(i64["iters"]), "GPU FP64 run"
        ot = OracleTimer(lp)
        ot.setup()
        for _ in range(args.cpu_samples):
            ot.sample()
        cpu = {"value": ot.estimate(ref_iters), "unit": "s", "cores": 1, "kind": "oracle",
               "sample": ot.describe(ref_iters, src), "value_is_estimate": True,
               "oracle_iters_per_s": 1.0 / ot.iter_s(),
               "oracle_iters_measured": len(ot.t_iter) * ORACLE_SAMPLE_ITERS, **cpu_info()}

    extra = None
    if rank == 0 and world == 1 and not args.no_extra and args.workload == "powerlaw":
        extra = {"dispatch": dispatch_leg(L, args.tol), "batch": batch_leg(L, args.tol),
                 "adjoint": adjoint_leg(L)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "nnz": lp.nnz, "tol": args.tol,
                       "precision": "FP32 matrix/iterates/SpMV accumulation, FP64 reductions",
                       "step": ("one lp_solve: Ruiz + power iteration + restarted adaptive PDHG "
                                "to tol (setup included)" if args.method == "pdhg" else
                                "one lp_solve: Ruiz + power iteration + restarted reflected "
                                "Halpern PDHG to tol (setup included)"),
                       "l2": (f"inputs larger than L2 (FP32 K and K^T "
                              f"{2 * lp.nnz * 8 / 1e6:.0f} MB + vectors)"
                              if 2 * lp.nnz * 8 > 129e6 else
                              "inputs smaller than L2 (launch-bound case)"),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "statuses": statuses, "iters_to_tol": iters,
            "pdhg_iters_per_s": iters / (ms / 1e3),
            "setup_s": statistics.mean(i["setup_s"] for i in infos),
            "fp64_error": err_mixed,
            "fp64_plain": {"time_to_tol_s": fp64_s, "iters": int(i64["iters"]),
                           "status": L.STATUS[i64["status"]],
                           "spmv_hbm_gbs": rows["fp64"][dom_name]["gbs"],
                           "fp64_error": err_fp64},
            "mixed_speedup_vs_fp64": fp64_s / (ms / 1e3),
            "spmv_hbm_gbs": dom["gbs"],
            "kernels": rows,
            "iteration_gbs": iter_bytes / (iter_ms * 1e-3) / 1e9,
            "roofline": roofline,
            "clocks": clk,
            "gpu_launches": launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "fishnet": fish,
            "halpern": halp,
            "workloads": extra,
        }
        print(json.dumps(line), flush=True)
    prob.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
