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
# dominant kernel from one ncu capture of the current kernel source; None when
# the kernel changed after the capture.  Summary: profiles/spmv_powerlaw_1Mx2M_fp32.md
NCU_TRAFFIC = {"spmv_KT_step": 186126336, "spmv_K_dual": 200254976}


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
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fishnet", action="store_true",
                   help="skip the Algorithm 7 warm-start measurement (extra key)")
    p.add_argument("--fp64-profile", action="store_true",
                   help="with --kernel-profile: also time the FP64 step kernels")
    p.add_argument("--fishnet-profile", action="store_true",
                   help="one lp_fishnet call on the workload (32 points, 2 steps per round), "
                        "for kernel profilers; prints its time")
    p.add_argument("--host-loop", action="store_true",
                   help="host-driven loop graph (lp_opts.loop_mode = 1), for ncu launch lists")
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
    names = ["primal_halpern", "spmv_K_halpern_dual", "spmv_KT_step"]
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
    all_lps = synth.batch_lps()
    # independent LPs: each rank solves its share (weak scaling: 512 LPs per rank,
    # the same 512 shifted by rank so that every rank has a full batch)
    lps = all_lps if world == 1 else synth.batch_lps(seed=20250819 + 512 * rank)
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
            "value": world * len(lps) / (ms / 1e3), "unit": "LP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "512 planted LPs, m log-uniform 500..50,000, n = 2m, 5-20 nnz/row",
                       "nnz": int(sum(lp.nnz for lp in lps)), "tol": args.tol,
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


def oracle_estimate(lp, iters_to_tol, small_sample=False):
    """Times the FP64 CPU oracle on a bounded sample of the workload and scales
    it to a time-to-tolerance estimate (seconds): Ruiz (10 passes, timed in
    full), 100 power iterations (per-iteration time from a short run), and
    iters_to_tol PDHG iterations (per-iteration time from the difference of a
    4- and a 12-iteration run, plus one KKT check per 64 iterations costed as
    two iterations)."""
    import oracle
    oracle.build()
    t = time.perf_counter()
    oracle.ruiz(lp, 10, 1e-4)
    t_ruiz = time.perf_counter() - t
    t = time.perf_counter()
    oracle.power_norm(lp, 1)
    t1 = time.perf_counter() - t
    t = time.perf_counter()
    oracle.power_norm(lp, 3)
    t3 = time.perf_counter() - t
    t_pow = max(t3 - t1, 0.0) / 2
    a, b = (4, 12)
    t = time.perf_counter()
    oracle.solve(lp, tol=0.0, max_iters=a, check_every=a, ruiz_iters=0, power_iters=1)
    ta = time.perf_counter() - t
    t = time.perf_counter()
    oracle.solve(lp, tol=0.0, max_iters=b, check_every=b, ruiz_iters=0, power_iters=1)
    tb = time.perf_counter() - t
    t_iter = max(tb - ta, 1e-9) / (b - a)
    est = t_ruiz + 100 * t_pow + iters_to_tol * t_iter * (1 + 2 / 64)
    sample = (f"Ruiz 10 passes ({t_ruiz:.2f} s), power iteration per-step {t_pow:.3f} s x 100, "
              f"PDHG {t_iter:.3f} s/iteration from a {a}- vs {b}-iteration run, scaled to "
              f"{iters_to_tol} iterations (+1 check per 64 iterations)")
    return est, t_iter, sample


def reference_iterations(tol):
    path = os.path.join(ROOT, "oracle", "reference_runs.json")
    try:
        for r in json.load(open(path)):
            if abs(r["tol"] - tol) < 1e-15 and r["status"] == 1:
                return int(r["iters"]), "oracle run to tolerance (oracle/reference_runs.json)"
    except Exception:
        pass
    return None, None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    lp, desc = workload(args.workload)
    iters, src = reference_iterations(args.tol)
    if iters is None:
        iters, src = 5000, "assumed 5000 iterations (no stored oracle run)"
    vals = []
    sample = ""
    for s in range(args.warmup + args.steps):
        est, t_iter, sample = oracle_estimate(lp, iters)
        if s >= args.warmup:
            vals.append(est)
    v = float(statistics.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "tol": args.tol, "iterations_to_tol": iters,
                       "iterations_source": src},
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": sample},
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
        _, _, info, _ = prob.solve(**opts)
        infos.append(info)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
    iters = statistics.mean(i["iters"] for i in infos)
    launches = int(sum(i["kernel_launches"] for i in infos))
    statuses = sorted({L.STATUS[i["status"]] for i in infos})

    # plain FP64 path on the same LP (outside the timed region)
    t0 = time.perf_counter()
    _, _, i64, _ = prob.solve(tol=args.tol, precision=L.LP_PREC_FP64, max_iters=2_000_000)
    torch.cuda.synchronize()
    fp64_s = time.perf_counter() - t0

    # per-kernel timing of one step attempt (CUDA events on the solver's stream)
    peak, peak_src = measured_peak()
    rows = {}
    for prec, tag in ((L.LP_PREC_MIXED, "fp32"), (L.LP_PREC_FP64, "fp64")):
        prob.solve(tol=args.tol, precision=prec, max_iters=256)
        ms_k, by_k = prob.profile_step(prec, reps=30)
        names = ["primal_update", "spmv_K_dual", "spmv_KT_step", "step_control"]
        rows[tag] = {n: {"ms": a, "bytes": b, "gbs": (b / (a * 1e-3) / 1e9) if a > 0 else None}
                     for n, a, b in zip(names, ms_k, by_k)}
    dom_name = max(("spmv_K_dual", "spmv_KT_step"), key=lambda n: rows["fp32"][n]["ms"])
    dom = rows["fp32"][dom_name]
    iter_ms = sum(r["ms"] for r in rows["fp32"].values())
    iter_bytes = sum(r["bytes"] for r in rows["fp32"].values())
    # the ncu counters were taken on the power-law LP only
    traffic = NCU_TRAFFIC.get(dom_name) if args.workload == "powerlaw" else None
    roofline = {"bound": "hbm", "achieved": dom["gbs"], "peak": peak, "unit": "GB/s",
                "frac": dom["gbs"] / peak, "traffic": traffic, "kernel": dom_name,
                "peak_source": peak_src,
                "bytes_per_launch": dom["bytes"], "ms_per_launch": dom["ms"]}

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
        ref_iters, src = reference_iterations(args.tol)
        if ref_iters is None:
            ref_iters, src = int(i64["iters"]), "iterations of the GPU FP64 run"
        est, t_iter, sample = oracle_estimate(lp, ref_iters)
        cpu = {"value": est, "unit": "s", "cores": 1, "kind": "oracle",
               "sample": sample + f"; iteration count from the {src}",
               "oracle_iters_per_s": 1.0 / t_iter}

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
            "fp64_plain": {"time_to_tol_s": fp64_s, "iters": int(i64["iters"]),
                           "status": L.STATUS[i64["status"]],
                           "spmv_hbm_gbs": rows["fp64"][dom_name]["gbs"]},
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
        }
        print(json.dumps(line), flush=True)
    prob.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
