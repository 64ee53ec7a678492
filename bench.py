#!/usr/bin/env python
"""LCP-field throughput on the paper-scale synthetic GP field, through the C ABI.

Workload (one step): build the GP model from m=500 observations (anisotropic SE,
lengths (0.15, 0.2, 0.25), noise 1e-4) and compute the level-crossing probability
field of a 128^3 grid (127^3 cells, 1600-sample SOV-QMC estimator) at the 25th,
50th and 75th percentile of y.  Metric: target grid points per second
(3 x 128^3 points per step), as the paper reports seconds per field (Sec. 6.2, Sec. 7.1).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode adaptive|dense]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent replica
(weak scaling, no collective on the data path).
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

import workloads  # noqa: E402

METRIC = "LCP grid points/s"
# Warp instructions k_sov issues per orthant-sample (one lattice point of one orthant,
# P(all < theta) or P(all > theta)): ncu's smsp__inst_executed.sum of the estimator launch of the
# default workload (50,103,618,421; one pass, the launch shapes of a shared tuning table) over the
# orthant-samples the device counted for it (4,051,083,200), profiles/sov_estimator_m500_grid64.txt
# (12.23 on the 64^3 case).  The estimator is issue-bound: its roofline is the
# issue rate, 4 warp instructions per clock on each of 152 SMs at 2.07 GHz; achieved =
# orthant-samples counted on the device x this figure / launch time.
SOV_WARP_INST_PER_ORTHANT_SAMPLE = 12.37
ISSUE_PEAK_GINST = 152 * 4 * 2.07
# Dense tensor peaks relative to BF16 (nominal dense rates: TF32 1.1, BF16 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25
UNIT = "grid points/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--mode", default="adaptive", choices=["dense", "adaptive", "backward", "batched", "sweep"],
                   help="backward: the differentiation workload (m=500 SE, 128^3, median isovalue, U(0,1) "
                        "cell weights): forward field + hand-written adjoint per step; batched: the "
                        "many-model workload (64 SE models, m in [100, 2000], grids 64^3/128^3/256^3) in one "
                        "gpr_lcp_adaptive_batched call per step; sweep: the alpha / beta study of Sec. 7.3 "
                        "(Fig. 5) on the paper-scale field at the median isovalue: per (alpha, beta) the adaptive "
                        "field's time, |S| and MSE against the dense field")
    p.add_argument("--batch-count", type=int, default=64, help="models of the batched workload")
    p.add_argument("--sweep-betas", default="0.5,1,2,6,8,-1", help="sweep mode: beta values (-1: full model)")
    p.add_argument("--api", default="batched", choices=["batched", "single"],
                   help="adaptive mode: the three isovalue fields in one gpr_lcp_adaptive_batched call "
                        "(concurrent fields of one model) or one gpr_lcp_adaptive call each")
    p.add_argument("--prec", default="tf32x3", choices=["fp32", "fp64", "tf32", "tf32x3", "bf16", "bf16x3"],
                   help="precision of the pre-classification / octree pass")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-side-by-side", action="store_true", help="skip the dense / FP32-SIMT comparison runs")
    p.add_argument("--cpu-sample", type=int, default=64, help="cells per axis of the oracle sample")
    p.add_argument("--est", default="sov", choices=["sov", "ordered"],
                   help="small cases only: the cell estimator (index-order or ordered SOV)")
    p.add_argument("--case", default="full", choices=["full", "small", "small_adaptive"],
                   help="small: one dense LCP field of the same field on a 64^3 grid (for ncu captures); "
                        "small_adaptive: one adaptive field (max depth 6) on that grid; "
                        "with --mode backward, the backward step on a 64^3 grid")
    return p.parse_args()


def max_over_ranks(x: float, world: int) -> float:
    """Largest value of x over the ranks (identity for one rank); a CUDA tensor under NCCL, a host
    tensor under gloo."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0])); mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_block(w, cells_per_axis):
    """Cell box [c0, c1) of the bounded oracle sample: a cube of cells at the centre of the grid."""
    c0 = (w.n - 1) // 2 - cells_per_axis // 2
    return (c0, c0, c0), (c0 + cells_per_axis,) * 3


def cpu_baseline(w, theta, cells_per_axis):
    """The FP64 oracle as it stands, on a bounded block of cells straddling the field.  Returns the
    baseline record and the oracle's LCP of the block (x-fastest)."""
    import oracle
    t0 = time.perf_counter()
    om = oracle.Model.from_workload(w)
    c, c1 = oracle_block(w, cells_per_axis)
    vals = om.lcp_block(w.n, theta, c, c1)
    dt = time.perf_counter() - t0
    cells = cells_per_axis ** 3
    return {"value": cells / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"model set-up + SOV-1600 LCP of a {cells_per_axis}^3-cell block at the median isovalue "
                      f"({cells} cells ~ grid points), {dt:.1f} s"}, vals


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workloads.config2()
    import oracle
    theta = w.isovalues[1]
    k = max(6, args.cpu_sample // 2)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        om = oracle.Model.from_workload(w)
        c0 = (w.n - 1) // 2 - k // 2
        om.lcp_block(w.n, theta, (c0, c0, c0), (c0 + k, c0 + k, c0 + k))
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    v = k ** 3 / t
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{w.name}, 3 isovalues (P25/P50/P75 of y), SOV-QMC 1600, {args.mode}",
                      "m": w.m, "grid": w.n, "mode": args.mode,
                      "sample": f"{k}^3 cells at the median isovalue (every cell of the block, oracle)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"{k}^3-cell block per step, model set-up included"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_backward(args, g, torch, rank, world, local):
    """Forward LCP field + gpr_lcp_backward on the differentiation workload; metric: grid points/s
    of (forward + backward) steps."""
    w = workloads.config5()
    n = 64 if args.case == "small" else w.n
    grid = g.make_grid(n)
    th = w.isovalues[0]
    opts = g.lcp_options(prec=g.GPR_P_TF32X3)
    cw = w.extra["cell_weights"] if n == w.n else np.random.default_rng(5).random((n - 1) ** 3)
    wts = torch.tensor(cw, dtype=torch.float32, device="cuda")
    field = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    split_ev, dstats = [], []

    def step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        M = g.gpr_model_create(w.X, w.y, w.kernel, w.ell, w.sf2, w.sn2, stream=stream)
        dstats[:] = [g.gpr_lcp_dense(M, grid, th, opts, field, stream=stream)]
        ev[1].record(stream)
        dy, dl = g.gpr_lcp_backward(M, grid, th, opts, wts, stream=stream)
        ev[2].record(stream)
        split_ev.append(ev)
        M.close()
        return dy, dl

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g.gpr_profile_reset(); g.gpr_profile_enable(True)
    split_ev.clear()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            dy, dl = step()
        e1.record(stream)
        torch.cuda.synchronize()
    g.gpr_profile_enable(False)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    prof = {k: g.gpr_profile_read(k) for k in ("w64", "oz_adig", "oz_w", "stats_ff", "tc_sumsq", "stats_from_w64", "sov", "adj_cell", "adj_prep", "adj_sample", "adj_chol", "adj_zhat", "adj_R", "adj_Z", "adj_points")}
    if rank != 0:
        return
    out = {"metric": METRIC + " (forward + backward)", "value": world * n ** 3 / (ms / 1e3), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
           "config": {"workload": f"{w.name}: loss = sum_c U(0,1)_c LCP_c, d/dy (500) and d/dlog l (3)",
                      "grid": n},
           "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
           "forward_ms": float(np.mean([e[0].elapsed_time(e[1]) for e in split_ev])),
           "corner_points": dstats[0]["recon_points"], "cells_estimated": dstats[0]["cells_estimated"],
           "backward_ms": float(np.mean([e[1].elapsed_time(e[2]) for e in split_ev])),
           "grad_norm_y": float(np.linalg.norm(dy)), "grad_loglen": [float(v) for v in dl],
           "clocks": clk.summary(), "gpu_launches": g.gpr_launch_count()}
    print(json.dumps(out), flush=True)


def run_batched(args, g, torch, rank, world, local):
    """Many-model workload: per step, every model is built from host arrays and all adaptive
    fields (median isovalue each) go out in one gpr_lcp_adaptive_batched call."""
    ws = workloads.config4(args.batch_count)
    opts = g.lcp_options(prec=g.GPR_P_TF32X3)
    stream = torch.cuda.current_stream()
    grids = [g.make_grid(w.n) for w in ws]
    fields = [torch.zeros((w.n - 1) ** 3, dtype=torch.float32, device="cuda") for w in ws]
    host = [torch.zeros((w.n - 1) ** 3, dtype=torch.float32).pin_memory() for w in ws]
    stats_last = []

    def step(e2e=False):
        models = [g.gpr_model_create(w.X, w.y, w.kernel, w.ell, w.sf2, w.sn2, stream=stream) for w in ws]
        st = g.gpr_lcp_adaptive_batched(models, grids, [w.isovalues[0] for w in ws], [w.max_depth for w in ws],
                                        opts, fields, stream=stream)
        stats_last[:] = st
        if e2e:
            for h, f in zip(host, fields):
                h.copy_(f, non_blocking=True)
        return models

    for _ in range(args.warmup):
        for M in step():
            M.close()
    torch.cuda.synchronize()
    g.gpr_sync(stream)
    g.gpr_profile_reset(); g.gpr_profile_enable(True)
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            for M in step():  # models are built and destroyed inside the step
                M.close()
        e1.record(stream)
        torch.cuda.synchronize()
    g.gpr_profile_enable(False)
    launches = g.gpr_launch_count()
    g.gpr_sync(stream)
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    prof = {k: g.gpr_profile_read(k) for k in ("oz_adig", "oz_w", "stats_ff", "tc_sumsq", "mean_ff", "w64", "cell_prep", "sov",
                                                "oct_eval_w", "oct_level")}
    orth = g.gpr_profile_units("sov_orthants")
    e0.record(stream)
    for _ in range(args.steps):
        for M in step(e2e=True):
            M.close()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    if rank != 0:
        return
    pts = sum(w.n ** 3 for w in ws)
    est = sum(s["cells_estimated"] for s in stats_last)
    roof = None
    c, n_launch = prof["sov"]
    if n_launch > 0:
        # the shared estimator runs alone on the caller's stream after every field's octree
        avg_s = c / n_launch / 1e3
        inst = SOV_WARP_INST_PER_ORTHANT_SAMPLE * orth * opts.n_samples / n_launch
        roof = {"bound": "alu", "achieved": inst / avg_s / 1e9, "peak": ISSUE_PEAK_GINST, "unit": "Gwarp-inst/s",
                "traffic": None, "kernel": "k_sov (SOV-QMC estimator over every field's cells, one persistent launch)",
                "peak_source": "issue rate 4 warp-inst/clk x 152 SMs x 2.07 GHz (recipe unit counts and clock)"}
        roof["frac"] = roof["achieved"] / roof["peak"]
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(ws[0], ws[0].isovalues[0], min(32, ws[0].n - 1))[0]
    out = {"metric": METRIC, "value": world * pts / (ms / 1e3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
           "config": {"workload": f"{len(ws)} SE models, m log-uniform [100, 2000], l in [0.05, 0.3], "
                                  f"grids 64^3/128^3/256^3, median isovalue, adaptive, batched",
                      "models": len(ws), "grid_points": pts, "m": [w.m for w in ws], "grid": [w.n for w in ws],
                      "l2": "working set > L2", "parallelism": f"replicas x{world}"},
           "roofline": roof,
           "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
           "kept_cells": sum(s["leaf_cells"] for s in stats_last), "cells_estimated": est,
           "cpu_baseline": cpu,
           "e2e": {"value": world * pts / (ms_e2e / 1e3), "unit": UNIT,
                   "h2d_bytes_per_step": int(sum(w.X.nbytes + w.y.nbytes for w in ws)),
                   "d2h_bytes_per_step": int(sum((w.n - 1) ** 3 * 4 for w in ws))},
           "gpu_launches": launches, "clocks": clk.summary()}
    print(json.dumps(out), flush=True)


def run_sweep(args, g, torch, rank, world, local):
    """Sec. 7.3's hyperparameter study on the paper-scale field (m=500, 128^3, median isovalue):
    for every alpha in 1e-1 .. 1e-7 and beta in --sweep-betas (full model: -1), the adaptive field
    of a freshly built model (CUDA-event time of the gpr_lcp_adaptive call; model set-up excluded),
    its |S| and its MSE and max |dLCP| against the dense field of the same estimator."""
    w = workloads.config2()
    n, th = w.n, w.isovalues[1]
    grid = g.make_grid(n)
    stream = torch.cuda.current_stream()
    dense = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
    field = torch.zeros_like(dense)
    M = g.gpr_model_create(w.X, w.y, w.kernel, w.ell, w.sf2, w.sn2, stream=stream)
    g.gpr_lcp_dense(M, grid, th, g.lcp_options(prec=g.GPR_P_TF32X3), dense, stream=stream)
    M.close()
    alphas = [1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7]
    # beta in length scales; 8 and above cover the domain on every axis here (the full model's
    # bound); 6 (the paper's value) leaves out a few far observations for boundary nodes
    betas = [float(b) for b in args.sweep_betas.split(",")]
    rows = []

    def one(alpha, beta):
        Mf = g.gpr_model_create(w.X, w.y, w.kernel, w.ell, w.sf2, w.sn2, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        st = g.gpr_lcp_adaptive(Mf, grid, th, w.max_depth, g.lcp_options(prec=g.GPR_P_TF32X3, alpha=alpha, beta=beta),
                                field, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        Mf.close()
        d = (field - dense).double()
        return {"alpha": alpha, "beta": beta if beta >= 0 else None, "ms": e0.elapsed_time(e1),
                "leaf_cells": st["leaf_cells"], "mse": float((d * d).mean()), "max_abs_dlcp": float(d.abs().max())}

    for _ in range(max(1, args.warmup)):
        one(1e-3, -1.0)
    with ClockSampler(local) as clk:
        for a in alphas:
            for b in betas:
                rows.append(one(a, b))
    if rank != 0:
        return
    ref = next(r for r in rows if r["alpha"] == 1e-3 and r["beta"] is None)
    out = {"metric": METRIC + " (alpha/beta study)", "value": n ** 3 / (ref["ms"] / 1e3), "unit": UNIT,
           "n_gpus": world, "steps": len(rows), "warmup": args.warmup, "ms_per_step": ref["ms"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
           "config": {"workload": f"{w.name}, median isovalue, adaptive D=7, SOV-QMC 1600; value/ms_per_step: "
                                  "alpha 1e-3 with the full model", "grid": n, "m": w.m},
           "sweep": rows, "dense_cells_nonzero": int((dense > 0).sum().item()),
           "clocks": clk.summary(), "gpu_launches": g.gpr_launch_count()}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import paper_2512_12442_gb300 as g

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = workloads.config2()
    if args.case in ("small", "small_adaptive") and args.mode != "backward":
        n = 64
        grid = g.make_grid(n)
        out = torch.zeros((n - 1) ** 3, dtype=torch.float32, device="cuda")
        M = g.gpr_model_create(w.X, w.y, w.kernel, w.ell, w.sf2, w.sn2)
        g.gpr_profile_reset(); g.gpr_profile_enable(True)
        est = g.GPR_EST_SOV_ORDERED if args.est == "ordered" else g.GPR_EST_SOV_QMC
        o = g.lcp_options(prec=g.GPR_P_TF32X3, est=est)
        if args.case == "small":
            st = g.gpr_lcp_dense(M, grid, w.isovalues[1], o, out)
        else:
            st = g.gpr_lcp_adaptive(M, grid, w.isovalues[1], 6, o, out)
        g.gpr_sync()
        g.gpr_profile_enable(False)
        print(json.dumps({"case": "small", "grid": n, "m": w.m, "est": args.est,
                          **{k: st[k] for k in ("recon_points", "leaf_cells", "cells_estimated")},
                          "sov_orthants": g.gpr_profile_units("sov_orthants"),
                          "sov_launches": g.gpr_profile_read("sov" if args.est == "sov" else "sov_ordered")[1]}))
        return
    if args.mode == "backward":
        run_backward(args, g, torch, rank, world, local)
        return
    if args.mode == "batched":
        run_batched(args, g, torch, rank, world, local)
        return
    if args.mode == "sweep":
        run_sweep(args, g, torch, rank, world, local)
        return
    n = w.n
    ncell = (n - 1) ** 3
    grid = g.make_grid(n)
    precs = {"fp64": g.GPR_P_FP64, "fp32": g.GPR_P_FP32, "tf32": g.GPR_P_TF32, "tf32x3": g.GPR_P_TF32X3,
             "bf16": g.GPR_P_BF16, "bf16x3": g.GPR_P_BF16X3}
    opts = g.lcp_options(prec=precs[args.prec])
    stream = torch.cuda.current_stream()
    fields = [torch.zeros(ncell, dtype=torch.float32, device="cuda") for _ in w.isovalues]
    host = [torch.zeros(ncell, dtype=torch.float32).pin_memory() for _ in w.isovalues]
    stats_last = {}

    def step(mode=args.mode, o=opts, e2e=False):
        M = g.gpr_model_create(w.X, w.y, w.kernel, w.ell, w.sf2, w.sn2, stream=stream)
        if mode == "adaptive" and args.api == "batched":
            nf = len(w.isovalues)
            sts = g.gpr_lcp_adaptive_batched([M] * nf, [grid] * nf, list(w.isovalues), [w.max_depth] * nf, o,
                                             fields, stream=stream)
            for t in range(nf):
                stats_last[t] = sts[t]
                if e2e:
                    host[t].copy_(fields[t], non_blocking=True)
            return M
        for t, th in enumerate(w.isovalues):
            if mode == "dense":
                st = g.gpr_lcp_dense(M, grid, th, o, fields[t], stream=stream)
            else:
                st = g.gpr_lcp_adaptive(M, grid, th, w.max_depth, o, fields[t], stream=stream)
            stats_last[t] = st
            if e2e:
                host[t].copy_(fields[t], non_blocking=True)
        return M

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    def timed(k, **kw):
        """CUDA-event milliseconds per step over k steps (barrier + synchronize on both sides)."""
        barrier()
        ev0 = torch.cuda.Event(enable_timing=True); ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(k):
            step(**kw).close()
        ev1.record(stream)
        barrier()
        g.gpr_sync(stream)
        return ev0.elapsed_time(ev1) / k

    for _ in range(args.warmup):
        step().close()
    g.gpr_sync(stream)

    # headline: device-resident inputs, tracing off
    g.gpr_profile_reset()
    with ClockSampler(local) as clk:
        ms = timed(args.steps)
    launches = g.gpr_launch_count()
    t_max = max_over_ranks(ms, world)
    pts_per_step = len(w.isovalues) * n ** 3
    value = world * pts_per_step / (t_max / 1e3)

    # end to end: host inputs in, the fields copied back to pinned host memory every step
    ms_e2e = max_over_ranks(timed(args.steps, e2e=True), world)

    # the same steps again with the tracer on: per-stage CUDA-event times and work units
    g.gpr_profile_reset()
    g.gpr_profile_enable(True)
    ms_traced = timed(args.steps)
    g.gpr_profile_enable(False)
    names = ("w64", "oz_adig", "oz_w", "stats_ff", "meanvar32", "tc_sumsq", "mean_ff", "stats_from_w64",
             "cell_prep", "sov", "classify", "oct_eval_w", "oct_level")
    prof = {k: g.gpr_profile_read(k) for k in names}
    units = {k: g.gpr_profile_units(k) for k in ("oz_w", "oz_adig", "stats_ff", "tc_sumsq", "sov_orthants")}
    g.gpr_sync(stream)

    # the same field by the other paths, side by side at the same accuracy (same FP64-class leaf
    # statistics and estimator): dense with the TF32x3 pre-pass, dense with the plain FP32 SIMT
    # pre-pass; and the adaptive path with the ordered SOV estimator (its own, more accurate
    # estimate: the largest and mean per-cell difference from the default fields are reported)
    side = {}
    if args.mode == "adaptive" and not args.no_side_by_side:
        ordered = None
        for label, mode, pr, est in (("dense_tf32x3", "dense", "tf32x3", g.GPR_EST_SOV_QMC),
                                     ("dense_fp32_simt", "dense", "fp32", g.GPR_EST_SOV_QMC),
                                     ("adaptive_ordered_sov", "adaptive", args.prec, g.GPR_EST_SOV_ORDERED)):
            o2 = g.lcp_options(prec=precs[pr], est=est)
            step(mode=mode, o=o2).close()
            k2 = max(1, min(args.steps, 3))
            t2 = max_over_ranks(timed(k2, mode=mode, o=o2), world)
            side[label] = {"ms_per_step": t2, "value": world * pts_per_step / (t2 / 1e3), "steps": k2}
            if est == g.GPR_EST_SOV_ORDERED:
                ordered = [f.clone() for f in fields]
        step().close()  # the default path's fields again, for the accuracy check below
        g.gpr_sync(stream)
        if ordered is not None:
            d = [(a - b).abs() for a, b in zip(ordered, fields)]
            side["adaptive_ordered_sov"]["max_abs_diff_vs_default"] = max(float(x.max()) for x in d)
            side["adaptive_ordered_sov"]["mean_abs_diff_vs_default_on_nonzero"] = float(
                sum(float(x[f != 0].sum()) for x, f in zip(d, fields)) / max(1, sum(int((f != 0).sum()) for f in fields)))

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    m = w.m
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    bf16_sus = float(peaks.get("bf16_tflops_sustained") or 1733.1)
    est_cells = sum(stats_last[t]["cells_estimated"] for t in stats_last)

    def per_step(k):
        return prof[k][0] / args.steps

    # roofline of the dominant kernel (oct_level spans whole octree levels, not one kernel)
    kern = {k: v for k, v in prof.items() if k != "oct_level" and v[1] > 0}
    dom = max(kern, key=lambda k: kern[k][0]) if kern else None
    roof = None
    if dom == "sov" and units["sov_orthants"] > 0:
        # orthant-samples counted on the device (orthants queued x samples), per launch
        avg_s = prof["sov"][0] / prof["sov"][1] / 1e3
        osamp = units["sov_orthants"] * opts.n_samples / prof["sov"][1]
        inst = SOV_WARP_INST_PER_ORTHANT_SAMPLE * osamp
        roof = {"bound": "alu", "achieved": inst / avg_s / 1e9, "peak": ISSUE_PEAK_GINST, "unit": "Gwarp-inst/s",
                "traffic": None, "kernel": "k_sov (SOV-QMC estimator, FP32)",
                "orthant_samples_per_launch": osamp, "orthant_samples_per_s": osamp / avg_s,
                "peak_source": "issue rate 4 warp-inst/clk x 152 SMs x 2.07 GHz (recipe unit counts and clock); "
                               f"{SOV_WARP_INST_PER_ORTHANT_SAMPLE} warp-inst per orthant-sample from ncu"}
    elif dom == "oz_w" and units["oz_w"] > 0:
        mp = (m + 63) // 64 * 64
        kk = sum(64 * ((min(n0 + 64, m) + 31) // 32 * 32) for n0 in range(0, mp, 64))
        flops = 28 * 2 * units["oz_w"] * kk
        roof = {"bound": "tensor", "achieved": flops / (prof["oz_w"][0] / 1e3) / 1e12, "peak": bf16_sus,
                "unit": "TFLOP/s", "traffic": None, "kernel": "k_oz_gemm (FP64-class whitening GEMM, BF16 digit split)",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained"}
    if roof:
        roof["frac"] = roof["achieved"] / roof["peak"]

    # tensor-pipe throughput of the two contractions (CUDA-event time, FLOPs from the rows processed)
    tensor = {}
    if prof["tc_sumsq"][1] > 0 and units["tc_sumsq"] > 0:
        nprod = {"tf32x3": 3, "bf16x3": 6, "tf32": 1, "bf16": 1}.get(args.prec, 1)
        fl = nprod * m * (m + 1) * units["tc_sumsq"]  # triangular whitening w = L^-1 k: m(m+1) per product
        pk = bf16_sus * (TF32_OVER_BF16 if args.prec.startswith("tf32") else 1.0)
        tensor["k_tc_sumsq"] = {"ms_per_step": per_step("tc_sumsq"), "points_per_step": units["tc_sumsq"] / args.steps,
                                "tflops": fl / (prof["tc_sumsq"][0] / 1e3) / 1e12, "peak_tflops": pk,
                                "flops": f"{nprod} products x m(m+1) per point (algorithmic)"}
        tensor["k_tc_sumsq"]["frac"] = tensor["k_tc_sumsq"]["tflops"] / pk
    if prof["oz_w"][1] > 0 and units["oz_w"] > 0:
        mp = (m + 63) // 64 * 64
        kk = sum(64 * ((min(n0 + 64, m) + 31) // 32 * 32) for n0 in range(0, mp, 64))
        fl = 28 * 2 * units["oz_w"] * kk
        tensor["k_oz_gemm"] = {"ms_per_step": per_step("oz_w"), "rows_per_step": units["oz_w"] / args.steps,
                               "tflops": fl / (prof["oz_w"][0] / 1e3) / 1e12, "peak_tflops": bf16_sus,
                               "fp64_equiv_tflops": m * (m + 1) * units["oz_w"] / (prof["oz_w"][0] / 1e3) / 1e12,
                               "flops": "28 digit products x 2 x sum of the 64-column tiles' K ranges per row "
                                        "(issued BF16 work); fp64_equiv: m(m+1) per row"}
        tensor["k_oz_gemm"]["frac"] = tensor["k_oz_gemm"]["tflops"] / bf16_sus

    # accuracy against the FP64 oracle on the bounded sample block (median isovalue)
    cpu, acc = None, None
    if not args.no_cpu_baseline:
        cpu, ovals = cpu_baseline(w, w.isovalues[1], args.cpu_sample)
        (a0, b0, z0), (a1, b1, z1) = oracle_block(w, args.cpu_sample)
        blk = fields[1].cpu().numpy().reshape(n - 1, n - 1, n - 1)[z0:z1, b0:b1, a0:a1].reshape(-1).astype(np.float64)
        d = np.abs(blk - ovals)
        acc = {"block": f"cells [{a0},{a1})^3 of the 127^3 grid, median isovalue, {ovals.size} cells",
               "max_abs_dLCP_vs_fp64": float(d.max()), "mean_abs_dLCP_vs_fp64": float(d.mean()),
               "tolerance": 1e-4}
        if args.mode == "adaptive":
            nodes, dec, _ = g.gpr_octree_trace(M_acc := g.gpr_model_create(w.X, w.y, w.kernel, w.ell, w.sf2, w.sn2),
                                               grid, w.isovalues[1], w.max_depth, opts, w.max_depth)
            M_acc.close()
            leaf = nodes[dec > 0]
            lin = (leaf & 0x1FFFFF) + (n - 1) * (((leaf >> 21) & 0x1FFFFF) + (n - 1) * ((leaf >> 42) & 0x1FFFFF))
            inS = np.zeros(ncell, bool); inS[lin] = True
            sblk = inS.reshape(n - 1, n - 1, n - 1)[z0:z1, b0:b1, a0:a1].reshape(-1)
            acc["on_S"] = {"cells": int(sblk.sum()), "max_abs_dLCP_vs_fp64": float(d[sblk].max()) if sblk.any() else 0.0}
            acc["off_S"] = {"cells": int((~sblk).sum()),
                            "max_oracle_LCP": float(ovals[~sblk].max()) if (~sblk).any() else 0.0,
                            "note": "cells Algorithm 1 dropped (adaptive field 0): the method's approximation, "
                                    "bounded by alpha per region"}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "fp32", "data": "synthetic",
        "config": {"workload": f"{w.name}, 3 isovalues (P25/P50/P75 of y), SOV-QMC 1600, {args.mode}",
                   "m": m, "grid": n, "mode": args.mode, "prepass": args.prec,
                   "arithmetic": "FP64 model set-up; FP64-class corner statistics (BF16 tensor-core digit split, "
                                 "float-float); FP32 estimator; pre-pass/octree in " + args.prec,
                   "api": args.api if args.mode == "adaptive" else "single",
                   "l2": "working set > L2 (FP64-class whitened rows of the kept points, GBs)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "tensor_pipe": tensor,
        "accuracy": acc,
        "side_by_side": side,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "traced_ms_per_step": ms_traced,
        "kernel_ms_note": ("CUDA-event times from a separate traced pass (the headline pass runs untraced); with "
                           "api=batched the three fields' octree and leaf stages run on worker streams and their "
                           "times overlap (the estimator is one launch)"),
        "kept_cells": [stats_last[t]["leaf_cells"] for t in stats_last],
        "recon_points": [stats_last[t]["recon_points"] for t in stats_last],
        "cells_estimated": est_cells,
        "cpu_baseline": cpu,
        "e2e": {"value": world * pts_per_step / (ms_e2e / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(w.X.nbytes + w.y.nbytes),
                "d2h_bytes_per_step": int(len(w.isovalues) * ncell * 4)},
        "gpu_launches": launches,
        "autotune": {f"{k[0]}@{k[1]}": v for k, v in g.gpr_autotune_table().items()},
        "clocks": clk.summary(),
        "measured_peaks": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained")},
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
