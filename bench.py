#!/usr/bin/env python
"""CTMRG moves/s on one GB300: U(1) one-site cell, D=6, chi=72, full move.

One step = the whole hot path on the fixed seeded inputs: double layer with
remover (S0), then the LEFT, RIGHT, UP, DOWN directional moves, each
building the four enlarged corners, the half systems, the SVD projectors,
and renormalising and normalising the renewed environment tensors.
The environment is restored from a device copy before every step.

Prints one JSON line (rank 0).  --impl reference times the dense FP64 CPU
oracle on the host cores instead.  With N>1 ranks every rank runs an
independent replica of the move (it does not shard; no collective on the
data path) and the value is the sum over ranks; the batch of independent
contractions is split over the ranks instead (balanced by block-pair work,
no exchange), timed as the slowest rank's share.
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

WORKLOAD = "d6chi72"
METRIC = "CTMRG moves/s & block-sparse TFLOP/s vs plain FP64 GPU path at rel err <=1e-9"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            with open(p) as f:
                d = json.load(f)
            d["source"] = "measured"
            return d
        except Exception:
            pass
    return dict(FALLBACK_PEAKS)


class Clocks:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index, self.lines, self.proc = index, [], None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
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
        sm, mx, reasons = [], 0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def ncu_traffic(kernel_class):
    """DRAM bytes per launch of a kernel class from the committed ncu capture
    (profiles/dram_traffic.json), or None when there is none or a source file
    of the kernel changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            e = json.load(f).get(kernel_class)
        if not e:
            return None
        for src, h in zip(e["sources"], e["sha256"]):
            with open(os.path.join(ROOT, src), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != h:
                    return None
        return float(e["bytes_per_launch"])
    except Exception:
        return None


def job_ms(ms_local, world):
    """Whole-job time per step: the slowest rank's (MAX over ranks, gloo)."""
    if world <= 1:
        return float(ms_local)
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(ms, world):
    """Replicas: every rank completes one move per step, so the job rate is
    world moves per (slowest) step time."""
    return world * 1e3 / ms


def cpu_oracle_time(steps=1, warmup=0):
    """Dense FP64 oracle: double layer + full move of the same workload on the
    host cores; returns (seconds per move list, cores)."""
    import numpy as np
    from oracle import ctm as octm
    from workloads import u1_config
    cfg = u1_config(WORKLOAD)
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        net = octm.u1_network(cfg)
        octm.full_move(net, cfg["chi"])
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
    return times, os.cpu_count()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    times, cores = cpu_oracle_time(args.steps, args.warmup)
    v = 1.0 / statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "moves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "u1_D6_chi72_full_move", "D": 6, "chi": 72},
            "cpu_baseline": {"value": v, "unit": "moves/s", "cores": cores, "kind": "oracle",
                             "sample": "one full move (double layer + L,R,U,D) per step, dense numpy FP64"},
            "e2e": {"value": v, "unit": "moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BATCH_LEGS = ((0, 2), (1, 0))   # X2[k_u, x_r, k_l, x_d] . a[k_l, k_u, k_r, k_d] over (k_u, k_l)


def batch_partition(costs, world):
    """Split independent contractions over `world` ranks with no exchange:
    longest first, each to the least loaded rank (ties: lower index).
    Returns one ascending index list per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load, parts = [0.0] * world, [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def batch_instances(bst, ctx, dev, count=64):
    """The batch of independent corner contractions (D ~ U{4..8},
    chi ~ U{32,64,96,128}): per entry the double layer a of a seeded site
    tensor and a seeded X2 block-sparse tensor."""
    import torch
    from workloads import batched_site_legs, batched_u1_configs, values
    out = []
    for cfg in batched_u1_configs(count):
        A = ctx.layout([bst.Leg(l["flow"], l["charges"], l["degs"]) for l in batched_site_legs(cfg)])
        aL, ad = ctx.double_layer(A, torch.tensor(values(cfg["seed"], "A", A.nnz), dtype=torch.float64,
                                                  device=dev))
        X = bst.Leg(-1, tuple(cfg["x"][0]), tuple(cfg["x"][1]))
        XL = ctx.layout([aL.legs[1].dual(), X, aL.legs[0].dual(), X])
        xd = torch.tensor(values(cfg["seed"], "X2", XL.nnz), dtype=torch.float64, device=dev)
        out.append((XL, xd, aL, ad))
    return out


def batch_bench(bst, ctx, dev, prec, steps, warmup, flush, pk):
    """One step = every contraction of the batch: gathers, one grouped GEMM,
    scatter, replayed from a captured CUDA graph.  Returns the report."""
    import numpy as np
    import torch
    rank, world, _ = dist_env()
    inst = batch_instances(bst, ctx, dev)
    la, lb = BATCH_LEGS
    # the contractions are independent: with several ranks each takes its
    # share (balanced by their block-pair work), no data exchange
    costs = [ctx.contract_flops(i[0], i[2], la, lb) for i in inst]
    parts = batch_partition(costs, world)
    total_count, total_flops = len(inst), sum(costs)
    inst = [inst[i] for i in parts[rank]]
    As, as_, Bs, bs = ([i[k] for i in inst] for k in range(4))
    Cls, c64 = ctx.contract_batched(As, as_, Bs, bs, la, lb, prec="fp64")
    Cls, cs = ctx.contract_batched(As, as_, Bs, bs, la, lb, prec=prec, Cls=Cls)
    torch.cuda.synchronize()
    err = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(cs, c64))
    stream = torch.cuda.current_stream()

    def timed(p, n):
        l0 = ctx.launches
        ctx.contract_batched(As, as_, Bs, bs, la, lb, prec=p, Cls=Cls, cs=cs)
        nl = ctx.launches - l0
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ctx.contract_batched(As, as_, Bs, bs, la, lb, prec=p, Cls=Cls, cs=cs)
        for _ in range(warmup):
            g.replay()
        ev = []
        for i in range(n):
            flush.fill_(float(i))
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b_.record(stream)
            ev.append((a, b_))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b_) for a, b_ in ev), nl

    ms, nl = timed(prec, steps)
    ms64, _ = timed("fp64", max(3, steps // 2))
    ms, ms64 = job_ms(ms, world), job_ms(ms64, world)   # the slowest rank's
    cheap = None
    if prec != "bf16x3":
        _, c3 = ctx.contract_batched(As, as_, Bs, bs, la, lb, prec="bf16x3", Cls=Cls)
        torch.cuda.synchronize()
        err3 = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(c3, c64))
        ms3, _ = timed("bf16x3", max(3, steps // 2))
        ms3 = job_ms(ms3, world)
        cheap = {"prec": "bf16x3", "ms_per_step": ms3, "value": total_flops / (ms3 / 1e3) / 1e12,
                 "rel_err_vs_fp64_path": err3}
        del c3
    ctx.profile(True)
    w0 = ctx.work_flops
    ctx.contract_batched(As, as_, Bs, bs, la, lb, prec=prec, Cls=Cls, cs=cs)
    flops = ctx.work_flops - w0
    local_flops = flops
    flops = total_flops
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    gk = "gemm_f64" if prec == "fp64" else "gemm_ozaki"
    # the data-movement kernel: gathers + scatter (FP64), or the pack
    # (gather and digit split in one pass; tensor-core arithmetic)
    mk = "pack_bf16" if (prec != "fp64" and "pack_bf16" in prof) else "relayout"
    out = {"workload": "u1_batch64_corner_contractions", "count": total_count,
           "value": flops / (ms / 1e3) / 1e12, "unit": "TFLOP/s (block-sparse, FP64-equivalent)",
           "contractions_per_s": total_count / (ms / 1e3), "ms_per_step": ms, "fp64_path_ms_per_step": ms64,
           "ranks": world, "per_rank_count": [len(p) for p in parts],
           "partition": "longest first to the least loaded rank by block-pair flops; no exchange",
           "algorithmic_gflop": flops / 1e9, "rel_err_vs_fp64_path": err, "gpu_launches": int(nl),
           "timing": "median of CUDA-graph replays, L2 flushed between replays",
           "kernel_ms": {k: round(v[1], 4) for k, v in prof.items()},
           "autotune": [ln.split(" ", 2)[2] for ln in ctx.tuning_log().splitlines() if "chosen" in ln],
           "cheaper_mode": cheap}
    tms = prof[gk][1] / 1e3
    if prec != "fp64":
        a = local_flops / tms / 1e12
        out["roofline"] = {"kernel": gk, "bound": "tensor", "achieved": a, "peak": pk["bf16_tflops"],
                           "unit": "TFLOP/s", "frac": a / pk["bf16_tflops"],
                           "work": "method flops (2MNK of the matched blocks, counted once)",
                           "digit_product_tflops": (15.0 if prec == "ozaki" else 6.0) * local_flops / tms / 1e12}
    else:
        peak = pk["bf16_tflops"] * 1.25 / 2250.0
        a = local_flops / tms / 1e12
        out["roofline"] = {"kernel": gk, "bound": "tensor", "achieved": a, "peak": peak, "unit": "TFLOP/s",
                           "frac": a / peak}
    if mk in prof:
        by_m, m_s = prof[mk][3], prof[mk][1] / 1e3
        out["roofline_" + mk] = {"bound": "hbm", "achieved": by_m / m_s / 1e9, "peak": pk["hbm_gbs"],
                                 "unit": "GB/s", "frac": by_m / m_s / 1e9 / pk["hbm_gbs"],
                                 "bytes": "FP64 read once + digits written" if mk == "pack_bf16"
                                 else "FP64 read + written per element"}
    del inst, cs, c64
    return out


def su2_move_bench(bst, dev, local, prec, steps, warmup, flush, pk):
    """SU(2) LEFT move of the D=10 (d=5), X=150 (chi=50) workload on seeded
    reduced blocks (env and site a[k,k,k^dual,k^dual]).  One step = the
    environment restored and one LEFT move."""
    import numpy as np
    import torch
    from workloads import su2_config, values
    cfg = su2_config("D10chi150")
    ctx = bst.Context(local)
    try:
        K, X = bst.Leg(1, *cfg["k"]), bst.Leg(1, *cfg["x"])
        Xf = lambda f: bst.Leg(f, X.charges, X.degs)
        legs = {"C1": [Xf(-1), Xf(-1)], "C2": [Xf(1), Xf(-1)], "C3": [Xf(1), Xf(1)], "C4": [Xf(1), Xf(-1)],
                "T1": [Xf(1), K.dual(), Xf(-1)], "T2": [Xf(1), K, Xf(-1)], "T3": [Xf(1), K, Xf(-1)],
                "T4": [Xf(1), K.dual(), Xf(-1)], "a": [K, K, K.dual(), K.dual()]}
        L = {r: ctx.layout(lg, group="su2") for r, lg in legs.items()}
        d = {r: torch.tensor(values(0, "A" if r == "a" else r, L[r].nnz), dtype=torch.float64, device=dev)
             for r in L}
        roles = bst.ROLES
        caps = {r: max(L[r].nnz, 50 * 150 * (42 if r.startswith("T") else 1) * 2) for r in roles}
        env = bst.Env(ctx, {r: L[r] for r in roles}, {r: d[r] for r in roles}, caps)
        pristine = {r: env.data(r).clone() for r in roles}
        L0 = dict(env.L)
        stream = torch.cuda.current_stream()

        def run(p):
            for r in roles:
                env.buf[r][:pristine[r].numel()].copy_(pristine[r])
            env.L = dict(L0)
            return ctx.ctm_move(env, L["a"], d["a"], bst.LEFT, 150, prec=p)

        run("fp64")
        ref = {r: env.data(r).cpu().numpy() for r in ("C1", "T4", "C4")}
        st = run(prec)
        torch.cuda.synchronize()
        err = max(float(np.linalg.norm(env.data(r).cpu().numpy() - ref[r]) / np.linalg.norm(ref[r])) for r in ref)

        def timed(p, n):
            for _ in range(warmup):
                run(p)
            ev = []
            for i in range(n):
                flush.fill_(float(i))
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record(stream)
                run(p)
                b_.record(stream)
                ev.append((a_, b_))
            torch.cuda.synchronize()
            return statistics.median(x.elapsed_time(y) for x, y in ev)

        ms = timed(prec, steps)
        ms64 = timed("fp64", max(3, steps // 2))
        ctx.profile(True)
        w0 = ctx.work_flops
        run(prec)
        flops = ctx.work_flops - w0
        torch.cuda.synchronize()
        prof = ctx.profile_read()
        ctx.profile(False)
        return {"workload": "su2_D10_X150_left_move", "value": 1e3 / ms, "unit": "moves/s", "ms_per_step": ms,
                "fp64_path_ms_per_step": ms64, "rel_err_vs_fp64_path": err, "kept_total_dim": st["kept"][0],
                "algorithmic_gflop": flops / 1e9, "block_sparse_tflops": flops / (ms / 1e3) / 1e12,
                "kernel_ms": {k: round(v[1], 3) for k, v in prof.items()}}
    finally:
        ctx.close()
        torch.cuda.empty_cache()


def su2_corner_bench(bst, ctx, dev, prec, steps, warmup, flush, pk):
    """SU(2) enlarged corner of the D=10 (d=5), X=150 (chi=50) workload:
    X1 = C1.T1, X2 = X1.T4, Q1 = X2.a on seeded reduced blocks.  One step =
    the three contractions."""
    import torch
    from workloads import su2_config, values
    cfg = su2_config("D10chi150")
    K = bst.Leg(1, *cfg["k"])
    X = bst.Leg(1, *cfg["x"])
    legs = {"C1": [X.dual(), X.dual()], "T1": [X, K.dual(), X.dual()], "T4": [X, K.dual(), X.dual()],
            "A": [K, K, K.dual(), K.dual()]}
    L = {n: ctx.layout(l, group="su2") for n, l in legs.items()}
    d = {n: torch.tensor(values(0, n, L[n].nnz), dtype=torch.float64, device=dev) for n in L}

    def corner(p):
        LX1, x1 = ctx.contract(L["C1"], d["C1"], L["T1"], d["T1"], (0,), (0,), prec=p)
        LX2, x2 = ctx.contract(LX1, x1, L["T4"], d["T4"], (0,), (0,), prec=p)
        return ctx.contract(LX2, x2, L["A"], d["A"], (0, 2), (1, 0), prec=p)

    _, q64 = corner("fp64")
    _, q = corner(prec)
    torch.cuda.synchronize()
    err = float(torch.linalg.norm(q - q64) / torch.linalg.norm(q64))
    stream = torch.cuda.current_stream()

    def timed(p, n):
        for _ in range(warmup):
            corner(p)
        ev = []
        for i in range(n):
            flush.fill_(float(i))
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            corner(p)
            b_.record(stream)
            ev.append((a, b_))
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b_) for a, b_ in ev)

    ms = timed(prec, steps)
    ms64 = timed("fp64", max(3, steps // 2))
    ctx.profile(True)
    w0 = ctx.work_flops
    corner(prec)
    flops = ctx.work_flops - w0
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    out = {"workload": "su2_D10_X150_enlarged_corner", "value": 1e3 / ms, "unit": "corners/s",
           "ms_per_step": ms, "fp64_path_ms_per_step": ms64, "algorithmic_gflop": flops / 1e9,
           "block_sparse_tflops": flops / (ms / 1e3) / 1e12, "rel_err_vs_fp64_path": err,
           "reduced_nnz_Q1": int(q.numel()),
           "kernel_ms": {k: round(v[1], 4) for k, v in prof.items()}}
    rc = prof.get("recouple")
    if rc:
        a = rc[3] / (rc[1] / 1e3) / 1e9
        out["roofline_recouple"] = {"bound": "hbm", "achieved": a, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                    "frac": a / pk["hbm_gbs"]}
    return out


def single_layer_bench(bst, dev, local, prec, steps, warmup, flush, pk):
    """Large U(1) single-layer LEFT move: D=8 (odd {-1:4,+1:4}, even
    {-2:2,0:4,+2:2}), chi=256 over charges -8..8, three-spin physical leg
    {-3:1,-1:3,1:3,3:1}; the double layer is never formed.  One step = the
    single-layer site (A with the remover absorbed) and one LEFT move."""
    import numpy as np
    import torch
    from paper_1808_10804_gb300.ctmrg import Network
    from workloads import u1_config, values
    cfg = u1_config("d8chi256")
    ctx = bst.Context(local)
    try:
        net = Network(ctx, {"A": cfg["A"], "R": cfg["R"]}, cfg["x"], cfg["chi"], lambda n, k: values(0, n, k),
                      device=dev, single_layer=True)
        stream = torch.cuda.current_stream()

        def run(p):
            net.reset()
            return net.step(p, direction=bst.LEFT)

        run("fp64")
        ref = {r: net.env.data(r).cpu().numpy() for r in ("C1", "T4", "C4")}
        stats = run(prec)
        torch.cuda.synchronize()
        err = max(float(np.linalg.norm(net.env.data(r).cpu().numpy() - ref[r]) / np.linalg.norm(ref[r]))
                  for r in ref)

        def timed(p, n, w):
            for _ in range(w):
                run(p)
            ev = []
            for i in range(n):
                flush.fill_(float(i))
                a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                run(p)
                b_.record(stream)
                ev.append((a, b_))
            torch.cuda.synchronize()
            return statistics.median(a.elapsed_time(b_) for a, b_ in ev)

        ms = timed(prec, max(3, steps // 3), max(1, warmup // 3))
        ms64 = timed("fp64", 1, 0)
        ctx.profile(True)
        w0 = ctx.work_flops
        run(prec)
        flops = ctx.work_flops - w0
        torch.cuda.synchronize()
        prof = ctx.profile_read()
        ctx.profile(False)
        gk = "gemm_f64" if prec == "fp64" else "gemm_ozaki"
        out = {"workload": "u1_D8_chi256_single_layer_left_move", "value": 1e3 / ms, "unit": "moves/s",
               "ms_per_step": ms, "fp64_path_ms_per_step": ms64, "rel_err_vs_fp64_path": err,
               "kept": stats["kept"][0], "algorithmic_gflop": flops / 1e9,
               "block_sparse_tflops": flops / (ms / 1e3) / 1e12,
               "kernel_ms": {k: round(v[1], 3) for k, v in prof.items()}}
        g = prof.get(gk)
        if g:
            a = flops / (g[1] / 1e3) / 1e12
            peak = pk["bf16_tflops"] if prec == "ozaki" else pk["bf16_tflops"] * 1.25 / 2250.0
            out["roofline"] = {"kernel": gk, "bound": "tensor", "achieved": a, "peak": peak, "unit": "TFLOP/s",
                               "frac": a / peak, "work": "method flops counted once"}
        del net
        return out
    finally:
        ctx.close()
        torch.cuda.empty_cache()


def run_profile_target(args):
    """--quick with --only: warm-up and steps of one workload, nothing else
    (a small, fixed command for profilers)."""
    import torch
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    from paper_1808_10804_gb300 import build as b
    b.build()
    from paper_1808_10804_gb300 import bst
    from workloads import su2_config, u1_config, values
    ctx = bst.Context(local)
    try:
        if args.only == "batch":
            inst = batch_instances(bst, ctx, dev)
            la, lb = BATCH_LEGS
            As, as_, Bs, bs = ([i[k] for i in inst] for k in range(4))
            Cls, cs = ctx.contract_batched(As, as_, Bs, bs, la, lb, prec=args.prec)
            for _ in range(args.warmup + args.steps):
                ctx.contract_batched(As, as_, Bs, bs, la, lb, prec=args.prec, Cls=Cls, cs=cs)
        elif args.only == "su2":
            cfg = su2_config("D10chi150")
            K, X = bst.Leg(1, *cfg["k"]), bst.Leg(1, *cfg["x"])
            legs = {"C1": [X.dual(), X.dual()], "T1": [X, K.dual(), X.dual()], "T4": [X, K.dual(), X.dual()],
                    "A": [K, K, K.dual(), K.dual()]}
            L = {n: ctx.layout(l, group="su2") for n, l in legs.items()}
            d = {n: torch.tensor(values(0, n, L[n].nnz), dtype=torch.float64, device=dev) for n in L}
            for _ in range(args.warmup + args.steps):
                LX1, x1 = ctx.contract(L["C1"], d["C1"], L["T1"], d["T1"], (0,), (0,), prec=args.prec)
                LX2, x2 = ctx.contract(LX1, x1, L["T4"], d["T4"], (0,), (0,), prec=args.prec)
                ctx.contract(LX2, x2, L["A"], d["A"], (0, 2), (1, 0), prec=args.prec)
        elif args.only == "large":
            from paper_1808_10804_gb300.ctmrg import Network
            cfg = u1_config("d8chi256")
            net = Network(ctx, {"A": cfg["A"], "R": cfg["R"]}, cfg["x"], cfg["chi"], lambda n, k: values(0, n, k),
                          device=dev, single_layer=True)
            for _ in range(args.warmup + args.steps):
                net.reset()
                net.step(args.prec, direction=bst.LEFT)
        torch.cuda.synchronize()
    finally:
        ctx.close()


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    from paper_1808_10804_gb300 import build as b
    b.build()
    from paper_1808_10804_gb300 import bst
    from paper_1808_10804_gb300.ctmrg import Network
    from workloads import u1_config, values

    cfg = u1_config(WORKLOAD)
    ctx = bst.Context(local)
    draw = lambda name, n: values(0, name, n)
    net = Network(ctx, {"A": cfg["A"], "R": cfg["R"]}, cfg["x"], cfg["chi"], draw, device=dev)
    prec = args.prec
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_step(p=prec):
        net.reset()
        return net.step(p)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if args.quick:
        # profiling mode: warm-up and the timed steps only
        for _ in range(args.steps):
            one_step()
        torch.cuda.synchronize()
        ctx.close()
        return
    # reference result of the FP64 path for the accuracy report
    one_step("fp64")
    ref64 = {r: net.env.data(r).cpu().numpy() for r in bst.ROLES}
    refL = {r: net.env.L[r] for r in bst.ROLES}
    one_step(prec)
    torch.cuda.synchronize()
    err_by = {}
    for r in bst.ROLES:
        if net.env.L[r] == refL[r]:
            x = net.env.data(r).cpu().numpy()
            err_by[r] = float(np.linalg.norm(x - ref64[r]) / np.linalg.norm(ref64[r]))
        else:
            err_by[r] = float("inf")
    err = max(err_by.values())

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    l0 = ctx.launches
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))          # L2 flush between steps (outside the events)
            ev[i][0].record(stream)
            one_step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        wall = time.perf_counter() - t0
    launches = (ctx.launches - l0) // args.steps
    ms = [a.elapsed_time(b_) for a, b_ in ev]
    ms_step = statistics.mean(ms)
    ms_step = job_ms(ms_step, world)

    # per-kernel-class profile of one extra step (events around every launch);
    # the method's work of the step from the plan-enumerated counter
    ctx.profile(True)
    w0 = ctx.work_flops
    one_step()
    algo_flops = ctx.work_flops - w0
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)

    # end to end through the public API: inputs from pinned host memory,
    # renewed environment read back every step
    e2e_ms, h2d, d2h = [], 0, 0
    for i in range(max(3, args.steps // 2)):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        h2d = net.reset_from_host()
        net.step(prec)
        outs = [net.env.data(r).cpu() for r in bst.ROLES]
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t1))
        d2h = sum(8 * o.numel() for o in outs)

    # plain FP64 GPU path, same steps, for the comparison the metric names
    fp64_ms = None
    if prec != "fp64":
        ev2 = []
        for i in range(max(3, args.steps // 2)):
            flush.fill_(float(i))
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            one_step("fp64")
            b_.record(stream)
            ev2.append((a, b_))
        torch.cuda.synchronize()
        fp64_ms = statistics.mean(a.elapsed_time(b_) for a, b_ in ev2)

    # the cheaper arithmetic (three BF16 slices in the block contractions,
    # the projector in the five-slice one): speed and error of the same step
    cheap = None
    if prec != "bf16x3":
        one_step("bf16x3")
        torch.cuda.synchronize()
        errc = {}
        for r in bst.ROLES:
            if net.env.L[r] == refL[r]:
                x = net.env.data(r).cpu().numpy()
                errc[r] = float(np.linalg.norm(x - ref64[r]) / np.linalg.norm(ref64[r]))
            else:
                errc[r] = float("inf")
        ev3 = []
        for i in range(max(3, args.steps // 2)):
            flush.fill_(float(i))
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            one_step("bf16x3")
            b_.record(stream)
            ev3.append((a, b_))
        torch.cuda.synchronize()
        cms = statistics.mean(a.elapsed_time(b_) for a, b_ in ev3)
        cheap = {"workload": "u1_D6_chi72_full_move", "prec": "bf16x3", "value": 1e3 / cms, "unit": "moves/s",
                 "ms_per_step": cms, "fp64_path_ms_per_step": fp64_ms, "rel_err_vs_fp64_path": max(errc.values()),
                 "rel_err_vs_fp64_path_by_tensor": {r: float(f"{e:.3e}") for r, e in errc.items()},
                 "note": "block contractions in three BF16 slices (6 products); projector in five"}

    pk = peaks()
    batched = su2 = su2m = large = None
    if not args.no_batch:
        batched = batch_bench(bst, ctx, dev, prec, args.steps, args.warmup, flush, pk)
        su2 = su2_corner_bench(bst, ctx, dev, prec, args.steps, args.warmup, flush, pk)
        su2m = su2_move_bench(bst, dev, local, prec, args.steps, args.warmup, flush, pk)
        large = single_layer_bench(bst, dev, local, prec, args.steps, args.warmup, flush, pk)

    if rank != 0:
        return
    # FP32 SIMT peak from the unit counts: 152 SMs x 128 FP32 lanes x 2 flops
    # (FMA) x the observed maximum SM clock
    clk_max = (clk.summary().get("sm_max_mhz") or 2070.0) * 1e6
    fp32_peak = 152 * 128 * 2 * clk_max / 1e12
    def roof_of(name, v):
        n, tms, fl, by = v
        sec = tms / 1e3
        if name == "gemm_ozaki":
            # the method's flops of the step (counted once, FP64-equivalent)
            # over the time of every launch of the class (projector
            # iterations included) against the BF16 tensor peak; the rate of
            # BF16 digit products the class performs is reported beside it
            a = algo_flops / sec / 1e12
            return {"kernel": name, "bound": "tensor", "achieved": a, "peak": pk["bf16_tflops"],
                    "unit": "TFLOP/s", "frac": a / pk["bf16_tflops"],
                    "work": "method flops of the step, counted once",
                    "digit_product_tflops": (15.0 if prec == "ozaki" else 6.0) * fl / sec / 1e12}
        if name == "gemm_f64":
            peak = pk["bf16_tflops"] * 1.25 / 2250.0   # FP64 tensor peak from the nominal ratio
            if prec == "fp64":
                a, work = algo_flops / sec / 1e12, "method flops of the step, counted once"
            else:
                # the mixed path runs only the projector's small FP64
                # products here: their own flops
                a, work = fl / sec / 1e12, "flops of the FP64 products of the class"
            return {"kernel": name, "bound": "tensor", "achieved": a, "peak": peak, "unit": "TFLOP/s",
                    "frac": a / peak, "work": work}
        if name in ("cholinv_f32", "jacobi_f32", "gram_f32"):
            a = fl / sec / 1e12
            return {"kernel": name, "bound": "alu", "achieved": a, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": a / fp32_peak}
        a = by / sec / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": a, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": a / pk["hbm_gbs"]}
    kernels = {k: v for k, v in prof.items() if k not in ("svd_cusolver", "proj_subspace")}
    dom_name, dom = max(kernels.items(), key=lambda kv: kv[1][1])
    roof = roof_of(dom_name, dom)
    roof.update({"traffic": ncu_traffic(dom_name), "launches_per_step": dom[0], "peak_source": pk["source"]})
    if roof["bound"] == "alu":
        roof["note"] = ("one CTA per sector problem (about a dozen of 152 SMs busy): latency bound; "
                        "peak = 152 SMs x 128 FP32 lanes x 2 x clock")
    roof_all = {k: {kk: (round(vv, 5) if isinstance(vv, float) else vv) for kk, vv in roof_of(k, v).items()
                    if kk in ("bound", "achieved", "frac", "unit")} | {"ms_per_step": round(v[1], 3)}
                for k, v in kernels.items()}
    cpu = None
    if world == 1 and not args.no_cpu:
        times, cores = cpu_oracle_time(1, 0)
        cpu = {"value": 1.0 / times[0], "unit": "moves/s", "cores": cores, "kind": "oracle",
               "sample": "one full move (double layer + L,R,U,D) of the same workload, dense numpy FP64"}
    v = job_value(ms_step, world)
    # the sub-workloads first, one JSON line each on stderr; the headline
    # line (stdout) stays short and carries their key numbers
    subs = {"cheaper_mode": cheap, "batched": batched, "su2_corner": su2, "su2_left_move": su2m,
            "single_layer_large": large}
    for name, rep in subs.items():
        if rep:
            print(json.dumps({"sub_workload": name, **rep}), file=sys.stderr, flush=True)
    def short(k, v):
        if not isinstance(v, float):
            return v
        return float(f"{v:.3e}") if k == "rel_err_vs_fp64_path" else round(v, 6)
    brief = {name: {k: short(k, rep.get(k))
                    for k in ("value", "unit", "ms_per_step", "fp64_path_ms_per_step", "rel_err_vs_fp64_path")}
             for name, rep in subs.items() if rep}
    line = {
        "metric": METRIC, "value": v, "unit": "moves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "ozaki": "bf16x5-slices->f64", "bf16x3": "bf16x3-slices->f64"}[prec],
        "data": "synthetic",
        "config": {"workload": "u1_D6_chi72_full_move", "D": 6, "chi": 72, "prec": prec,
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas{world}"},
        "fp64_path_ms_per_step": fp64_ms,
        "fp64_path_moves_per_s": (1e3 / fp64_ms) if fp64_ms else None,
        "rel_err_vs_fp64_path": err,
        "rel_err_vs_fp64_path_by_tensor": {r: float(f"{e:.3e}") for r, e in err_by.items()},
        "algorithmic_gflop_per_step": algo_flops / 1e9,
        "block_sparse_tflops": algo_flops / (ms_step / 1e3) / 1e12,
        "e2e": {"value": 1e3 / statistics.mean(e2e_ms), "unit": "moves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "roofline": roof,
        "wall_ms_per_step": 1e3 * wall / args.steps,
        "kernel_ms_per_step": {k: round(v_[1], 3) for k, v_ in prof.items()},
        "roofline_by_kernel": roof_all,
        "sub_workloads": brief,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="ozaki", choices=["fp64", "ozaki", "bf16x3"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-contraction report")
    ap.add_argument("--quick", action="store_true", help="warm-up and steps only, no report (for profilers)")
    ap.add_argument("--only", default="ctm", choices=["ctm", "batch", "su2", "large"],
                    help="with --quick: the workload to run (CTMRG move, batched contractions, SU(2) corner, "
                         "large single-layer move)")
    args = ap.parse_args()
    if args.quick and args.only != "ctm":
        run_profile_target(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
