#!/usr/bin/env python
"""Benchmark of the GB300 tile-recursive PLUQ over GF(p).

Workload: one 32768 x 32768 matrix over GF(65521) with entries i.i.d. uniform
in [0, p) (full rank with high probability; the shape of the paper's dense
experiments, Sec. 3 and Table 3, at the largest size one GPU holds), factored
by pluq_modp (P, L, U, Q, rank, both rank profiles).  One step = restore the
input in HBM + one full factorization.  Metric: effective Gfops =
F(m, n, r) / t with F = 2mnr - (m+n)r^2 + 2r^3/3 field operations.  The
8192 x 8192 rank-4096 matrix over GF(131071) with random rank profiles (A = L R
U, the S16K-like shape of Sec. 4.1) is timed as a second workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain row-by-row elimination in int64,
test infrastructure) on the host cores, on a bounded sample of the workload.
Several GPUs run independent replicas (the single-matrix path does not
shard); value is the work of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOAD = "uniform-32768-p65521"
SECOND_WORKLOAD = "lru-8192-r4096-p131071"
METRIC = "PLUQ mod p effective Gfops (2n³/3/s), tensor-limb vs FP64 form, bit-exact"

# DRAM traffic (read + write bytes) per launch of a kernel class on a workload,
# from the committed ncu captures (profiles/); absent where no capture of the
# current kernel exists.
NCU_TRAFFIC_PER_LAUNCH: dict[tuple[str, str], float] = {
    # k_fgemm_limb<2, 1>, mean of the 833 launches of one 32768^2 factorization
    # (profiles/launch_list_uniform32768_p65521.md, second capture)
    ("uniform-32768-p65521", "fgemm"): 108.6e6,
}


def class_rooflines(classes: dict, peaks: dict) -> dict:
    """Per kernel class of the profiled pass: launches, device ms, achieved HBM
    bandwidth from its algorithmic bytes (and its fraction of the measured copy
    bandwidth), and for the fgemm class its tensor rate and fraction of the
    measured sustained bf16 peak (the fp16 dense rate equals the bf16 rate)."""
    out = {}
    for k, v in classes.items():
        e = {"launches": v["launches"], "ms": round(v["ms"], 3)}
        if v["ms"] > 0 and v["bytes"] > 0:
            gbs = v["bytes"] / (v["ms"] / 1e3) / 1e9
            e["hbm_gbs"] = round(gbs, 1)
            e["hbm_frac"] = round(gbs / peaks["hbm_gbs"], 4)
        if v["ms"] > 0 and v.get("tensor_flops", 0) > 0:
            tf = v["tensor_flops"] / (v["ms"] / 1e3) / 1e12
            e["tensor_tflops"] = round(tf, 1)
            e["tensor_frac"] = round(tf / peaks["bf16_sustained"], 4)
        out[k] = e
    return out


def clock_log_path(rank: int) -> str:
    """Where the raw nvidia-smi samples of the timed region go (their summary is in
    the JSON line): BENCH_CLOCK_DIR if set, else the system's temporary directory."""
    import tempfile
    return os.path.join(os.environ.get("BENCH_CLOCK_DIR", tempfile.gettempdir()),
                        f"bench_clocks_{rank}.csv")


def golden_rpm(key: str, seed: int = 1):
    """The oracle's rank profile matrix of a uniform workload, as stored under
    tests/golden/ by its writer script (None when no such file exists)."""
    path = os.path.join(ROOT, "tests", "golden", f"oracle_rpm_{key}_seed{seed}.npz")
    if not os.path.exists(path):
        return None
    d = np.load(path)
    return {"rank": int(d["rank"][0]), "rpm": set(zip(d["piv_rows"].tolist(),
                                                      d["piv_cols"].tolist())),
            "rrp": d["rrp"].tolist(), "crp": d["crp"].tolist()}


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the platform's description."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def field_ops(m: int, n: int, r: int) -> float:
    return 2.0 * m * n * r - (m + n) * r * r + 2.0 * r ** 3 / 3.0


def read_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "bf16": d.get("bf16_tflops", 1900.0),
                "bf16_sustained": d.get("bf16_tflops_sustained", 1700.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index: int, path: str):
        self.path = path
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if parts[5 + k].lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (the slowest rank's time); x itself without dist."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gfops(world: int, work_per_rank: float, ms_slowest: float) -> float:
    """Independent replicas: the work of all ranks over the slowest rank's time."""
    return world * work_per_rank / (ms_slowest / 1e3) / 1e9


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_sample(cfg, budget_s: float, cores: int):
    """A matrix of the workload's construction sized for about budget_s of oracle time.

    Returns (A, m, n, expected rank or None, description); the full workload when it
    fits the budget.  The oracle's rate is calibrated on a 1024 x 1024 matrix.
    """
    import oracle
    r_full = cfg.r if cfg.r is not None else min(cfg.m, cfg.n)
    cal = workloads.prescribed_rank_matrix(1024, 1024, 512, cfg.p, seed=1)
    t = time.time()
    oracle.pluq(cal.A, cfg.p, threads=cores)
    rate = field_ops(1024, 1024, 512) / max(time.time() - t, 1e-3)
    f = min(1.0, (budget_s * rate / field_ops(cfg.m, cfg.n, r_full)) ** (1 / 3))
    m = cfg.m if f >= 1.0 else max(256, int(cfg.m * f) // 256 * 256)
    n = cfg.n if f >= 1.0 else max(256, int(cfg.n * f) // 256 * 256)
    full = m == cfg.m and n == cfg.n
    if cfg.kind == "uniform":
        A, r = workloads.uniform_matrix(m, n, cfg.p, seed=1), None
        what = f"{m}x{n} uniform matrix (p={cfg.p}, seed 1)"
    else:
        r = r_full if full else max(1, r_full * m // cfg.m)
        A = workloads.prescribed_rank_matrix(m, n, r, cfg.p, seed=1).A
        what = f"{m}x{n} rank {r} matrix of the same construction (p={cfg.p}, seed 1)"
    if full:
        return A, m, n, r, f"the full {cfg.m}x{cfg.n} workload matrix"
    return A, m, n, r, f"{what}; the {cfg.m}x{cfg.n} workload scaled by size to fit the run"


def bench_reference(args, world, rank):
    """Time the CPU oracle on the host cores on a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    cfg = workloads.CONFIGS[args.workload]
    if cfg.kind == "batched":
        cfg = workloads.Config(cfg.key, "lru", cfg.hi, cfg.hi, cfg.p, r=cfg.hi // 2)
    cores = os.cpu_count() or 1
    # a sample size that keeps the whole run near 2 minutes
    budget = 110.0 / max(1, args.steps + args.warmup)
    A, m, n, r, sample = oracle_sample(cfg, budget, cores)
    for _ in range(args.warmup):
        oracle.pluq(A, cfg.p, threads=cores)
    times = []
    for _ in range(args.steps):
        t = time.time()
        res = oracle.pluq(A, cfg.p, threads=cores)
        times.append(time.time() - t)
    assert r is None or res.rank == r
    r = res.rank
    ms = 1e3 * float(np.mean(times))
    value = field_ops(m, n, r) / (ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Gfops", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": args.workload, "m": cfg.m, "n": cfg.n, "rank": cfg.r, "p": cfg.p},
        "cpu_baseline": {"value": round(value, 3), "unit": "Gfops", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "Gfops", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def time_steps(pq, ctx, A, A0, p, form, steps, stream):
    import torch
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(steps):
        A.copy_(A0)
        pq.pluq_modp(A, p, form=form, ctx=ctx, profiles=True)
    stop.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(stop) / steps


def batch_shard(cfg, rank: int):
    """Shard `rank` of the batched workload across GPUs: its own batch of cfg.count
    matrices of the workload's distribution (shard 0 is the workload itself), so the
    global batch grows with the number of ranks and no data crosses between them.

    Returns (tag, m, n, r): the generator tag of the shard's matrices and their shapes.
    """
    tag = "batched" if rank == 0 else f"batched-shard{rank}"
    ms, ns, rs = workloads.batched_shapes(cfg.count, cfg.lo, cfg.hi, seed=1, tag=tag)
    return tag, ms, ns, rs


def bench_batched(args, world, rank, local):
    """Many small rank-deficient matrices in one persistent graph-captured launch;
    several GPUs each factor their own shard of the global batch (weak scaling)."""
    import torch
    import paper_1402_3501_gb300 as pq

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cfg = workloads.CONFIGS[args.workload]
    p = cfg.p
    tag, ms, ns, rs = batch_shard(cfg, rank)
    gens = [workloads.prescribed_rank_matrix(int(ms[b]), int(ns[b]), int(rs[b]), p, seed=1,
                                             tag=f"{tag}:{b}", device="cuda")
            for b in range(cfg.count)]
    sizes = [int(g.A.size) for g in gens]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    flat = np.concatenate([g.A.ravel() for g in gens]).astype(np.int32)
    A0 = torch.from_numpy(flat).cuda()
    A = torch.empty_like(A0)
    views = [A[offs[b]:offs[b + 1]].view(int(ms[b]), int(ns[b])) for b in range(cfg.count)]
    F = sum(field_ops(int(ms[b]), int(ns[b]), int(rs[b])) for b in range(cfg.count))
    ctx = pq.Context(local)
    plan = pq.BatchPlan(views, p, ctx=ctx)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        A.copy_(A0)
        st = plan.run()
    torch.cuda.synchronize()
    exact = st == 0 and all(plan.ranks[b] == gens[b].rank for b in range(cfg.count))
    for b in range(0, cfg.count, 97):  # spot-check rank profile matrices
        r = plan.ranks[b]
        P = plan.Ps[b][:ms[b]].cpu().numpy()
        Q = plan.Qs[b][:ns[b]].cpu().numpy()
        exact = exact and set(zip(P[:r].tolist(), Q[:r].tolist())) == gens[b].rpm
    ctx.profile(False)
    sampler = ClockSampler(local, clock_log_path(rank))
    ms_step = time_batched(plan, A, A0, args.steps, stream)
    clocks = sampler.stop()
    launches = sum(c["launches"] for c in ctx.profile_read().values())
    ms_step = max_over_ranks(ms_step, dist, "cuda")
    # per-matrix launches on a sample of the same matrices
    sample = list(range(0, cfg.count, 32))
    A.copy_(A0)
    torch.cuda.synchronize()
    t0 = time.time()
    for b in sample:
        pq.pluq_modp(views[b], p, ctx=ctx)
    torch.cuda.synchronize()
    per_ms = (time.time() - t0) * 1e3 / len(sample)
    F_sample = sum(field_ops(int(ms[b]), int(ns[b]), int(rs[b])) for b in sample)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(whole_job_gfops(world, F, ms_step), 3), "unit": "Gfops",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_step, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "count": cfg.count, "m_n_range": [cfg.lo, cfg.hi],
                       "p": p, "step": "restore inputs (D2D copy) + pluq_modp_batched",
                       "parallelism": f"batch sharded x{world} ({cfg.count} matrices a rank)"},
            "bitexact": bool(exact),
            "matrices_per_s": round(world * cfg.count / (ms_step / 1e3), 1),
            "per_matrix_launches": {"ms_per_matrix": round(per_ms, 4),
                                    "matrices_per_s": round(1e3 / per_ms, 1),
                                    "value": round(F_sample / len(sample) * 1e3 / per_ms / 1e9, 3),
                                    "sample": f"every 32nd matrix ({len(sample)})"},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def time_batched(plan, A, A0, steps, stream):
    import torch
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(steps):
        A.copy_(A0)
        plan.run()
    stop.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(stop) / steps


def bench_ours(args, world, rank, local):
    import torch
    import paper_1402_3501_gb300 as pq

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cfg = workloads.CONFIGS[args.workload]
    m, n, p = cfg.m, cfg.n, cfg.p
    if cfg.kind == "uniform":
        # full rank with high probability; checked against the oracle's rank
        # profile matrix where one is stored (tests/golden/)
        g = None
        A_host = workloads.uniform_matrix(m, n, p, seed=1)
    else:
        g = workloads.prescribed_rank_matrix(m, n, cfg.r, p, seed=1, device="cuda")
        A_host = g.A
    A0 = torch.from_numpy(A_host.astype(np.int32)).cuda()
    A = torch.empty_like(A0)
    ctx = pq.Context(local)
    stream = torch.cuda.current_stream()
    form = args.form

    # schedule chosen by the library's autotuner on this matrix (untimed), then
    # warm-up (not timed) and bit-exact validation against the construction
    schedule = None
    if args.winograd_min:
        ctx.set_option("winograd_min", args.winograd_min)
    ctx.set_option("fgemm_tile", args.fgemm_tile)
    ctx.set_option("fused_kmax", args.fused_kmax)
    ctx.set_option("thin_gemm", 0 if args.no_thin else 1)
    if args.decomposition == "iterative":
        ctx.set_option("decomposition", 1)
        ctx.set_option("slab_rows", args.slab_rows)
    if args.schedule:
        leaf, kind, fork = (int(x) for x in args.schedule.split(","))
        ctx.set_option("leaf_dim", leaf)
        ctx.set_option("leaf_kind", kind)
        ctx.set_option("fork_depth", fork)
        schedule = {"leaf_dim": leaf, "leaf_kind": ctx.LEAF_KINDS[kind], "fork_depth": fork,
                    "fgemm_tile": args.fgemm_tile, "set": "by --schedule"}
    elif not args.no_autotune:
        schedule = ctx.autotune(A0, p, form=form, budget_ms=args.tune_budget_ms)
    for _ in range(args.warmup):
        A.copy_(A0)
        res = pq.pluq_modp(A, p, form=form, ctx=ctx)
    torch.cuda.synchronize()
    r = res.rank
    exact = None
    want = ({"rank": g.rank, "rpm": g.rpm, "rrp": g.rrp.tolist(), "crp": g.crp.tolist()}
            if g is not None else golden_rpm(args.workload))
    if want is not None:
        P = res.P.cpu().numpy()
        Q = res.Q.cpu().numpy()
        exact = (r == want["rank"] and set(zip(P[:r].tolist(), Q[:r].tolist())) == want["rpm"]
                 and res.rrp.cpu().tolist() == want["rrp"]
                 and res.crp.cpu().tolist() == want["crp"])

    # timed region: CUDA events on the launching stream around K steps; the
    # library counts its own kernel launches
    ctx.profile(False)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local, clock_log_path(rank))
    wall0 = time.time()
    ms = time_steps(pq, ctx, A, A0, p, form, args.steps, stream)
    wall = time.time() - wall0
    clocks = sampler.stop()
    launches = sum(c["launches"] for c in ctx.profile_read().values())
    # the same K steps again with a CUDA-event pair around every launch
    # (per-class device time for the roofline; this pass is not the headline)
    ctx.profile(True)
    ms_profiled = time_steps(pq, ctx, A, A0, p, form, args.steps, stream)
    classes = ctx.profile_read()
    ctx.profile(False)
    ms = max_over_ranks(ms, dist, "cuda")
    if dist:
        dist.barrier()
    F = field_ops(m, n, r)
    value = whole_job_gfops(world, F, ms)

    # FP64-embedding form on the same input (the paper's representation)
    fp64 = None
    if not args.no_fp64:
        A.copy_(A0)
        pq.pluq_modp(A, p, form="fp64", ctx=ctx)
        ms64 = time_steps(pq, ctx, A, A0, p, "fp64", max(1, min(args.steps, args.fp64_steps)),
                          stream)
        ms64 = max_over_ranks(ms64, dist, "cuda")
        fp64 = {"value": round(whole_job_gfops(world, F, ms64), 3), "ms_per_step": round(ms64, 3)}

    # end to end through the public API: pinned host input -> device -> PLUQ ->
    # L\U, P, Q back to pinned host memory
    Ah = torch.from_numpy(A_host.astype(np.int32)).pin_memory()
    LUh = torch.empty_like(Ah).pin_memory()
    Ph = torch.empty(m, dtype=torch.int32).pin_memory()
    Qh = torch.empty(n, dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        Ad = Ah.to("cuda", non_blocking=True)
        res = pq.pluq_modp(Ad, p, form=form, ctx=ctx)
        LUh.copy_(res.LU, non_blocking=True)
        Ph.copy_(res.P, non_blocking=True)
        Qh.copy_(res.Q, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")

    # roofline of the dominant kernel class
    peaks = read_peaks()
    dom = max(classes, key=lambda k: classes[k]["ms"])
    c = classes[dom]
    timed = c["launches"] if dom not in ("perm", "pack") else c["launches"] / 2
    avg_ms = c["ms"] / max(1, timed)
    if dom == "fgemm":
        # algorithmic work = the field operations 2MNK of the Schur updates; the
        # limb form issues L^2 digit products for each (L = 2 below p ~ 2^18)
        achieved = c["flops"] / (c["ms"] / 1e3) / 1e12
        issued = c["tensor_flops"] / (c["ms"] / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": round(achieved, 2),
                "peak": peaks["bf16_sustained"], "unit": "TFLOP/s",
                "peak_note": f"fp16 dense = bf16 rate; {peaks['source']} sustained bf16",
                "achieved_issued": round(issued, 2),
                "frac_issued": round(issued / peaks["bf16_sustained"], 4),
                "issued_note": "tensor flops actually issued (digit products, tile padding)"}
    else:
        achieved = c["bytes"] / (c["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "peak_note": f"{peaks['source']} HBM copy bandwidth"}
    roof["frac"] = round(roof["achieved"] / roof["peak"], 4)
    roof["kernel_class"] = dom
    roof["traffic"] = NCU_TRAFFIC_PER_LAUNCH.get((args.workload, dom))
    roof["avg_launch_ms"] = round(avg_ms, 4)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        cores = os.cpu_count() or 1
        As, ms_, ns_, rs_, sample = oracle_sample(cfg, 20.0, cores)
        t = time.time()
        ref = oracle.pluq(As, p, threads=cores)
        dt = time.time() - t
        assert rs_ is None or ref.rank == rs_
        cpu = {"value": round(field_ops(ms_, ns_, ref.rank) / dt / 1e9, 3), "unit": "Gfops",
               "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
               "sample": f"{sample}, one run ({dt:.1f} s)"}

    # the second workload (rank deficient, random rank profiles), same context
    second = None
    if not args.no_second and args.workload == WORKLOAD:
        second = bench_second(pq, ctx, args, stream)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "Gfops", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "m": m, "n": n, "rank": r, "p": p, "form": form,
                       "l2": f"inputs ({m * n * 4 / 1e6:.0f} MB) larger than L2 (129 MB), no flush",
                       "step": "restore input (D2D copy) + pluq_modp",
                       "schedule": schedule or "default (leaf 1024, per-leaf kind, fork depth 2)",
                       "winograd_min": args.winograd_min,
                       "decomposition": ("tile recursive" if args.decomposition == "recursive"
                                         else f"tiled iterative (slab rows "
                                              f"{args.slab_rows or 'leaf cut-off'})"),
                       "parallelism": f"replicas x{world}"},
            "bitexact": exact,
            "fgemm_dtype": "f16 digits, f32 accumulate" if form != "fp64" else "f64",
            "fp64_form": fp64,
            "e2e": {"value": round(whole_job_gfops(world, F, e2e_ms), 3), "unit": "Gfops",
                    "ms_per_step": round(e2e_ms, 3), "h2d_bytes_per_step": int(m * n * 4),
                    "d2h_bytes_per_step": int(m * n * 4 + 4 * (m + n))},
            "gpu_launches": int(launches),
            "roofline": roof,
            "kernel_classes": class_rooflines(classes, peaks),
            "profiled_pass_ms_per_step": round(ms_profiled, 3),
            "clocks": clocks,
            "wall_s_timed": round(wall, 3),
            "cpu_baseline": cpu,
            "second_workload": second,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def bench_second(pq, ctx, args, stream) -> dict:
    """The 8192 x 8192 rank-4096 workload on the same context: autotuned schedule,
    warm-up, then timed steps, checked against its construction."""
    import torch
    cfg = workloads.CONFIGS[SECOND_WORKLOAD]
    g = workloads.prescribed_rank_matrix(cfg.m, cfg.n, cfg.r, cfg.p, seed=1, device="cuda")
    A0 = torch.from_numpy(g.A.astype(np.int32)).cuda()
    A = torch.empty_like(A0)
    sched = ctx.autotune(A0, cfg.p, form=args.form, budget_ms=min(args.tune_budget_ms, 8000.0))
    for _ in range(3):
        A.copy_(A0)
        res = pq.pluq_modp(A, cfg.p, form=args.form, ctx=ctx)
    torch.cuda.synchronize()
    r = res.rank
    P, Q = res.P.cpu().numpy(), res.Q.cpu().numpy()
    exact = (r == g.rank and set(zip(P[:r].tolist(), Q[:r].tolist())) == g.rpm
             and res.rrp.cpu().tolist() == g.rrp.tolist()
             and res.crp.cpu().tolist() == g.crp.tolist())
    ms = time_steps(pq, ctx, A, A0, cfg.p, args.form, 10, stream)
    return {"workload": SECOND_WORKLOAD, "value": round(field_ops(cfg.m, cfg.n, r) / ms / 1e6, 3),
            "unit": "Gfops", "ms_per_step": round(ms, 3), "steps": 10, "bitexact": bool(exact),
            "schedule": sched}


def profile_fgemm(args):
    """One kernel-level case for ncu captures: C (M x N) -= A (M x K) B (K x N) mod p
    through fgemm_modp, `--repeat` times on seeded uniform residues; prints one line
    (not a bench line: nothing is checked here, the parity tests do that)."""
    import torch
    import paper_1402_3501_gb300 as pq
    M, N, K = (int(x) for x in args.fgemm.lower().split("x"))
    p = args.p
    dev = lambda X: torch.from_numpy(X.astype(np.int32)).cuda()  # noqa: E731
    A = dev(workloads.uniform_matrix(M, K, p, 1, "casea"))
    B = dev(workloads.uniform_matrix(K, N, p, 1, "caseb"))
    C = dev(workloads.uniform_matrix(M, N, p, 1, "casec"))
    ctx = pq.Context(0)
    ctx.set_option("winograd_min", args.winograd_min)
    ctx.set_option("fgemm_tile", args.fgemm_tile)
    ctx.set_option("fused_kmax", args.fused_kmax)
    ctx.set_option("thin_gemm", 0 if args.no_thin else 1)
    form = "fp64" if args.form == "fp64" else "limb"
    ms = []
    for _ in range(max(1, args.repeat)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        pq.fgemm_modp(C, A, B, p, form=form, ctx=ctx)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(f"fgemm {M}x{N}x{K} p={p} {form} tile={args.fgemm_tile} fused_kmax={args.fused_kmax} "
          f"thin={0 if args.no_thin else 1} winograd_min={args.winograd_min}: "
          f"last {ms[-1]:.3f} ms "
          f"({2.0 * M * N * K / ms[-1] / 1e9:.1f} field Tops/s)", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--form", choices=["limb", "fp64", "auto"], default="limb")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="timed steps of the FP64-embedding form (after one untimed)")
    ap.add_argument("--no-second", action="store_true",
                    help="skip the second (8192^2 rank-4096) workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the default schedule instead of the autotuned one")
    ap.add_argument("--tune-budget-ms", type=float, default=25000.0)
    ap.add_argument("--schedule", default="",
                    help="leaf_dim,leaf_kind,fork_depth to time instead of autotuning "
                         "(leaf kind 0 barrier, 1 wavefront, 2 per leaf, 3 cluster)")
    ap.add_argument("--decomposition", choices=["recursive", "iterative"], default="recursive",
                    help="tile recursive (default) or tiled iterative (row slabs by column "
                         "tiles), the paper's two rank-deficient eliminations")
    ap.add_argument("--slab-rows", type=int, default=0,
                    help="rows of a tiled-iterative slab (0: the leaf cut-off)")
    ap.add_argument("--workload", default=WORKLOAD, choices=list(workloads.CONFIGS),
                    help="matrix to factor (the default is the measured workload; the "
                         "others serve as small profiling cases)")
    ap.add_argument("--winograd-min", type=int, default=0,
                    help="Strassen-Winograd levels on Schur updates with M, N, K all at least "
                         "this (0: classical products only)")
    ap.add_argument("--fgemm", default="",
                    help="MxNxK: profiling case of one fgemm_modp call instead of the bench "
                         "(with --p, --form, --repeat)")
    ap.add_argument("--p", type=int, default=65521, help="prime of the --fgemm case")
    ap.add_argument("--fused-kmax", type=int, default=0,
                    help="limb products with K up to this split digits in the fgemm's producer")
    ap.add_argument("--no-thin", action="store_true",
                    help="no CUDA-core path for thin products (--fgemm case)")
    ap.add_argument("--fgemm-tile", type=int, default=0,
                    help="limb fgemm tile variant (0-2) of the --fgemm case, and of the bench "
                         "with --schedule (the autotuner picks it otherwise)")
    ap.add_argument("--repeat", type=int, default=2, help="calls of the --fgemm case")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world, rank, local = dist_setup()
    if args.fgemm:
        profile_fgemm(args)
    elif args.impl == "reference":
        bench_reference(args, world, rank)
    elif workloads.CONFIGS[args.workload].kind == "batched":
        bench_batched(args, world, rank, local)
    else:
        bench_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
