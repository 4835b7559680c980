#!/usr/bin/env python
"""Throughput benchmark of the fused D2Q9 SmrtLBM step on GB300.

One "step" is one application of the update (pull-stream + bounce-back +
moments + f^eq + SmrtLBM collision + store) over the whole lattice.  The
default workload is the periodic Taylor-Green vortex on 8192 x 8192 nodes
(u0 = 0.05, k = 2 pi / 8192, tau = 0.51), FP32 storage of f - w, two-buffer
layout; inputs (4.8 GB of populations) exceed the 129 MB L2, so no flush is
needed between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(a deliberately slow, plain program) on a bounded window of the same workload.
Multi-GPU runs are independent replicas (the update needs no collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

BYTES_PER_NODE = {"f64": 144, "f32": 72, "f16": 36, "bf16": 36}


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=["tgv8192", "cavity4096"], default="tgv8192")
    p.add_argument("--layout", choices=["ab", "aa"], default="ab")
    p.add_argument("--prec", choices=["f32", "f16", "bf16", "f64", "f16-sr", "bf16-sr"], default="f32",
                   help="storage precision; -sr: 16-bit storage with stochastic rounding")
    p.add_argument("--kind", choices=["smrt", "srt"], default="smrt")
    p.add_argument("--variant-steps", type=int, default=2000,
                   help="steps per extra variant line (0 disables the variants)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--size", type=int, default=0,
                   help="override the lattice side (profiling on a smaller case of the same workload)")
    p.add_argument("--report", choices=["", "precision", "batched", "batched-throughput", "learned", "paper", "unet"],
                   default="",
                   help="precision: 16-bit vs FP32 storage report; batched: 512 cavities to steady state "
                        "(each prints its own JSON line)")
    p.add_argument("--no-learned", action="store_true",
                   help="leave the learned warm-start leg (training + time to steady at the same error) out")
    p.add_argument("--learned-count", type=int, default=2000)
    p.add_argument("--learned-iters", type=int, default=12000)
    p.add_argument("--learned-cap", type=int, default=150000)
    p.add_argument("--learned-cap-1024", type=int, default=1000000)
    p.add_argument("--batch-count", type=int, default=512)
    p.add_argument("--batch-sides", default="64,128,256,512,1024")
    p.add_argument("--batch-re", default="100,5000", help="Re range (log-uniform) of the batched reports")
    p.add_argument("--batch-shape", type=int, default=-1,
                   help="batched-throughput: this tile shape (smrt_batch_set_shape) instead of autotuning")
    p.add_argument("--unet-batch", type=int, default=16)
    p.add_argument("--unet-iters", type=int, default=10)
    p.add_argument("--unet-backend", choices=["all", "tcgen05", "tcgen05-gather", "wmma"], default="all",
                   help="tcgen05: TMA-fed convolutions; tcgen05-gather: thread-gathered A tiles; wmma: legacy MMA")
    p.add_argument("--tol", type=float, default=1e-7)
    p.add_argument("--residual", choices=["stride", "step"], default="stride",
                   help="batched report: stride (mean change per update over a check) or one-step residual")
    p.add_argument("--check-every", type=int, default=500)
    p.add_argument("--max-steps", type=int, default=200000)
    p.add_argument("--oracle-steps", type=int, default=200)
    p.add_argument("--long-steps", type=int, default=20000)
    return p.parse_args(argv)


def workload(name, size=0):
    from paper_2409_01076_gb300 import workloads as W
    if name == "tgv8192":
        n = size or 8192
        return dict(name="tgv%d" % n, nx=n, ny=n, tau=0.51, u_lid=0.0, bc=W.ALL_PERIODIC, u0=0.05,
                    desc="periodic Taylor-Green vortex %dx%d, u0=0.05, k=2pi/%d, tau=0.51" % (n, n, n))
    n, U, re = size or 4096, 0.1, 1e4
    return dict(name="cavity%d" % n, nx=n, ny=n, tau=W.cavity_tau(n, U, re), u_lid=U, bc=W.CAVITY, u0=None,
                desc="lid-driven cavity %dx%d, Re=10000, U_lid=0.1, halfway bounce-back" % (n, n))


def initial_fields(wl):
    """Seeded/analytic initial (rho, u) on the host, float64."""
    from paper_2409_01076_gb300 import workloads as W
    if wl["u0"] is not None:
        return W.tgv_fields(wl["nx"], wl["ny"], wl["u0"])
    return W.rest_fields(wl["nx"], wl["ny"])


# ---- distributed plumbing (replicas only) ----------------------------------------

def dist_setup(n_gpus):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """Largest value of x over all ranks (the job is as slow as its slowest rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks during the timed region ------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, local_rank):
        self.proc = None
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        self.index = ids[local_rank] if local_rank < len(ids) and ids[local_rank].strip().isdigit() else str(local_rank)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], [], [], set()
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ---- measured peaks and committed ncu traffic ------------------------------------------

def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the sources the step kernel is compiled from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2409_01076_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name in ("d2q9.cuh", "kernels.cuh") or (name.startswith("prec_") and name.endswith(".cu")):
            with open(os.path.join(csrc, name), "rb") as fh:
                h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def committed_traffic(prec, layout, kind):
    """DRAM bytes per node update of the step kernel from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "step_kernel_traffic.md")
    try:
        text = open(path).read()
    except OSError:
        return None, None
    key = "%s-%s-%s" % (prec, layout, kind)
    src = None
    val = None
    for line in text.splitlines():
        if line.startswith("source_hash:"):
            src = line.split(":", 1)[1].strip()
        if line.startswith("traffic_bytes_per_node[%s]:" % key):
            val = float(line.split(":", 1)[1].strip())
    if val is None or src != kernel_source_hash():
        return None, src
    return val, src


# ---- the GPU arm ---------------------------------------------------------------------

def make_handle(S, wl, prec, layout, kind, check=True):
    """prec: f64, f32, f16 or bf16, with "-sr" for stochastic rounding of the 16-bit formats."""
    h = S.smrt_create(wl["nx"], wl["ny"], wl["tau"], wl["u_lid"], wl["bc"])
    if prec.endswith("-sr"):
        prec = prec[:-3]
        S.smrt_set_option(h, S.SMRT_OPT_ROUNDING, S.SMRT_ROUND_STOCHASTIC)
    S.smrt_set_option(h, S.SMRT_OPT_PRECISION, {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}[prec])
    S.smrt_set_option(h, S.SMRT_OPT_LAYOUT, {"ab": 0, "aa": 1}[layout])
    S.smrt_set_option(h, S.SMRT_OPT_COLLISION, {"smrt": 0, "srt": 1}[kind])
    S.smrt_set_option(h, S.SMRT_OPT_CHECK_DIVERGENCE, 1 if check else 0)
    return h


def time_steps(S, h, steps, world):
    """CUDA-event time (ms) of `steps` updates on the handle's stream (the legacy default stream)."""
    import torch
    barrier(world)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    S.smrt_step(h, steps)
    end.record()
    torch.cuda.synchronize()
    barrier(world)
    return start.elapsed_time(end)


def run_variant(S, wl, rho_d, u_d, prec, layout, kind, steps, warmup, world):
    h = make_handle(S, wl, prec, layout, kind)
    if wl["u0"] is not None:
        S.smrt_init_macros(h, rho_d, u_d)
    S.smrt_step(h, warmup)
    ms = max_over_ranks(time_steps(S, h, steps, world), world)
    S.smrt_destroy(h)
    nodes = wl["nx"] * wl["ny"]
    mlups = nodes * steps / (ms * 1e-3) / 1e6
    return {"mlups": round(mlups, 1), "ms_per_step": round(ms / steps, 5),
            "hbm_gbs": round(BYTES_PER_NODE[prec.replace("-sr", "")] * nodes / (ms / steps * 1e-3) / 1e9, 1),
            "steps": steps}


def host_link_gbs(host, reps=3):
    """Pinned host <-> device copy bandwidth (GB/s, best of reps, CUDA events) for a pinned tensor."""
    import torch
    dev = torch.empty(host.shape, dtype=host.dtype, device="cuda")
    best = {"h2d": 0.0, "d2h": 0.0}
    for _ in range(reps):
        for name, (dst, src) in (("h2d", (dev, host)), ("d2h", (host, dev))):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            dst.copy_(src, non_blocking=True)
            b.record()
            torch.cuda.synchronize()
            best[name] = max(best[name], host.numel() * host.element_size() / (a.elapsed_time(b) * 1e-3) / 1e9)
    del dev
    return best


def precision_errors(S, n=1024, re=5000.0, steps=20000, U=0.1):
    """Velocity error of each storage format against the FP64 path after `steps` updates of an n^2
    cavity (SmrtLBM, two-buffer layout): max and rms over nodes of |u - u_FP64| / U_lid.  The FP64
    path itself matches the FP64 CPU oracle to <= 1e-12 (parity tests)."""
    import torch
    from paper_2409_01076_gb300 import workloads as W
    wl = dict(nx=n, ny=n, tau=W.cavity_tau(n, U, re), u_lid=U, bc=W.CAVITY)
    us = {}
    for prec in ("f64", "f32", "f16", "bf16", "f16-sr", "bf16-sr"):
        h = make_handle(S, wl, prec, "ab", "smrt", check=False)
        S.smrt_step(h, steps)
        rho = torch.empty((n, n), dtype=torch.float64, device="cuda")
        u = torch.empty((2, n, n), dtype=torch.float64, device="cuda")
        S.smrt_macros(h, rho, u)
        S.smrt_destroy(h)
        us[prec] = u
    out = {"lattice": "lid-driven cavity %dx%d, Re %g, U_lid %g, tau %.5f" % (n, n, re, U, wl["tau"]),
           "steps": steps, "reference": "FP64 storage and arithmetic (same kernels)", "unit": "|du| / U_lid",
           "note": "-sr: stochastic rounding of the stored 16-bit offsets (SMRT_ROUND_STOCHASTIC)"}
    for prec in ("f32", "f16", "bf16", "f16-sr", "bf16-sr"):
        d = us[prec] - us["f64"]
        out[prec] = {"max": float(d.abs().amax()) / U, "rms": float((d * d).sum(0).mean().sqrt()) / U}
    return out


def e2e_run(S, wl, prec, layout, kind, steps, world, ms_per_step=None):
    """Same metric through the public C ABI with host buffers: pinned host (rho, u)
    in, K updates, pinned host (rho, u) out, all inside the timed region.  The
    library's kernels read and write the pinned buffers directly over the host link."""
    import torch
    rho, u = initial_fields(wl)
    rho_h = torch.from_numpy(rho).pin_memory()
    u_h = torch.from_numpy(u).pin_memory()
    rho_o = torch.empty_like(rho_h).pin_memory()
    u_o = torch.empty_like(u_h).pin_memory()
    link = host_link_gbs(u_h)
    h = make_handle(S, wl, prec, layout, kind)
    S.smrt_step(h, 1)                      # allocate the state outside the timed region
    S.smrt_macros(h, rho_o, u_o)           # and the staging buffer
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S.smrt_init_macros(h, rho_h, u_h)
    S.smrt_step(h, steps)
    S.smrt_macros(h, rho_o, u_o)
    t1 = time.perf_counter()
    barrier(world)
    S.smrt_destroy(h)
    sec = max_over_ranks(t1 - t0, world)
    nodes = wl["nx"] * wl["ny"]
    h2d = rho_h.numel() * 8 + u_h.numel() * 8
    d2h = rho_o.numel() * 8 + u_o.numel() * 8
    finite = bool(torch.isfinite(u_o).all())
    out = {"value": round(world * nodes * steps / sec / 1e6, 1), "unit": "MLUPS",
           "h2d_bytes_per_step": round(h2d / steps, 1), "d2h_bytes_per_step": round(d2h / steps, 1),
           "h2d_bytes_total": h2d, "d2h_bytes_total": d2h, "seconds": round(sec, 4), "steps": steps,
           "api": "smrt_init_macros(host) + smrt_step(K) + smrt_macros(host)", "result_finite": finite,
           "host_link_gbs": {k: round(v, 1) for k, v in link.items()},
           "host_buffers": "page-locked (pinned torch tensors), read and written by the kernels over the host link"}
    if ms_per_step:
        bound = h2d / (link["h2d"] * 1e9) + d2h / (link["d2h"] * 1e9) + steps * ms_per_step * 1e-3
        out["link_bound_seconds"] = round(bound, 4)
        out["frac_of_link_bound"] = round(bound / sec, 3)
    return out


# ---- the CPU oracle (baseline / reference arm) ------------------------------------------------

def oracle_sample(wl, side, steps):
    """Time the FP64 oracle on a side x side window of the same workload; returns (MLUPS, seconds)."""
    import oracle as O
    from paper_2409_01076_gb300 import workloads as W
    if wl["u0"] is not None:
        rho, u = W.tgv_fields(wl["nx"], wl["ny"], wl["u0"], 0, 0, side, side)
        f0 = O.init_equilibrium(rho, u)
        bc = O.ALL_PERIODIC
    else:
        f0 = O.cavity_initial(side, side)
        bc = O.CAVITY
    t0 = time.perf_counter()
    O.run(f0, steps, bc, wl["tau"], u_lid=wl["u_lid"])
    sec = time.perf_counter() - t0
    return side * side * steps / sec / 1e6, sec


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (x86 'model name'; Arm implementer and part codes)."""
    import platform
    fields = {}
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if "model name" in fields:
        return fields["model name"]
    if "CPU part" in fields:
        return "%s implementer %s part %s" % (platform.machine(), fields.get("CPU implementer", "?"), fields["CPU part"])
    return platform.machine() or "unknown"


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_init():
    import oracle as O
    O.lib()


def _oracle_job(job):
    wl, side, steps = job
    if wl is None:
        return 0.0
    return oracle_sample(wl, side, steps)[1]


def oracle_pool(cores):
    """One spawned process per host core, each with the oracle loaded (spawn: the parent may
    already hold a CUDA context)."""
    import multiprocessing
    pool = multiprocessing.get_context("spawn").Pool(cores, initializer=_oracle_init)
    try:
        pool.map_async(_oracle_job, [(None, 0, 0)] * cores, chunksize=1).get(timeout=300)
    except BaseException:
        pool.terminate()
        raise
    return pool


def oracle_all_cores(pool, cores, wl, side, steps):
    """Every core runs the unmodified oracle on its own side x side window; returns
    (aggregate MLUPS, wall seconds)."""
    t0 = time.perf_counter()
    pool.map_async(_oracle_job, [(wl, side, steps)] * cores, chunksize=1).get(timeout=900)
    sec = time.perf_counter() - t0
    return cores * side * side * steps / sec / 1e6, sec


def cpu_baseline(wl, budget_s=8.0):
    side = 512
    rate = oracle_sample(wl, side, 1)[0] * 1e6
    steps = max(1, int(budget_s * rate / (side * side)))
    mlups1, sec1 = oracle_sample(wl, side, steps)
    cores = host_cores()
    pool = oracle_pool(cores)
    try:
        mlups, sec = oracle_all_cores(pool, cores, wl, side, steps)
    finally:
        pool.terminate()
    return {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "single_core_value": round(mlups1, 3), "cpu": cpu_model(),
            "sample": "%dx%d window of the same workload (%s), %d steps, FP64 C oracle: one process per host "
                      "core (%d), each on its own window, %.1f s wall; single-threaded %.1f s"
                      % (side, side, wl["name"], steps, cores, sec, sec1)}


METRIC = "D2Q9 SmrtLBM MLUPS + % HBM roofline"


def reference_arm(args):
    rank, world, _ = dist_setup(args.gpus)
    if rank != 0:
        return 0
    wl = workload(args.workload, args.size)
    total = args.steps + args.warmup
    rate = oracle_sample(wl, 256, 1)[0] * 1e6
    side = int(math.sqrt(60.0 * rate / max(total, 1)))
    side = max(16, min(1024, side))
    cores = host_cores()
    pool = oracle_pool(cores)
    try:
        for _ in range(args.warmup):
            oracle_all_cores(pool, cores, wl, side, 1)
        sec = 0.0
        for _ in range(args.steps):
            sec += oracle_all_cores(pool, cores, wl, side, 1)[1]
    finally:
        pool.terminate()
    mlups = cores * side * side * args.steps / sec / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(sec / args.steps * 1e3, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"], "nodes": wl["nx"] * wl["ny"], "storage": "f64 populations (CPU oracle)",
                   "layout": args.layout, "collision": args.kind, "l2": "CPU run; no GPU L2 involved",
                   "parallelism": "one process per host core", "sample": "%dx%d window per core per step"
                   % (side, side)},
        "cpu_baseline": {"value": round(mlups, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "cpu": cpu_model(), "sample": "%dx%d window of %s per core, one update per step, FP64 C oracle in one "
                                   "process per host core" % (side, side, wl["name"])},
        "e2e": {"value": round(mlups, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def gpu_arm(args):
    import torch
    import paper_2409_01076_gb300 as S

    rank, world, local = dist_setup(args.gpus)
    wl = workload(args.workload, args.size)
    nodes = wl["nx"] * wl["ny"]
    S._lib.load()

    rho, u = initial_fields(wl)
    rho_d = torch.from_numpy(rho).cuda()
    u_d = torch.from_numpy(u).cuda()
    del rho, u

    h = make_handle(S, wl, args.prec, args.layout, args.kind)
    S.smrt_init_macros(h, rho_d, u_d)
    S.smrt_step(h, max(args.warmup, 3))
    clocks = ClockSampler(local)
    clocks.start()
    ms = time_steps(S, h, args.steps, world)
    clk = clocks.stop()
    r, sums = S.smrt_residual(h)
    S.smrt_destroy(h)
    ms = max_over_ranks(ms, world)
    sec = ms * 1e-3
    mlups = world * nodes * args.steps / sec / 1e6
    per_launch = sec / args.steps
    peak, peak_src = measured_hbm_peak()
    achieved = BYTES_PER_NODE[args.prec.replace("-sr", "")] * nodes / per_launch / 1e9
    traffic_per_node, _ = committed_traffic(args.prec, args.layout, args.kind)

    result = {
        "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": round(ms / args.steps, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if args.prec == "f32" else args.prec, "data": "synthetic",
        "config": {"workload": wl["desc"], "nodes": nodes, "storage": "%s offsets f - w" % args.prec,
                   "layout": args.layout, "collision": args.kind,
                   "l2": "no flush: populations (%.2f GB) exceed the 129 MB L2"
                         % (BYTES_PER_NODE[args.prec.replace("-sr", "")] / 2 * nodes * (2 if args.layout == "ab" else 1) / 1e9),
                   "parallelism": "replicas x%d" % world},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src
                     if peak_src == "measured" else "fallback 6.8 TB/s",
                     "traffic": (round(traffic_per_node * nodes) if traffic_per_node else None),
                     "algorithmic_bytes_per_launch": BYTES_PER_NODE[args.prec.replace("-sr", "")] * nodes,
                     "kernel": "step_kernel<%s,%s,%s>" % (args.prec, args.kind, args.layout)},
        "gpu_launches": args.steps,
        "clocks": clk,
        "check": {"residual_after": r, "mass_rel_err": abs(sums[0] / nodes - 1.0)},
    }

    if args.variant_steps > 0:
        variants = {}
        vs = args.variant_steps
        for prec, layout, kind in [("f32", "ab", "srt"), ("f32", "aa", "smrt"), ("f32", "aa", "srt"),
                                   ("f16", "ab", "smrt"), ("bf16", "ab", "smrt"), ("f16", "aa", "smrt"),
                                   ("f16-sr", "ab", "smrt"), ("bf16-sr", "ab", "smrt"), ("f16-sr", "aa", "smrt")]:
            if (prec, layout, kind) == (args.prec, args.layout, args.kind):
                continue
            variants["%s-%s-%s" % (prec, layout, kind)] = run_variant(S, wl, rho_d, u_d, prec, layout, kind, vs,
                                                                      10, world)
        if wl["name"] == "tgv8192":
            cav = workload("cavity4096")
            for layout, kind in [("ab", "smrt"), ("ab", "srt"), ("aa", "smrt")]:
                variants["cavity4096-f32-%s-%s" % (layout, kind)] = run_variant(
                    S, cav, None, None, "f32", layout, kind, vs, 10, world)
            variants["batched512-f32-ab-smrt"] = batched_throughput(S, max(vs // 10, 20))
        result["variants"] = variants
        if rank == 0:
            result["precision_error"] = precision_errors(S)

    del rho_d, u_d
    torch.cuda.empty_cache()
    if not args.no_e2e:
        result["e2e"] = e2e_run(S, wl, args.prec, args.layout, args.kind, args.steps, world, ms / args.steps)
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(wl)
    elif not args.no_cpu:
        result["cpu_baseline"] = None
    if rank == 0 and world == 1 and not args.no_learned:
        result["learned"] = learned_leg(args)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def batched_setup(S, count=512, seed=0, layout="ab", sides=(64, 128, 256, 512, 1024), re=(100.0, 5000.0)):
    """The seeded uneven batch: sides uniform over {64..1024}, Re log-uniform in [100, 5000], U_lid = 0.1."""
    from paper_2409_01076_gb300 import workloads as W
    cav = W.batched_cavities(count, seed, sides=tuple(sides), re_lo=re[0], re_hi=re[1])
    nx = [n for n, _ in cav]
    taus = [W.cavity_tau(n, 0.1, re) for n, re in cav]
    b = S.smrt_batch_create(nx, nx, taus, [0.1] * count, W.CAVITY, S.SMRT_PREC_F32,
                            {"ab": 0, "aa": 1}[layout], S.SMRT_COLLISION_SMRT)
    return b, cav


def batched_throughput(S, steps, layout="ab", count=512, sides=(64, 128, 256, 512, 1024), re=(100.0, 5000.0),
                       shape=-1):
    """MLUPS of smrt_batch_step over the lattices active when the timed call starts (a lattice that
    diverges is still updated until the call returns, and retired after it)."""
    import numpy as np
    import torch
    b, cav = batched_setup(S, count=count, layout=layout, sides=sides, re=re)
    if shape >= 0:
        S.smrt_batch_set_shape(b, shape)
        choice = shape
    else:
        choice = S.smrt_batch_autotune(b, 10)
    S.smrt_batch_step(b, 4)
    torch.cuda.synchronize()
    side = np.array([n for n, _ in cav], dtype=np.int64)
    active = S.smrt_batch_status(b)[2] == S.SMRT_BATCH_ACTIVE
    nodes = int((side[active] ** 2).sum())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    S.smrt_batch_step(b, steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    after = int((S.smrt_batch_status(b)[2] == S.SMRT_BATCH_ACTIVE).sum())
    S.smrt_batch_destroy(b)
    return {"mlups": round(nodes * steps / (ms * 1e-3) / 1e6, 1), "ms_per_step": round(ms / steps, 5),
            "hbm_gbs": round(72 * nodes / (ms / steps * 1e-3) / 1e9, 1), "steps": steps, "cavities": len(cav),
            "active": int(active.sum()), "active_after": after, "re": list(re),
            "nodes": nodes, "tile_shape_choice": choice, "layout": layout}


def batched_report(args):
    """512 uneven cavities (seed 0) run to stride residual 1e-7 in one batch, with a step cap."""
    import numpy as np
    import torch
    import paper_2409_01076_gb300 as S
    torch.cuda.set_device(0)
    S._lib.load()
    b, cav = batched_setup(S, count=args.batch_count, layout=args.layout, sides=_sides(args), re=_re(args))
    nodes = S.smrt_batch_nodes(b)
    t0 = time.perf_counter()
    choice = S.smrt_batch_autotune(b, 10)
    t1 = time.perf_counter()
    kind = S.SMRT_BATCH_RESIDUAL_STRIDE if args.residual == "stride" else S.SMRT_BATCH_RESIDUAL_STEP
    S.smrt_batch_run(b, args.tol, args.check_every, args.max_steps, kind)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    steps, res, state = S.smrt_batch_status(b)
    node_steps = sum(n * n * int(s) for (n, _), s in zip(cav, steps))
    out = {"report": "batched", "cavities": len(cav), "nodes": nodes, "tol": args.tol, "residual": args.residual,
           "check_every": args.check_every, "max_steps": args.max_steps, "layout": args.layout,
           "tile_shape_choice": choice, "autotune_s": round(t1 - t0, 3), "run_s": round(t2 - t1, 3),
           "node_updates": node_steps, "mlups_effective": round(node_steps / (t2 - t1) / 1e6, 1),
           "converged": int((state == S.SMRT_BATCH_CONVERGED).sum()),
           "capped": int((state == S.SMRT_BATCH_CAPPED).sum()),
           "diverged": int((state == S.SMRT_BATCH_DIVERGED).sum()),
           "by_side": {}}
    for side in sorted(set(n for n, _ in cav)):
        idx = [k for k, (n, _) in enumerate(cav) if n == side]
        conv = [k for k in idx if state[k] == S.SMRT_BATCH_CONVERGED]
        out["by_side"][str(side)] = {
            "count": len(idx), "converged": len(conv),
            "steps_median": float(np.median([steps[k] for k in conv])) if conv else None,
            "steps_max": int(max(steps[k] for k in conv)) if conv else None,
            "final_residual_quartiles": [float(np.quantile([res[k] for k in idx], q)) for q in (0.0, 0.25, 0.5,
                                                                                              0.75, 1.0)],
            "re_range": [round(min(cav[k][1] for k in idx), 1), round(max(cav[k][1] for k in idx), 1)]}
    S.smrt_batch_destroy(b)
    print(json.dumps(out), flush=True)
    return 0


def paper_experiments_report(args):
    """The paper's cavity experiments as stability demonstrations, SmrtLBM against SRT on the same GPU.

    Lattice parameters follow the paper's statement (tau fixed, Re = U L / nu with L = n under halfway
    bounce-back, nu = (tau - 1/2) / 3), so U_lid = Re nu / n:
      E1: 100^2, Re 1,000, tau 0.51, 60,000 steps (steady state claimed);
      E2: Re 10,000, tau 0.51 on 100^2, 200^2, 250^2;
      E4: 400^2, Re 100,000, tau 0.502, 100,000 steps (no instability claimed).
    Reports divergence (the flag), steps completed and the final one-step and stride residuals."""
    import numpy as np
    import torch
    import paper_2409_01076_gb300 as S
    from paper_2409_01076_gb300 import workloads as W
    torch.cuda.set_device(0)
    S._lib.load()
    cases = [("E1", 100, 1000.0, 0.51, 60000), ("E2", 100, 1e4, 0.51, 60000), ("E2", 200, 1e4, 0.51, 60000),
             ("E2", 250, 1e4, 0.51, 100000), ("E4", 400, 1e5, 0.502, 100000)]
    out = {"report": "paper-experiments", "cases": []}
    for name, n, re, tau, steps in cases:
        nu = (tau - 0.5) / 3.0
        u_lid = re * nu / n
        for kind, kname in ((S.SMRT_COLLISION_SMRT, "smrt"), (S.SMRT_COLLISION_SRT, "srt")):
            h = S.smrt_create(n, n, tau, u_lid, W.CAVITY)
            S.smrt_set_option(h, S.SMRT_OPT_PRECISION, S.SMRT_PREC_F32)
            S.smrt_set_option(h, S.SMRT_OPT_COLLISION, kind)
            status, done, chunk = "finite", 0, 1000
            t0 = time.perf_counter()
            while done < steps:
                try:
                    S.smrt_step(h, chunk)
                except S.SmrtError as e:
                    if e.status != S.SMRT_ERR_DIVERGED:
                        raise
                    status = "diverged"
                    done += chunk
                    break
                done += chunk
            sec = time.perf_counter() - t0
            entry = {"case": name, "n": n, "re": re, "tau": tau, "u_lid": round(u_lid, 6), "collision": kname,
                     "status": status, "steps": done if status == "finite" else "<= %d" % done,
                     "seconds": round(sec, 3)}
            if status == "finite":
                r1, sums = S.smrt_residual(h)
                rho = np.empty((n, n))
                u = np.empty((2, n, n))
                S.smrt_macros(h, rho, u)
                S.smrt_step(h, 1000)
                u2 = np.empty((2, n, n))
                S.smrt_macros(h, rho, u2)
                entry.update({"residual_one_step": r1,
                              "residual_stride_1000": float(np.linalg.norm(u2 - u) / (1000 * np.linalg.norm(u2))),
                              "mass_rel_change": sums[0] / (n * n) - 1.0,
                              "max_speed_over_U": float(np.sqrt(u2[0] ** 2 + u2[1] ** 2).max() / u_lid)})
            S.smrt_destroy(h)
            out["cases"].append(entry)
    print(json.dumps(out), flush=True)
    return 0


def _geomean(xs):
    import numpy as np
    xs = [x for x in xs if x]
    return float(np.exp(np.mean(np.log(xs)))) if xs else None


def learned_leg(args, held_out=((256, "f64", (130.0, 400.0, 1200.0, 2500.0), 400000, (1e-3,)),
                                (1024, "f32", (130.0, 400.0, 1200.0), 1200000, (1e-3,)))):
    """The learned warm start of the 256^2 cavity workload, trained in this run: 2,000 solver-generated
    steady cavities (Re log-uniform in [100, 1e4]), U-Net training on the GPU, then time to steady state
    at the same error, cold vs warm, on held-out Re (warmstart.time_to_same_error): 256^2 in FP64 and
    1024^2 in FP32, each at the plain method's own error at its criterion and at 1e-3 U."""
    import torch
    import paper_2409_01076_gb300 as S
    from paper_2409_01076_gb300 import warmstart as WS
    from paper_2409_01076_gb300.unet import UNet
    t0 = time.perf_counter()
    res_train = WS.sample_res(args.learned_count, seed=1)
    targets, info = WS.generate_dataset(res_train, 256, args.tol, 1000, args.learned_cap)
    net = UNet(base=32, seed=0)
    hist, train_s = WS.train(net, res_train, targets, iters=args.learned_iters, batch=16, lr=1e-3, warmup=100)
    del targets
    torch.cuda.empty_cache()
    out = {"workload": "U-Net (4 levels, 32 base channels, half operands / float32 accumulation) trained on "
                       "%d solver-generated 256^2 cavities, U_lid 0.1, Re log-uniform in [100, 1e4]"
                       % args.learned_count,
           "dataset": info, "params": net.n_params(),
           "training": {"iters": args.learned_iters, "batch": 16, "lr": 1e-3, "seconds": round(train_s, 2),
                        "loss_first_last": [hist[0][1], hist[-1][1]]},
           "error_definition": "each run (cold from rest, warm from the prediction) is continued past the plain "
                               "method's criterion (stride residual < %g) until its residual < 1e-11 or 4x (FP64) "
                               "/ 3x (FP32) the criterion's steps: its own converged field u_inf; "
                               "e(t) = max over nodes |u(t) - u_inf| / U_lid; same error = the cold run's e at "
                               "its criterion; the warm run's steps are those until its e falls to that; "
                               "final_diff = max |u_inf,warm - u_inf,cold| / U_lid (the steady state depends on "
                               "the start: halfway bounce-back leaves it non-unique)" % args.tol,
           "residual": "stride: ||u(t) - u(t-K)|| / (K ||u(t)||), K = 1000", "cases": []}
    for n, prec, res, cap, levels in held_out:
        p = {"f64": S.SMRT_PREC_F64, "f32": S.SMRT_PREC_F32}[prec]
        rows = WS.time_to_same_error(net, res, n, p, args.tol, 1e-11, levels, 1000, cap,
                                     ref_factor=4 if prec == "f64" else 3)
        out["cases"].extend(rows)
        summary = {"precision": prec, "cavities": len(rows)}
        for name in ["same_error"] + ["level_%g" % lv for lv in levels]:
            done = [r["targets"][name] for r in rows if not r["capped"] and "steps_factor" in r["targets"][name]]
            summary[name] = {"steps_factor_geomean": _geomean([t["steps_factor"] for t in done]),
                             "wall_factor_geomean": _geomean([t["wall_factor"] for t in done]),
                             "compared": len(done)}
        out["n%d_%s" % (n, prec)] = summary
    out["seconds"] = round(time.perf_counter() - t0, 1)
    return out


def learned_report(args):
    """The learned leg of the default line on the full held-out set (256^2 and 1024^2 at Re 130, 400,
    1,200, 3,500 and 8,000), printed as its own JSON line."""
    import torch
    import paper_2409_01076_gb300 as S
    torch.cuda.set_device(0)
    S._lib.load()
    full = (130.0, 400.0, 1200.0, 3500.0, 8000.0)
    out = learned_leg(args, held_out=((256, "f64", full, args.learned_cap * 2, (1e-3,)),
                                      (256, "f32", full, args.learned_cap * 2, (1e-3,)),
                                      (1024, "f32", full, args.learned_cap_1024, (1e-3,))))
    out["report"] = "learned"
    print(json.dumps(out), flush=True)
    return 0


def unet_report(args):
    """Training-step time of the warm-start U-Net (32 base channels, 256^2 inputs, seeded synthetic
    inputs and targets) for each GEMM backend: CUDA events over --unet-iters steps after 3 warm-up steps."""
    import torch
    import paper_2409_01076_gb300 as S
    from paper_2409_01076_gb300.unet import UNet, input_grid
    torch.cuda.set_device(0)
    S._lib.load()
    B = args.unet_batch
    res = [100.0 * 100.0 ** (k / max(B - 1, 1)) for k in range(B)]
    x = input_grid(res, 256, 256)
    g = torch.Generator(device="cuda").manual_seed(0)
    target = 0.1 * torch.randn((B, 256, 256, 3), device="cuda", generator=g)
    out = {"report": "unet", "batch": B, "side": 256, "base_channels": 32, "iters": args.unet_iters}
    variants = {"tcgen05": ("tcgen05", "tma"), "tcgen05-gather": ("tcgen05", "gather"), "wmma": ("wmma", "gather")}
    for backend in (list(variants) if args.unet_backend == "all" else [args.unet_backend]):
        gemm, conv = variants[backend]
        for graph in ((False, True) if backend == "tcgen05" else (False,)):
            net = UNet(base=32, gemm=gemm, conv=conv)
            for _ in range(3):
                net.train_step(x, target, 1e-3)
            if graph:
                net.capture(x, target)          # forward + backward as one CUDA graph; Adam eager
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.unet_iters):
                if graph:
                    net.replay()
                else:
                    net.loss_and_grad(x, target)
                net.adam_step(1e-3)
            e1.record()
            torch.cuda.synchronize()
            out[backend + ("+graph" if graph else "")] = {
                "ms_per_step": round(e0.elapsed_time(e1) / args.unet_iters, 3),
                "gemm_timeouts": net.gemm_timeouts(), "params": net.n_params()}
    print(json.dumps(out), flush=True)
    return 0


def _oracle_cavity_u(n, re, steps):
    """FP64 oracle: u after `steps` updates of an n x n cavity (U_lid = 0.1) at Reynolds number re."""
    import oracle as O
    from paper_2409_01076_gb300 import workloads as W
    tau = W.cavity_tau(n, 0.1, re)
    f = O.run(O.cavity_initial(n, n), steps, O.CAVITY, tau, u_lid=0.1)
    return O.macros(f)[1]


def precision_report(args):
    """16-bit offset storage vs FP32 storage: throughput on 8192^2 cavities at Re 5000 / 20000, and
    velocity error of each storage format on the 1024^2 cavity at the same Re, against the FP64
    oracle (short horizon) and against the FP64 GPU path (long horizon)."""
    import multiprocessing as mp
    import numpy as np
    n_err, s_oracle, s_long = 1024, args.oracle_steps, args.long_steps
    res_list = (5000.0, 20000.0)
    # the oracle runs in spawned processes, started before this process touches CUDA
    pool = mp.get_context("spawn").Pool(len(res_list))
    pending = {re: pool.apply_async(_oracle_cavity_u, (n_err, re, s_oracle)) for re in res_list}
    pool.close()

    import torch
    import paper_2409_01076_gb300 as S
    from paper_2409_01076_gb300 import workloads as W
    torch.cuda.set_device(0)
    S._lib.load()
    precs = {"f64": 0, "f32": 1, "f16": 2, "bf16": 3}

    def gpu_u(n, re, steps, prec, layout=0):
        h = S.smrt_create(n, n, W.cavity_tau(n, 0.1, re), 0.1, W.CAVITY)
        if prec.endswith("-sr"):
            prec = prec[:-3]
            S.smrt_set_option(h, S.SMRT_OPT_ROUNDING, S.SMRT_ROUND_STOCHASTIC)
        S.smrt_set_option(h, S.SMRT_OPT_PRECISION, precs[prec])
        S.smrt_set_option(h, S.SMRT_OPT_LAYOUT, layout)
        S.smrt_step(h, steps)
        rho = np.empty((n, n))
        u = np.empty((2, n, n))
        S.smrt_macros(h, rho, u)
        S.smrt_destroy(h)
        return u

    out = {"report": "precision", "unit_error": "velocity error / U_lid", "U_lid": 0.1, "error_lattice": n_err,
           "oracle_steps": s_oracle, "long_steps": s_long, "by_re": {}}
    for re in res_list:
        entry = {"tau_1024": W.cavity_tau(n_err, 0.1, re), "tau_8192": W.cavity_tau(8192, 0.1, re)}
        # throughput on the 8192^2 cavity
        wl = dict(name="cavity8192", nx=8192, ny=8192, tau=W.cavity_tau(8192, 0.1, re), u_lid=0.1, bc=W.CAVITY,
                  u0=None, desc="")
        thr = {}
        for prec in ("f32", "f16", "bf16", "f16-sr", "bf16-sr"):
            for layout in ("ab", "aa"):
                thr["%s-%s" % (prec, layout)] = run_variant(S, wl, None, None, prec, layout, "smrt",
                                                            args.variant_steps or 1000, 10, 1)
        entry["throughput_8192"] = thr
        u64_long = gpu_u(n_err, re, s_long, "f64")
        long_err = {}
        for prec in ("f32", "f16", "bf16", "f16-sr", "bf16-sr"):
            d = gpu_u(n_err, re, s_long, prec) - u64_long
            long_err[prec] = {"max": float(np.abs(d).max() / 0.1), "rms": float(np.sqrt((d * d).mean()) / 0.1)}
        entry["error_vs_gpu_f64_long"] = long_err
        entry["gpu_f64_speed_max"] = float(np.abs(u64_long).max())
        u_ref = pending[re].get()
        short_err = {}
        for prec in ("f64", "f32", "f16", "bf16", "f16-sr", "bf16-sr"):
            d = gpu_u(n_err, re, s_oracle, prec) - u_ref
            short_err[prec] = {"max": float(np.abs(d).max() / 0.1), "rms": float(np.sqrt((d * d).mean()) / 0.1)}
        entry["error_vs_oracle"] = short_err
        out["by_re"]["%d" % re] = entry
    pool.join()
    print(json.dumps(out), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return reference_arm(args)
    if args.report == "precision":
        return precision_report(args)
    if args.report == "batched":
        return batched_report(args)
    if args.report == "learned":
        return learned_report(args)
    if args.report == "paper":
        return paper_experiments_report(args)
    if args.report == "unet":
        return unet_report(args)
    if args.report == "batched-throughput":
        import torch
        import paper_2409_01076_gb300 as S
        torch.cuda.set_device(0)
        S._lib.load()
        out = batched_throughput(S, args.steps, args.layout, args.batch_count, _sides(args), _re(args),
                                 args.batch_shape)
        out["report"] = "batched-throughput"
        print(json.dumps(out), flush=True)
        return 0
    return gpu_arm(args)


def _sides(args):
    return tuple(int(s) for s in args.batch_sides.split(","))


def _re(args):
    lo, hi = (float(s) for s in args.batch_re.split(","))
    return lo, hi


if __name__ == "__main__":
    sys.exit(main())
