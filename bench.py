"""Throughput of the GB300 particle-mesh step with quantum pressure.

Workload: one simulation of 128^3 particles on a 256^3 periodic mesh,
L = 2 Mpc/h, m = 2.5e-22 eV, Omega_m = 0.3, Omega_L = 0.7, h = 0.7, fp32
(int32 cell + fp32 offset positions, fp32 mesh and cuFFT), Zel'dovich initial
conditions at z = 100 from the seed-42 Gaussian field with
P ~ k^0.96 T_BBKS^2 T_FDM^2, 500 leapfrog steps (uniform in ln a) to z = 3.
A step is one pass of the whole path: interpolate + kick + drift, radix sort
by cell, row starts, deterministic CIC deposit, R2C FFT, Green's function,
C2R FFT, quantum-pressure stencil.  The timed steps are W..W+K of that
schedule.  Each step touches ~0.5 GB (> the 126 MB L2), so no L2 flush is
inserted between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 (torchrun): independent replicas, one per GPU, no data-path collective.
--impl reference times the FP64 CPU oracle on the host cores instead.
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="single sim 128^3 particles on 256^3 mesh, L=2 Mpc/h, m22=2.5, z=100->3 in 500 steps",
                n_side=128, n_mesh=256, box=2.0, m22=2.5, z_start=100.0, z_end=3.0, nsteps=500, seed=42)
METRIC = "particle-steps/s"
PROFILES = os.path.join(ROOT, "profiles")


def schedule(w):
    a0, a1 = 1.0 / (1.0 + w["z_start"]), 1.0 / (1.0 + w["z_end"])
    return a0 * (a1 / a0) ** (np.arange(w["nsteps"] + 1) / w["nsteps"])


def algorithmic_bytes(stage, n, n_mesh, rsz=4):
    """Minimal DRAM bytes of one launch of each kernel (fp32 path)."""
    n3 = n_mesh ** 3
    spec = n_mesh * n_mesh * (n_mesh // 2 + 1) * 2 * rsz
    rec = 4 * rsz
    return {
        # pos + mom read and written, new key written; phi~ and Q~ read once
        "kick": n * (4 * rec + 4) + 2 * n3 * rsz,
        # particle positions read once, row starts read once, rho written
        "deposit": n * rec + n_mesh * n_mesh * 4 + n3 * rsz,
        # rho read, Q~ written
        "stencil": 2 * n3 * rsz,
        # half spectrum read and written
        "green": 2 * spec,
        "fft_r2c": n3 * rsz + spec,
        "fft_c2r": spec + n3 * rsz,
        # re-sort after a drift: keys read twice (count, scatter), stayer keys + previous slots written
        "sort_partition": n * 16,
        # stayers (key, slot) read, sorted keys written, records gathered (read) and written
        "sort_merge": n * (8 + 4 + 4 * rec),
        # the histogram and radix passes see only the movers, a data-dependent count
        "sort_histogram": None,
        "sort_pass": None,
        "row_start": n * 4 + n_mesh * n_mesh * 4,
    }.get(stage)


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def csrc_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1608_00802_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (profiles/traffic.json)."""
    try:
        with open(os.path.join(PROFILES, "traffic.json")) as fh:
            d = json.load(fh)
        e = d[kernel]
        if e.get("csrc") != csrc_hash() or e.get("workload") != workload:
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [c.strip() for c in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, col in (("hw_slowdown", 5), ("hw_thermal_slowdown", 6), ("sw_thermal_slowdown", 7),
                                  ("sw_power_cap", 8)):
                    if f[col].lower().startswith("active"):
                        reasons.add(name)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group("gloo")
    return dist


def max_over_ranks(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------- CPU oracle
def oracle_step_rate(w, budget_s=30.0):
    """Times the FP64 CPU oracle on a bounded sample of the workload: the same
    recipe, one step, on the full problem if one step fits the budget, else on
    a proportionally smaller box (the mesh/particle ratio kept)."""
    from oracle import pm_oracle as O
    from paper_1608_00802_gb300 import ics
    n_side, n_mesh, box = w["n_side"], w["n_mesh"], w["box"]
    # per-step cost is ~13 s for 128^3 on 256^3 on one core; shrink by 2 per dimension until it fits
    est = 13.0 * (n_side / 128.0) ** 3
    while est > budget_s and n_side > 16:
        n_side, n_mesh, box, est = n_side // 2, n_mesh // 2, box / 2, est / 8
    a = schedule(w)
    x, p = ics.zeldovich(n_side, n_mesh, box, a[0], w["seed"], m22=w["m22"])
    cfg = O.Config(n_mesh=n_mesh, box=box, m22=w["m22"], force_mode=O.HYBRID)
    parts = O.force_parts(x, cfg)
    t0 = time.perf_counter()
    O.kdk_step(x, p, a[0], a[1], cfg, parts)
    dt = time.perf_counter() - t0
    sample = "1 KDK step (one force evaluation) of %d^3 particles on %d^3 mesh, L=%g" % (n_side, n_mesh, box)
    return n_side ** 3 / dt, dt, sample


def cpu_cores_used():
    # the oracle's numpy kernels (bincount, fancy indexing, numpy.fft/pocketfft,
    # elementwise ufuncs) run on one thread
    return 1


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = WORKLOAD
    total = args.steps + args.warmup
    budget = max(2.0, 150.0 / max(total, 1))
    from oracle import pm_oracle as O
    from paper_1608_00802_gb300 import ics
    n_side, n_mesh, box = w["n_side"], w["n_mesh"], w["box"]
    est = 13.0
    while est > budget and n_side > 16:
        n_side, n_mesh, box, est = n_side // 2, n_mesh // 2, box / 2, est / 8
    a = schedule(w)
    x, p = ics.zeldovich(n_side, n_mesh, box, a[0], w["seed"], m22=w["m22"])
    cfg = O.Config(n_mesh=n_mesh, box=box, m22=w["m22"], force_mode=O.HYBRID)
    parts = None
    for i in range(args.warmup):
        x, p, parts = O.kdk_step(x, p, a[i], a[i + 1], cfg, parts)
    t0 = time.perf_counter()
    for i in range(args.warmup, args.warmup + args.steps):
        x, p, parts = O.kdk_step(x, p, a[i], a[i + 1], cfg, parts)
    dt = time.perf_counter() - t0
    value = n_side ** 3 * args.steps / dt
    sample = "%d KDK steps of %d^3 particles on %d^3 mesh, L=%g (bounded sample of the workload)" % (
        args.steps, n_side, n_mesh, box)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["name"], "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch

    from paper_1608_00802_gb300 import build as _b
    rank, world, local = dist_env()
    dist = init_dist(world)
    torch.cuda.set_device(local)
    if rank == 0 or dist is None:
        _b.build()
    if dist is not None:
        dist.barrier()
    from paper_1608_00802_gb300 import ics, pm

    w = WORKLOAD
    a = schedule(w)
    K, W = args.steps, args.warmup
    if W + 2 * K > w["nsteps"]:
        raise SystemExit("warmup + 2 * steps must be <= %d" % w["nsteps"])
    x, p = ics.zeldovich(w["n_side"], w["n_mesh"], w["box"], a[0], w["seed"] + rank, m22=w["m22"])
    n = len(x)
    cfg = pm.make_config(n, w["n_mesh"], w["box"], precision=pm.FP32, m22=w["m22"],
                         force_mode=pm.FORCE_HYBRID, fft_jit=True)  # a long-lived simulation
    stream = torch.cuda.Stream()
    sim = pm.Sim(cfg, stream=stream)
    sim.set_particles(x, p)
    # launch shapes measured on this simulation (untimed), or given
    if args.tuning:
        sim.set_tuning(dict(sim.get_tuning(), **json.loads(args.tuning)))
        tuning = sim.get_tuning()
    else:
        tuning = sim.autotune(reps=5)
    # warm-up steps (untimed): the first W steps of the schedule
    with torch.cuda.stream(stream):
        if W > 0:
            sim.run(W, a[0], a[W])
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        with Clocks(local) as clk:
            ev0.record(stream)
            sim.run(K, a[W], a[W + K])
            ev1.record(stream)
            torch.cuda.synchronize()
        t_ms = ev0.elapsed_time(ev1)
        # per-kernel durations: the next K steps again, launched one by one with an
        # event pair around every launch (kernel times do not depend on graph replay)
        sim.profile_begin(64 * (K + 2))
        sim.run(K, a[W + K], a[W + 2 * K])
        stages = sim.profile_end()
    if dist is not None:
        dist.barrier()
    t_max = max_over_ranks(dist, t_ms)
    units = sum_over_ranks(dist, n * K)
    value = units / (t_max / 1e3)

    # per-kernel roofline (ours only; cuFFT reported beside)
    peak, peak_kind = read_peaks()
    per_stage = {}
    for name, (ms, cnt) in stages.items():  # ms over the K profiled steps
        if cnt == 0:
            continue
        b = algorithmic_bytes(name, n, w["n_mesh"])
        avg = ms / cnt
        per_stage[name] = {"ms_per_step": ms / K, "launches": cnt, "avg_launch_ms": avg,
                           "GBps": (b / (avg / 1e3) / 1e9) if b else None}
    ours = {k: v for k, v in per_stage.items() if k not in pm.CUFFT_STAGES and v["GBps"] is not None}
    dom = max(ours, key=lambda k: ours[k]["ms_per_step"])
    d = per_stage[dom]
    achieved = d["GBps"]
    kernel_names = {"kick": "k_kick_stream", "deposit": "k_deposit", "stencil": "k_stencil", "green": "k_green",
                    "sort_pass": "k_sort_pass", "sort_histogram": "k_sort_histogram",
                    "row_start": "k_row_start", "sort_partition": "k_mover_partition",
                    "sort_merge": "k_merge_gather"}
    roofline = {"bound": "hbm", "kernel": kernel_names.get(dom, dom), "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak if achieved else None,
                "traffic": ncu_traffic(kernel_names.get(dom, dom), "c2"), "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": algorithmic_bytes(dom, n, w["n_mesh"])}
    # our kernels per timed region: the profiled pass launches the same kernels one by one; the replayed
    # graph adds one step-counter kernel per step
    launches = sum(v["launches"] for k, v in per_stage.items() if k not in pm.CUFFT_STAGES) + K
    # the whole step against the copy bandwidth: algorithmic bytes of every stage with a fixed count
    # (the radix passes over the movers are left out) over the graph-timed step, with and without cuFFT
    step_bytes, step_bytes_fft, fft_ms = 0.0, 0.0, 0.0
    for name, (ms, cnt) in stages.items():
        b = algorithmic_bytes(name, n, w["n_mesh"])
        if cnt and b:
            step_bytes += b * cnt / K
            if name in pm.CUFFT_STAGES:
                step_bytes_fft += b * cnt / K
                fft_ms += ms / K
    t_step = t_max / K
    step_roofline = {"bytes_per_step": step_bytes, "achieved_GBps": step_bytes / (t_step / 1e3) / 1e9,
                     "frac": step_bytes / (t_step / 1e3) / 1e9 / peak,
                     "frac_excl_cufft": ((step_bytes - step_bytes_fft) / (max(t_step - fft_ms, 1e-9) / 1e3) / 1e9
                                         / peak),
                     "note": "cuFFT time taken from the profiled pass; peak as in roofline"}

    # end to end through the C ABI with pinned host buffers
    xh = torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()
    ph = torch.from_numpy(np.ascontiguousarray(p)).pin_memory().numpy()
    xo = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    po = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    sim2 = sim
    with torch.cuda.stream(stream):
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2.set_particles(xh, ph)
        sim2.run(K, a[0], a[K])
        sim2.get_particles(xo, po)
        t_e2e = time.perf_counter() - t0
    t_e2e = max_over_ranks(dist, t_e2e)
    e2e = {"value": units / t_e2e, "unit": "particle-steps/s", "h2d_bytes_per_step": 48 * n / K,
           "d2h_bytes_per_step": 48 * n / K,
           "note": "set_particles(pinned host x,p) + run(K) + get_particles(host) per job of K steps"}

    # plain fp64 path on the same workload
    fp64 = None
    if not args.no_fp64:
        cfg64 = pm.make_config(n, w["n_mesh"], w["box"], precision=pm.FP64, m22=w["m22"],
                               force_mode=pm.FORCE_HYBRID)
        del sim
        torch.cuda.empty_cache()
        s64 = pm.Sim(cfg64, stream=stream)
        s64.set_particles(x, p)
        K64 = max(2, min(K, 10))
        with torch.cuda.stream(stream):
            s64.run(1, a[0], a[1])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s64.run(K64, a[1], a[1 + K64])
            e1.record(stream)
            torch.cuda.synchronize()
        t64 = max_over_ranks(dist, e0.elapsed_time(e1))
        fp64 = {"value": sum_over_ranks(dist, n * K64) / (t64 / 1e3), "unit": "particle-steps/s",
                "steps": K64, "ms_per_step": t64 / K64}
        s64.close()

    # the same workload with the paper's cubic spline kernel (h = 3.5 dx): three more transforms per step
    spline = None
    if not args.no_spline:
        cfgs = pm.make_config(n, w["n_mesh"], w["box"], precision=pm.FP32, m22=w["m22"],
                              force_mode=pm.FORCE_HYBRID, kernel=pm.KERNEL_SPLINE, smooth_h=3.5, fft_jit=True)
        torch.cuda.empty_cache()
        ssp = pm.Sim(cfgs, stream=stream)
        ssp.set_particles(x, p)
        ssp.autotune(reps=3)
        with torch.cuda.stream(stream):
            ssp.run(W, a[0], a[W])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ssp.run(K, a[W], a[W + K])
            e1.record(stream)
            torch.cuda.synchronize()
        ts = max_over_ranks(dist, e0.elapsed_time(e1))
        spline = {"value": sum_over_ranks(dist, n * K) / (ts / 1e3), "unit": "particle-steps/s", "steps": K,
                  "ms_per_step": ts / K, "kernel": "cubic spline, h = 3.5 dx (Sec. II.A)"}
        ssp.close()

    batched = None
    if not args.no_batch:
        torch.cuda.empty_cache()
        batched = run_batched(pm, ics, K, W, stream)
        t_b = max_over_ranks(dist, batched["ms_per_step"])
        batched["value"] = sum_over_ranks(dist, batched["particles"] * K) / (t_b * K / 1e3)
    served = None
    if args.serve_requests > 0:
        from paper_1608_00802_gb300 import serve
        torch.cuda.empty_cache()
        served = run_served(serve, args.serve_requests)
    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        v, dt, sample = oracle_step_rate(w)
        cpu = {"value": v, "unit": "particle-steps/s", "cores": cpu_cores_used(), "kind": "oracle",
               "sample": sample, "seconds": dt}
    line = {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["name"], "precision": "fp32 cell+offset, fp32 mesh/FFT",
                       "force_mode": "hybrid (PM gravity + Q by the kernel gradient, Sec. II.A step iii)", "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (~0.5 GB touched per step), no flush"},
            "roofline": roofline, "step_roofline": step_roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches,
            "launch_shapes": tuning,
            "clocks": clk.summary(), "stages": per_stage, "fp64_plain": fp64, "spline_kernel": spline,
            "batched": batched, "served": served,
            "fp32_vs_fp64": (value / fp64["value"]) if fp64 else None}
    print(json.dumps(line))
    return 0


BATCH = dict(name="48 sims: 32^3/64^3/128^3 particles on 2x meshes (16 each), m22 in {1,2.5,5,10}, "
                   "seeds 0-47, L ~ U(1,4) Mpc/h, z=100->3 in 200 steps, fp32, hybrid force, graph-captured",
             nsims=48, sizes=(32, 64, 128), masses=(1.0, 2.5, 5.0, 10.0), nsteps=200, z_start=100.0, z_end=3.0)


def batch_members():
    """(n_side, n_mesh, box, m22, seed) of the 48-simulation batch: size class
    i mod 3, mass (i div 3) mod 4, box 1 + 3 U_i from Philox(0xB00), seed i."""
    u = np.random.Generator(np.random.Philox(0xB00)).uniform(size=BATCH["nsims"])
    out = []
    for i in range(BATCH["nsims"]):
        n = BATCH["sizes"][i % 3]
        out.append((n, 2 * n, 1.0 + 3.0 * float(u[i]), BATCH["masses"][(i // 3) % 4], i))
    return out


def run_batched(pm, ics, K, W, stream):
    import torch
    members = batch_members()
    a = schedule(dict(z_start=BATCH["z_start"], z_end=BATCH["z_end"], nsteps=BATCH["nsteps"]))
    cfgs = [pm.make_config(n ** 3, nm, box, precision=pm.FP32, m22=m22, force_mode=pm.FORCE_HYBRID, fft_jit=True)
            for n, nm, box, m22, _ in members]
    batch = pm.Batch(cfgs, stream=stream)
    cache = pm.TuningCache()  # one autotuner run per member size, shared by the others (untimed)
    for mem, (n, nm, box, m22, seed) in zip(batch.members, members):
        mem.set_particles(*ics.zeldovich(n, nm, box, a[0], seed, m22=m22))
        mem.autotune(reps=5, cache=cache)
    with torch.cuda.stream(stream):
        if W > 0:
            batch.run(W, a[0], a[W])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.run(K, a[W], a[W + K])
        e1.record(stream)
        torch.cuda.synchronize()
    t = e0.elapsed_time(e1)
    units = sum(n ** 3 for n, *_ in members) * K
    batch.close()
    return {"value": units / (t / 1e3), "unit": "particle-steps/s", "steps": K, "ms_per_step": t / K,
            "workload": BATCH["name"], "particles": sum(n ** 3 for n, *_ in members)}


SERVE = dict(name="Poisson arrivals 20 req/s, particles {32,64,128,192}^3 (weights .4/.3/.2/.1), mesh 2x, "
                   "m22 log-uniform 1-10, L ~ U(1,4), z=50->5 in 200 steps, fp32, hybrid force, HBM budget 64 GB",
             rate=20.0, budget=64 << 30, chunk=20)


def _initial_conditions(req):
    from paper_1608_00802_gb300 import serve
    return serve.initial_conditions(req)


def run_served(serve, n_requests):
    """Continuous batching on the request stream; initial conditions are made
    before the timed stream (in a spawned process pool), the rest is timed."""
    import multiprocessing as mp
    reqs = serve.request_stream(n_requests, rate=SERVE["rate"], seed=0)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        initial = dict(zip([r.rid for r in reqs], pool.map(_initial_conditions, reqs)))
    # launch shapes of each request size, measured before the stream (untimed)
    cache = serve.tune_sizes(sorted({(r.n_side, r.n_mesh) for r in reqs}))
    srv = serve.Server(SERVE["budget"], max_slots=64, chunk_steps=SERVE["chunk"], tuning=cache)
    res = srv.run(reqs, realtime=True, initial=initial)
    lat = serve.latency_percentiles(res)
    offered = SERVE["rate"] * float(np.mean([r.n_side ** 3 * r.nsteps for r in reqs]))
    return {"value": srv.stats["particle_steps"] / srv.stats["makespan"], "unit": "particle-steps/s",
            "p50_s": lat["p50"], "p99_s": lat["p99"], "requests": n_requests,
            "offered_particle_steps_per_s": offered, "makespan_s": srv.stats["makespan"],
            "max_active": srv.stats["max_active"], "peak_arena_gb": srv.stats["peak_bytes"] / 2 ** 30,
            "workload": SERVE["name"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-spline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=60)
    ap.add_argument("--tuning", default=None, help="launch shapes (pm_tuning fields as JSON) instead of the "
                    "autotuner's, for the single simulation")
    args = ap.parse_args()
    if args.warmup < 0 or args.steps < 1:
        raise SystemExit("steps >= 1, warmup >= 0")
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
