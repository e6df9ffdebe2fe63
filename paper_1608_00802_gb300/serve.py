"""Continuous-batching request loop for many independent simulations.

Requests (axion mass, seed, box, particle and mesh size, redshift range) arrive
over time.  The server admits a waiting request as soon as its device arena
fits in the HBM budget and a slot is free, keeps every admitted simulation's
particle and mesh state resident on the device, and advances all admitted
simulations together in chunks of leapfrog steps, each on its own CUDA stream
so that their kernels overlap on the GPU.  Between chunks it retires finished
simulations (result = final energies and power spectrum), frees their arenas
and admits newcomers: requests that arrive while others run join the mix at
the next chunk boundary.  A simulation's result does not depend on what else
runs beside it (its kernels only touch its own arena and are deterministic).
"""
from __future__ import annotations

import math
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

from . import ics, pm


@dataclass
class Request:
    rid: int
    n_side: int
    n_mesh: int
    box: float
    m22: float
    seed: int
    z_start: float = 50.0
    z_end: float = 5.0
    nsteps: int = 200
    arrival: float = 0.0          # seconds after the start of the stream
    force_mode: int = pm.FORCE_HYBRID

    def config(self):
        return pm.make_config(self.n_side ** 3, self.n_mesh, self.box, precision=pm.FP32, m22=self.m22,
                              force_mode=self.force_mode)

    @property
    def a_start(self):
        return 1.0 / (1.0 + self.z_start)

    @property
    def a_end(self):
        return 1.0 / (1.0 + self.z_end)


@dataclass
class Result:
    rid: int
    energy: np.ndarray
    k: np.ndarray
    pk: np.ndarray
    x: np.ndarray | None
    p: np.ndarray | None
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self):
        return self.finished - self.arrival


@dataclass
class _Active:
    req: Request
    sim: pm.Sim
    stream: object
    done_steps: int = 0
    admitted: float = 0.0
    event: object = None


def request_stream(n_requests, rate=20.0, seed=0, sizes=(32, 64, 128, 192), weights=(0.4, 0.3, 0.2, 0.1),
                   m22_range=(1.0, 10.0), box_range=(1.0, 4.0), z_start=50.0, z_end=5.0, nsteps=200):
    """Poisson arrivals (mean `rate` per second) of requests with particles per
    side drawn from `sizes` with `weights`, mesh 2x particles per side, m22
    log-uniform in `m22_range`, box uniform in `box_range`, seed = index."""
    rng = np.random.Generator(np.random.Philox(seed))
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate)
        n = int(rng.choice(sizes, p=np.asarray(weights) / np.sum(weights)))
        m22 = float(math.exp(rng.uniform(math.log(m22_range[0]), math.log(m22_range[1]))))
        box = float(rng.uniform(*box_range))
        out.append(Request(i, n, 2 * n, box, m22, i, z_start, z_end, nsteps, t))
    return out


class Server:
    """Admits requests under an HBM budget and steps the admitted simulations
    together; `run` returns one Result per request."""

    def __init__(self, hbm_budget_bytes, max_slots=64, chunk_steps=20, keep_particles=False, device="cuda",
                 admit_threads=4, tuning=None):
        import torch
        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.max_slots = int(max_slots)
        self.chunk = int(chunk_steps)
        self.keep_particles = keep_particles
        dev = torch.device(device)
        self.device = dev if dev.index is not None else torch.device("cuda", torch.cuda.current_device())
        self.in_use = 0
        # admissions (arena, plans, upload and first sort) run on worker threads so that the
        # loop keeps feeding the running simulations meanwhile
        self.admit_threads = int(admit_threads)
        # launch shapes by configuration (a pm.TuningCache): a size not yet in it is measured
        # by the autotuner on its first admission
        self.tuning = tuning
        self.stats = {"admitted": 0, "max_active": 0, "chunks": 0, "particle_steps": 0, "peak_bytes": 0}

    def _bytes(self, req):
        return pm.arena_bytes(req.config())

    def _admit(self, req, now, initial=None):
        torch = self.torch
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(device=self.device)
        sim = pm.Sim(req.config(), device=self.device, stream=stream)
        x, p = initial if initial is not None else initial_conditions(req)
        sim.set_particles(x, p)
        if self.tuning is not None:
            sim.autotune(cache=self.tuning)
        act = _Active(req, sim, stream, admitted=now)
        return act

    def _schedule(self, req, k0, k1):
        """a at step k of the request's ln-a-uniform schedule."""
        a0, a1 = req.a_start, req.a_end

        def a(k):
            return a1 if k == req.nsteps else a0 * (a1 / a0) ** (k / req.nsteps)
        return a(k0), a(k1)

    def run(self, requests, realtime=True, initial=None):
        """Serves `requests` (their `arrival` times relative to now when
        `realtime`, else all at once).  `initial` may map rid -> (x, p) initial
        conditions prepared in advance (else they are generated at admission).
        Returns results ordered by rid."""
        torch = self.torch
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        sizes = {r.rid: self._bytes(r) for r in pending}
        for r in pending:
            if sizes[r.rid] > self.budget:
                raise ValueError("request %d needs %d bytes, more than the budget" % (r.rid, sizes[r.rid]))
        waiting = []            # arrived, not admitted (FIFO)
        admitting = []          # admissions in flight on the worker threads
        active = []
        pool = ThreadPoolExecutor(max(1, self.admit_threads))
        results = {}
        t0 = time.perf_counter()
        i = 0

        def now():
            return time.perf_counter() - t0

        while i < len(pending) or waiting or admitting or active:
            t = now()
            while i < len(pending) and (not realtime or pending[i].arrival <= t):
                waiting.append(pending[i])
                i += 1
            # admission: FIFO while memory and slots allow
            while (waiting and len(active) + len(admitting) < self.max_slots
                   and self.in_use + sizes[waiting[0].rid] <= self.budget):
                req = waiting.pop(0)
                self.in_use += sizes[req.rid]
                admitting.append(pool.submit(self._admit, req, now(),
                                             None if initial is None else initial.get(req.rid)))
                self.stats["admitted"] += 1
            ready = [f for f in admitting if f.done()]
            admitting = [f for f in admitting if not f.done()]
            active.extend(f.result() for f in ready)
            self.stats["peak_bytes"] = max(self.stats["peak_bytes"], self.in_use)
            self.stats["max_active"] = max(self.stats["max_active"], len(active))
            if not active:
                if admitting:
                    time.sleep(0.0005)
                    continue
                if i < len(pending):
                    time.sleep(max(0.0, min(0.01, pending[i].arrival - now())))
                continue
            # every simulation whose last chunk has finished gets its next chunk (on
            # its own stream) or is retired; the others keep running meanwhile
            progressed = False
            still = []
            for act in active:
                if act.event is not None and not act.event.query():
                    still.append(act)
                    continue
                progressed = True
                if act.done_steps < act.req.nsteps:
                    k1 = min(act.req.nsteps, act.done_steps + self.chunk)
                    a0, a1 = self._schedule(act.req, act.done_steps, k1)
                    act.sim.run(k1 - act.done_steps, a0, a1)
                    self.stats["particle_steps"] += act.req.n_side ** 3 * (k1 - act.done_steps)
                    self.stats["chunks"] += 1
                    act.done_steps = k1
                    act.event = torch.cuda.Event()
                    act.event.record(act.stream)
                    still.append(act)
                    continue
                e = act.sim.energy(act.req.a_end)
                k, pk, _ = act.sim.power_spectrum()
                x = p = None
                if self.keep_particles:
                    x, p = act.sim.get_particles()
                results[act.req.rid] = Result(act.req.rid, e, k, pk, x, p, act.req.arrival if realtime else 0.0,
                                              act.admitted, now())
                act.sim.close()
                del act.sim
                self.in_use -= sizes[act.req.rid]
            active = still
            if not progressed:
                time.sleep(0.0002)
        pool.shutdown()
        self.stats["makespan"] = now()
        return [results[r.rid] for r in sorted(requests, key=lambda r: r.rid)]


def tune_sizes(sizes, cache=None, m22=2.5, box=2.0):
    """Autotuner results for (particles per side, mesh) pairs of the request
    mix, measured on one sample simulation each; returns the cache."""
    cache = pm.TuningCache() if cache is None else cache
    for n_side, n_mesh in sizes:
        req = Request(-1, n_side, n_mesh, box, m22, 0)
        sim = pm.Sim(req.config())
        sim.set_particles(*initial_conditions(req))
        sim.autotune(cache=cache)
        sim.close()
    return cache


def initial_conditions(req):
    return ics.zeldovich(req.n_side, req.n_mesh, req.box, req.a_start, req.seed, m22=req.m22)


def run_alone(req, chunk_steps=10):
    """The same request on a simulation of its own (no server, default stream),
    in the same chunks of steps: (energy, k, P, x, p)."""
    sim = pm.Sim(req.config())
    sim.set_particles(*initial_conditions(req))
    a0, a1 = req.a_start, req.a_end

    def a(k):
        return a1 if k == req.nsteps else a0 * (a1 / a0) ** (k / req.nsteps)
    k = 0
    while k < req.nsteps:
        k1 = min(req.nsteps, k + chunk_steps)
        sim.run(k1 - k, a(k), a(k1))
        k = k1
    e = sim.energy(a1)
    kk, pk, _ = sim.power_spectrum()
    x, p = sim.get_particles()
    sim.close()
    return e, kk, pk, x, p


def latency_percentiles(results, qs=(50, 99)):
    lat = np.array([r.latency for r in results])
    return {("p%d" % q): float(np.percentile(lat, q)) for q in qs}
