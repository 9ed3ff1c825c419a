"""Continuous batching of elastic-plastic contact solves on one GPU.

A request is one full solve (Algorithm 1 of the paper over a load ramp) of its own
problem: grid, depth nodes, material, surface and loads.  The server keeps a pool of
contexts (one CUDA stream each, plastic state resident on the device), admits a
waiting request as soon as a slot is free and its device footprint fits the HBM
budget, and runs the admitted solves concurrently from worker threads: the C ABI
releases the GIL, so kernels of different requests overlap on the device while each
request's host loop waits on its own stream.  Finished contexts go back to the pool
(state reset on the device) for the next request of the same shape.

Results are independent of the mix: every solve only touches its own context and its
reductions have a fixed order, so a request gives the same bits alone and in a mix.
"""
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import fvim


@dataclass
class Request:
    rid: int
    n: int
    z: np.ndarray
    h: np.ndarray            # surface [n, n]
    loads: list              # total loads of the increments
    precision: str = "fp32"
    E: float = 1.0
    nu: float = 0.3
    sigma_y: float = 0.05
    E_h: float = 0.1
    L: float = 1.0
    arrival: float = 0.0     # seconds after the start of the stream
    opts: dict = field(default_factory=dict)

    @property
    def shape(self):
        return (self.n, int(np.asarray(self.z).size), self.precision, np.asarray(self.z, dtype=np.float64).tobytes(),
                self.L)

    def footprint(self):
        return int(fvim.lib().fvim_footprint(self.n, self.n, int(np.asarray(self.z).size),
                                             0 if self.precision == "fp32" else 1))


@dataclass
class Result:
    rid: int
    pressure: np.ndarray
    report: dict
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self):
        return self.finished - self.arrival


class Admission:
    """Slots and HBM budget; admit(fp) blocks until both allow the request (FIFO)."""

    def __init__(self, slots, budget_bytes):
        self.slots = int(slots)
        self.budget = int(budget_bytes)
        self.active = 0
        self.used = 0
        self.cv = threading.Condition()
        self.next_ticket = 0
        self.serving = 0

    def admit(self, fp):
        if fp > self.budget:
            raise ValueError("request needs %d bytes, budget is %d" % (fp, self.budget))
        with self.cv:
            ticket = self.next_ticket
            self.next_ticket += 1
            while not (ticket == self.serving and self.active < self.slots and self.used + fp <= self.budget):
                self.cv.wait()
            self.active += 1
            self.used += fp
            self.serving += 1
            self.cv.notify_all()

    def release(self, fp):
        with self.cv:
            self.active -= 1
            self.used -= fp
            self.cv.notify_all()


class Server:
    def __init__(self, slots=4, hbm_budget=None):
        import torch

        self.torch = torch
        if hbm_budget is None:
            free, _total = torch.cuda.mem_get_info()
            hbm_budget = int(0.8 * free)
        self.adm = Admission(slots, hbm_budget)
        self.pool = {}
        self.pool_lock = threading.Lock()

    def _context(self, req):
        torch = self.torch
        with self.pool_lock:
            lst = self.pool.get(req.shape)
            if lst:
                ctx, stream = lst.pop()
                return ctx, stream
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            ctx = fvim.Context(req.n, req.n, req.z, req.L, req.L, precision=req.precision, E=req.E, nu=req.nu,
                               sigma_y=req.sigma_y, E_h=req.E_h)
        return ctx, stream

    def _recycle(self, req, ctx, stream):
        with self.pool_lock:
            self.pool.setdefault(req.shape, []).append((ctx, stream))

    def prepare(self, requests, autotune=True, reps=20):
        """Before serving: create one pooled context per distinct shape of `requests` and, with
        autotune, time the depth kernel's tile plans on it while nothing else runs on the
        device (fvim_autotune); later contexts of that grid start with the tuned plan, so
        every request of a shape runs the same kernels alone and in a mix.  Returns
        {shape index: plan}."""
        torch = self.torch
        plans = {}
        seen = set()
        for req in requests:
            if req.shape in seen:
                continue
            seen.add(req.shape)
            ctx, stream = self._context(req)
            with torch.cuda.stream(stream):
                if autotune and not ctx.plan["tuned"]:
                    ctx.autotune(reps)
            stream.synchronize()
            plans[len(plans)] = dict(ctx.plan, n=req.n, nz=int(np.asarray(req.z).size), precision=req.precision)
            self._recycle(req, ctx, stream)
        return plans

    def solve(self, req, t0=None):
        """Solve one request (admission included); returns a Result."""
        torch = self.torch
        t0 = time.perf_counter() if t0 is None else t0
        fp = req.footprint()
        self.adm.admit(fp)
        admitted = time.perf_counter() - t0
        try:
            ctx, stream = self._context(req)
            with torch.cuda.stream(stream):
                ctx.set_material(req.E, req.nu, req.sigma_y, req.E_h)
                ctx.reset_state()
                dt = ctx.dtype
                h = torch.from_numpy(np.ascontiguousarray(req.h)).to(device="cuda", dtype=dt, non_blocking=False)
                p = torch.empty(ctx.surf_shape, dtype=dt, device="cuda")
                opts = ctx.default_opts(**req.opts)
                rep = ctx.solve_contact(h, req.loads, p, opts, allow_not_converged=True)
                pressure = p.cpu().numpy()
            self._recycle(req, ctx, stream)
        finally:
            self.adm.release(fp)
        return Result(req.rid, pressure, rep, req.arrival, admitted, time.perf_counter() - t0)

    def run(self, requests):
        """Play a request stream in real time (arrival offsets in seconds); returns the
        results in request order and the wall time of the whole stream."""
        results = [None] * len(requests)
        t0 = time.perf_counter()
        threads = []

        def work(i, r):
            results[i] = self.solve(r, t0)

        for i, r in sorted(enumerate(requests), key=lambda ir: ir[1].arrival):
            delay = r.arrival - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            th = threading.Thread(target=work, args=(i, r))
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        return results, time.perf_counter() - t0


def percentiles(values, qs=(50, 99)):
    v = np.sort(np.asarray(values, dtype=np.float64))
    return {q: float(np.percentile(v, q)) for q in qs}


def poisson_arrivals(n, rate, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=n)) if rate > 0 and math.isfinite(rate) else np.zeros(n)
