"""Continuous-batching request loop for projection solves on one GPU.

Requests (a grid, a precision, a seed, an arrival time) are admitted in
arrival order as soon as a slot (a CUDA stream) and enough of the device-memory
budget are free; admitted work runs concurrently on the slot streams, so
requests that arrive while others are on the GPU overlap with them.  Plans
(workspace, twiddles, tables) stay resident per size class and are reused;
idle plans are evicted, least recently used first, when the budget needs the
room.  Each request's fields live in device memory for its lifetime.  The loop
reports throughput and arrival-to-completion latency percentiles.

The device side sits behind a small executor interface (prepare / launch /
poll / release) so that the admission logic can be exercised without a GPU.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np

FIELD_COUNT_IO = 11  # 7 inputs + p, u, v, w outputs (FP64)


@dataclasses.dataclass
class Request:
    rid: int
    shape: tuple          # (nx, ny, nz)
    precision: int        # ppe.FP64 or ppe.FP32_REFINE
    seed: int
    arrival: float        # seconds after the start of the run
    admitted: float = math.nan
    done: float = math.nan
    sweeps: int = -1
    rel_residual: float = math.nan


def poisson_requests(count: int, rate: float, shapes, probs=None, fp32_share: float = 0.5, seed: int = 0,
                     fp64=0, fp32=1):
    """`count` requests with exponential inter-arrival times (mean 1/rate),
    shapes drawn from `shapes` (weights `probs`), precision FP32_REFINE with
    probability fp32_share."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    idx = rng.choice(len(shapes), size=count, p=probs)
    prec = rng.random(count) < fp32_share
    return [Request(i, tuple(shapes[idx[i]]), fp32 if prec[i] else fp64, 1000 + i, float(t[i]))
            for i in range(count)]


@dataclasses.dataclass
class Stats:
    completed: int
    wall_s: float
    solves_per_s: float
    latency_ms_p50: float
    latency_ms_p99: float
    wait_ms_p50: float
    wait_ms_p99: float
    peak_bytes: int
    max_active: int
    plans_created: int
    evictions: int
    rejected: int

    def as_dict(self):
        return dataclasses.asdict(self)


class Server:
    """FIFO continuous batching under a device-memory budget."""

    def __init__(self, executor, budget_bytes: int, slots: int = 8):
        self.ex = executor
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.idle = collections.OrderedDict()  # plan key -> list of idle plans (LRU order)
        self.plan_bytes = 0                    # resident plan workspace
        self.live_bytes = 0                    # fields of admitted requests
        self.plans_created = 0
        self.evictions = 0

    # -- memory -----------------------------------------------------------------
    def _in_use(self):
        return self.plan_bytes + self.live_bytes

    def _evict_for(self, need: int) -> bool:
        while self._in_use() + need > self.budget and self.idle:
            key, plans = next(iter(self.idle.items()))
            plan = plans.pop()
            if not plans:
                del self.idle[key]
            self.plan_bytes -= self.ex.plan_bytes(plan)
            self.ex.destroy_plan(plan)
            self.evictions += 1
        return self._in_use() + need <= self.budget

    def _take_plan(self, req):
        key = (req.shape, req.precision)
        plans = self.idle.get(key)
        if plans:
            plan = plans.pop()
            if not plans:
                del self.idle[key]
            return plan, 0
        return None, self.ex.plan_bytes_for(req.shape, req.precision)

    def reserve(self, classes, per_class: int = 2) -> int:
        """Create idle plans ahead of traffic, so that each (shape, precision)
        class holds at least `per_class` resident plans and no request waits
        for a plan to be built (allocation and graph capture take tens of ms
        for the large grids).  Stops at the memory budget; returns the number
        of plans created."""
        made = 0
        for shape, precision in classes:
            key = (shape, precision)
            while len(self.idle.get(key, [])) < per_class:
                need = self.ex.plan_bytes_for(shape, precision)
                if self._in_use() + need > self.budget:
                    return made
                plan = self.ex.create_plan(shape, precision)
                self.plans_created += 1
                self.plan_bytes += need
                self.idle.setdefault(key, []).append(plan)
                made += 1
        return made

    def _return_plan(self, req, plan):
        key = (req.shape, req.precision)
        self.idle.setdefault(key, []).append(plan)
        self.idle.move_to_end(key)

    # -- loop -------------------------------------------------------------------
    def run(self, requests, clock=time.perf_counter, sleep=time.sleep, keep=()):
        """Serve `requests` (sorted by arrival); returns (Stats, {rid: result})."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        active = []      # (request, handle, plan, field bytes)
        free_slots = list(range(self.slots))
        results = {}
        rejected = []
        peak = 0
        max_active = 0
        t0 = clock()
        done = []
        while pending or active:
            now = clock() - t0
            # completions
            still = []
            for req, h, plan, nbytes, slot in active:
                if self.ex.poll(h):
                    req.done = clock() - t0
                    req.sweeps, req.rel_residual = self.ex.info(h)
                    if req.rid in keep:
                        results[req.rid] = self.ex.result(h)
                    self.ex.release(h)
                    self.live_bytes -= nbytes
                    self._return_plan(req, plan)
                    free_slots.append(slot)
                    done.append(req)
                else:
                    still.append((req, h, plan, nbytes, slot))
            active = still
            # admissions, in arrival order (the head blocks those behind it);
            # a request that cannot fit even into an empty budget is rejected
            while pending and free_slots and pending[0].arrival <= now:
                req = pending[0]
                if self.ex.plan_bytes_for(req.shape, req.precision) + self.ex.field_bytes(req.shape) > self.budget:
                    pending.popleft()
                    rejected.append(req)
                    continue
                plan, plan_need = self._take_plan(req)
                need = plan_need + self.ex.field_bytes(req.shape)
                if not self._evict_for(need):
                    if plan is not None:
                        self._return_plan(req, plan)
                    break
                pending.popleft()
                if plan is None:
                    plan = self.ex.create_plan(req.shape, req.precision)
                    self.plans_created += 1
                    self.plan_bytes += plan_need
                slot = free_slots.pop()
                nbytes = self.ex.field_bytes(req.shape)
                self.live_bytes += nbytes
                req.admitted = clock() - t0
                h = self.ex.launch(req, plan, slot)
                active.append((req, h, plan, nbytes, slot))
            peak = max(peak, self._in_use())
            max_active = max(max_active, len(active))
            if not active and pending:
                wait = pending[0].arrival - (clock() - t0)
                if wait > 0:
                    sleep(min(wait, 0.01))
        wall = max((r.done for r in done), default=0.0)
        lat = np.array([1e3 * (r.done - r.arrival) for r in done])
        wt = np.array([1e3 * (r.admitted - r.arrival) for r in done])
        span = wall - min((r.arrival for r in done), default=0.0)
        stats = Stats(len(done), wall, len(done) / span if span > 0 else math.nan,
                      float(np.percentile(lat, 50)) if len(lat) else math.nan,
                      float(np.percentile(lat, 99)) if len(lat) else math.nan,
                      float(np.percentile(wt, 50)) if len(wt) else math.nan,
                      float(np.percentile(wt, 99)) if len(wt) else math.nan,
                      int(peak), int(max_active), self.plans_created, self.evictions, len(rejected))
        return stats, results

    def close(self):
        for plans in self.idle.values():
            for p in plans:
                self.ex.destroy_plan(p)
        self.idle.clear()
        self.plan_bytes = 0


class CudaExecutor:
    """libppe on one GPU: slot streams, ppe_project on the slot's stream,
    completion events.

    Inputs: every request projects its own seeded fields (the single-interface
    recipe of fields.make_fields).  Generating a large grid's fields on the host
    takes seconds, so they are drawn ahead of the traffic into a resident pool
    of `pool` distinct seeded sets per shape: request seed s uses set s mod pool
    (field seed field_seed(shape, s mod pool)).  Each slot keeps one set of
    field buffers (seven inputs, four outputs) per shape it has served, and a
    request copies its set into them device to device instead of allocating (an
    allocation can synchronise the whole device); `prealloc` creates the
    buffers and `prepare` the pool up front."""

    def __init__(self, slots: int = 8, device=None, pool: int = 4, inputs=None, autotune_cache=None):
        import torch

        from . import fields as F
        from . import ppe
        self.torch, self.ppe, self.F = torch, ppe, F
        self.dev = torch.device("cuda", device if device is not None else torch.cuda.current_device())
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(slots)]
        self.pool = max(1, int(pool))
        self.inputs = inputs if inputs is not None else {}  # (shape, k) -> (device arrays, host Fields)
        self.autotune_cache = autotune_cache
        self.buffers = {}  # (slot, shape) -> (inputs, outputs)

    @staticmethod
    def field_seed(shape, k):
        """Seed of pool set k of a shape (distinct across shapes and sets)."""
        nx, ny, nz = shape
        return 100003 * k + 7 * nx + 3 * ny + nz

    def fields_of(self, shape, seed):
        """(device arrays, host Fields) of the set a request with this seed projects."""
        k = int(seed) % self.pool
        t = self.inputs.get((shape, k))
        if t is None:
            nx, ny, nz = shape
            fl = self.F.make_fields(nx, ny, nz, seed=self.field_seed(shape, k), recipe="single", width=2.0)
            t = ({n: self.torch.from_numpy(v).to(self.dev) for n, v in fl.arrays().items()}, fl)
            self.inputs[(shape, k)] = t
        return t

    def prepare(self, shapes):
        """Draw every pool set of these shapes (before the clock starts)."""
        for shape in shapes:
            for k in range(self.pool):
                self.fields_of(shape, k)
        self.torch.cuda.synchronize(self.dev)

    def _bufs(self, slot, shape):
        b = self.buffers.get((slot, shape))
        if b is None:
            torch = self.torch
            tmpl, _ = self.fields_of(shape, 0)
            with torch.cuda.stream(self.streams[slot]):
                d = {k: torch.empty_like(v) for k, v in tmpl.items()}
                out = dict(p=torch.empty_like(d["rho"]), u=torch.empty_like(d["u"]), v=torch.empty_like(d["v"]),
                           w=torch.empty_like(d["w"]))
            b = self.buffers[(slot, shape)] = (d, out)
        return b

    def prealloc(self, shapes):
        for slot in range(len(self.streams)):
            for shape in shapes:
                self._bufs(slot, shape)
        self.torch.cuda.synchronize(self.dev)

    def field_bytes(self, shape):
        nx, ny, nz = shape
        return 8 * (FIELD_COUNT_IO * nx * ny * nz + 2 * nx * nz)  # v has one more plane (in and out)

    def plan_bytes_for(self, shape, precision):
        import ctypes
        nx, ny, nz = shape
        g = self.ppe.Grid(nx, ny, nz, 1.0, 1.0, 1.0)
        o = self.ppe.Options(precision, 0, 1e-10, 8, 1e-12)
        return int(self.ppe.lib().ppe_workspace_bytes(ctypes.byref(g), ctypes.byref(o)))

    def plan_bytes(self, plan):
        return plan.workspace_bytes()

    def create_plan(self, shape, precision):
        nx, ny, nz = shape
        _, fl = self.fields_of(shape, 0)  # the box lengths (the same for every set of a shape)
        plan = self.ppe.Plan(nx, ny, nz, fl.lx, fl.ly, fl.lz, precision=precision, refine_tol=1e-10, max_sweeps=8,
                             stream=self.streams[0])
        if self.autotune_cache:
            from . import autotune
            autotune.apply_cached(plan, self.autotune_cache)
        return plan

    def destroy_plan(self, plan):
        plan.close()

    def launch(self, req, plan, slot):
        torch = self.torch
        s = self.streams[slot]
        src, fl = self.fields_of(req.shape, req.seed)
        d, out = self._bufs(slot, req.shape)
        with torch.cuda.stream(s):
            for k, v in src.items():  # this request's fields, in the slot's buffers
                d[k].copy_(v, non_blocking=True)
        plan.set_stream(s)
        plan.project(d["u"], d["v"], d["w"], d["S"], d["rho"], d["p_n"], d["p_nm1"], fl.dt, out["p"], out["u"],
                     out["v"], out["w"])
        ev = torch.cuda.Event()
        ev.record(s)
        return {"ev": ev, "d": d, "out": out, "plan": plan}

    def poll(self, h):
        return h["ev"].query()

    def info(self, h):
        inf = h["plan"].info(allow_not_converged=True)
        return inf.sweeps, inf.rel_residual

    def result(self, h):
        return {k: v.cpu().numpy() for k, v in h["out"].items()}

    def release(self, h):
        h["d"] = h["out"] = None  # the slot's buffers are reused by its next request


class FakeExecutor:
    """Executor without a GPU for testing the loop: each launch finishes a fixed
    (or shape-dependent) time later on a virtual clock."""

    def __init__(self, duration, clock):
        self.duration = duration
        self.clock = clock
        self.created = 0
        self.live = set()

    def field_bytes(self, shape):
        return 8 * FIELD_COUNT_IO * shape[0] * shape[1] * shape[2]

    def plan_bytes_for(self, shape, precision):
        return 4 * shape[0] * shape[1] * shape[2]

    def plan_bytes(self, plan):
        return plan["bytes"]

    def create_plan(self, shape, precision):
        self.created += 1
        return {"bytes": self.plan_bytes_for(shape, precision), "shape": shape, "busy": False}

    def destroy_plan(self, plan):
        assert not plan["busy"]

    def launch(self, req, plan, slot):
        assert not plan["busy"], "a plan is never shared by two requests in flight"
        plan["busy"] = True
        self.live.add(req.rid)
        return {"req": req, "plan": plan, "end": self.clock() + self.duration(req)}

    def poll(self, h):
        return self.clock() >= h["end"]

    def info(self, h):
        return 1, 1e-13

    def result(self, h):
        return {"rid": h["req"].rid}

    def release(self, h):
        h["plan"]["busy"] = False
        self.live.discard(h["req"].rid)
