"""Continuous-batching server for FISTA reconstruction requests.

Requests of several grid sizes arrive over time. Each geometry gets one
engine (a plan with `slots` request slots, its resident impulse-response
library, and its own CUDA stream) when its memory fits the budget. Between
steps the server admits waiting requests into free slots and retires finished
ones; each step advances every active slot of an engine by one FISTA
iteration in one batched launch sequence (pat_slots_step), so requests that
arrive while others run share the table stream and overlap on the device.

Latency is arrival (host clock) to the device event after the request's last
iteration; the result is copied to a per-request device buffer right after
that step.

The engine interface (`load`, `move`, `step`, `read`, `time_of`, `ready`,
`bytes`, `close`) lets a CPU stand-in drive the same scheduler in tests.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Geometry:
    """One served grid: n x n sensor/voxel grid (padded to pad), nz depths, nt samples."""
    n: int
    nz: int
    nt: int
    pad: int
    c: float = 1500.0
    dx: float = 50e-6
    dt: float = 10e-9
    mz: int = 0
    z0: int = 1

    @property
    def key(self):
        return (self.n, self.nz, self.nt)

    def depth_period(self) -> int:
        if self.mz:
            return self.mz
        need = self.z0 + self.nz + int(np.ceil(self.c * self.nt * self.dt / self.dx)) + 1
        m = 1
        while m < need:
            m *= 2
        return m


class QueueTrace:
    """Queue depth (requests arrived but not yet started) sampled at most every
    `every` seconds of the run; summarised as mean / max / last and a coarse
    timeline (max depth per `bucket` seconds)."""

    def __init__(self, every: float = 0.1, bucket: float = 5.0):
        self.every, self.bucket = every, bucket
        self.samples = []

    def sample(self, now: float, depth: int, active: int = 0) -> None:
        if not self.samples or now - self.samples[-1][0] >= self.every:
            self.samples.append((now, depth, active))

    def summary(self) -> dict:
        if not self.samples:
            return {"samples": 0}
        d = np.array([s[1] for s in self.samples], dtype=np.float64)
        a = np.array([s[2] for s in self.samples], dtype=np.float64)
        nb = int(self.samples[-1][0] // self.bucket) + 1
        line = [0] * nb
        for t, q, _ in self.samples:
            b = int(t // self.bucket)
            line[b] = max(line[b], q)
        return {"samples": len(self.samples), "mean": float(d.mean()), "max": int(d.max()),
                "last": int(d[-1]), "mean_active": float(a.mean()),
                f"max_per_{self.bucket:g}s": line}


@dataclass
class Request:
    rid: int
    key: tuple
    y: object          # data [nt][n][n] (device or host tensor)
    iters: int
    lam: float
    arrival: float     # seconds after the run start
    steps: int = 0
    slot: int = -1
    admitted: float | None = None
    finish: float | None = None
    out: object = None
    handle: object = None
    engine: object = None


class CudaEngine:
    """A plan with `slots` FISTA slots on its own stream (library generated on
    the device). `priority` is the CUDA stream priority (0 = default; lower
    values are scheduled first when several engines have work queued)."""

    def __init__(self, geom: Geometry, slots: int, power_iters: int = 50, force_complex=False,
                 priority: int = 0):
        import torch

        from .pat import Medium, Plan
        self.geom, self.slots = geom, slots
        self.stream = torch.cuda.Stream(priority=priority)
        with torch.cuda.stream(self.stream):
            med = Medium(geom.c, geom.dx, geom.dx, geom.dx, geom.dt, geom.depth_period(), geom.z0)
            self.plan = Plan(geom.n, geom.n, geom.nz, geom.nt, geom.pad, geom.pad,
                             max_batch=slots, medium=med, force_complex=force_complex,
                             bf16_split=self.tensor_ok(geom, slots) and not force_complex)
            v0 = torch.ones((geom.nz, geom.n, geom.n), dtype=torch.float32, device="cuda")
            self.L = 1.01 * self.plan.power_norm(v0, power_iters)
        self.ref = None
        self.kernels = 0

    @staticmethod
    def priorities(ranks: int):
        """Stream priorities for `ranks` engines, most urgent first: a short
        step of a small geometry then starts at the next kernel boundary of a
        large one instead of queueing behind its whole step."""
        import torch
        least, greatest = torch.cuda.Stream.priority_range()
        return [max(greatest, least - (ranks - 1 - r)) for r in range(ranks)]

    @staticmethod
    def tensor_ok(geom: Geometry, slots: int) -> bool:
        """Grids the split-BF16 tensor-core contraction takes (batched slots)."""
        return slots >= 2 and geom.nz == 128 and geom.nt % 128 == 0 and geom.nt <= 512

    @classmethod
    def estimate(cls, geom: Geometry, slots: int) -> int:
        from .pat import plan_estimate
        # the served libraries are k-space libraries of an isotropic grid:
        # D4-folded and radially shared
        tb, ws = plan_estimate(geom.n, geom.n, geom.nz, geom.nt, geom.pad, geom.pad, slots,
                               bf16_split=cls.tensor_ok(geom, slots), fold=True, radial=True)
        return tb + ws

    def bytes(self) -> int:
        inf = self.plan.info()
        return inf["table_bytes"] + inf["workspace_bytes"]

    def set_origin(self, host_time: float):
        """Records the stream's reference event; it stands for `host_time`
        (seconds after the run start). The stream must be idle."""
        import torch
        self.ref = torch.cuda.Event(enable_timing=True)
        self.ref_host = host_time
        self.ref.record(self.stream)

    def load(self, slot, req):
        self.plan.slot_load(slot, req.y, req.lam, self.L, stream=self.stream)

    def move(self, dst, src):
        self.plan.slot_move(dst, src, stream=self.stream)

    def step(self, n):
        import torch
        self.kernels += self.plan.slots_step(n, stream=self.stream)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(self.stream)
        return ev

    def read(self, slot, req):
        import torch
        if req.out is None:
            req.out = torch.empty((self.geom.nz, self.geom.n, self.geom.n), dtype=torch.float32,
                                  device="cuda")
        self.plan.slot_read(slot, out=req.out, stream=self.stream)

    def ready(self, handle) -> bool:
        return handle.query()

    def sync(self):
        self.stream.synchronize()

    def time_of(self, handle) -> float:
        handle.synchronize()
        return self.ref_host + self.ref.elapsed_time(handle) / 1e3

    def close(self):
        self.plan.close()


class Server:
    """Admission by memory, slot assignment, per-geometry batched steps."""

    def __init__(self, geometries, budget_bytes: int, slots, engine_factory=CudaEngine,
                 max_inflight: int = 2):
        self.geoms = {g.key: g for g in geometries}
        self.budget = budget_bytes
        self.slots = slots if isinstance(slots, dict) else {k: slots for k in self.geoms}
        self.factory = engine_factory
        # smaller geometries (shorter steps) get the more urgent streams
        order = sorted(self.geoms, key=lambda k: engine_factory.estimate(self.geoms[k],
                                                                         self.slots[k]))
        prio = engine_factory.priorities(len(order)) if hasattr(engine_factory, "priorities") \
            else [0] * len(order)
        self.priority = {k: prio[i] for i, k in enumerate(order)}
        self.max_inflight = max_inflight
        self.engines = {}
        self.active = collections.defaultdict(list)     # key -> requests in slot order
        self.inflight = collections.defaultdict(collections.deque)
        self.queue = collections.deque()
        self.done, self.rejected = [], []
        self.used = 0
        self.max_queue = 0
        self.trace = QueueTrace()
        self.t0 = None

    # -------------------------------------------------------------- admission
    def _engine_for(self, key):
        eng = self.engines.get(key)
        if eng is not None:
            return eng
        need = self.factory.estimate(self.geoms[key], self.slots[key])
        if need > self.budget:
            return "never"
        if self.used + need > self.budget:
            self._evict_idle(need)
        if self.used + need > self.budget:
            return None
        eng = self.factory(self.geoms[key], self.slots[key], priority=self.priority[key])
        if self.t0 is not None:
            eng.set_origin(self.now())
        self.engines[key] = eng
        self.used += need
        return eng

    def _evict_idle(self, need):
        waiting = {r.key for r in self.queue}
        for key in list(self.engines):
            if self.used + need <= self.budget:
                break
            if not self.active[key] and key not in waiting:
                eng = self.engines[key]
                q = self.inflight[key]
                while q:  # its last steps must finish before its memory goes
                    eng.time_of(q.popleft())
                del self.engines[key]
                self.used -= self.factory.estimate(self.geoms[key], self.slots[key])
                eng.close()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def admit(self):
        """Fills free slots from the queue in arrival order; a request whose
        geometry has no free slot does not block requests of other geometries."""
        keep = collections.deque()
        while self.queue:
            req = self.queue.popleft()
            eng = self._engine_for(req.key)
            if eng == "never":
                self.rejected.append(req)
                continue
            act = self.active[req.key]
            if eng is None or len(act) >= self.slots[req.key]:
                keep.append(req)
                continue
            req.slot = len(act)
            req.admitted = self.now()
            eng.load(req.slot, req)
            act.append(req)
        self.queue = keep

    # -------------------------------------------------------------- stepping
    def step_all(self) -> bool:
        stepped = False
        for key, act in self.active.items():
            if not act:
                continue
            eng = self.engines[key]
            q = self.inflight[key]
            while q and eng.ready(q[0]):
                q.popleft()
            if len(q) >= self.max_inflight:
                # this engine is a few steps ahead of its GPU work: leave it and
                # serve the others instead of waiting on it
                continue
            h = eng.step(len(act))
            q.append(h)
            stepped = True
            finished = []
            for r in act:
                r.steps += 1
                if r.steps >= r.iters:
                    finished.append(r)
            for r in finished:
                r.handle, r.engine = h, eng
                eng.read(r.slot, r)
            for r in sorted(finished, key=lambda r: -r.slot):   # retire from the end down
                last = len(act) - 1
                if r.slot != last:
                    mover = act[last]
                    eng.move(r.slot, last)
                    mover.slot = r.slot
                    act[r.slot] = mover
                act.pop()
                self.done.append(r)
        return stepped

    # -------------------------------------------------------------- run
    def run(self, requests, drain_seconds: float = 60.0, idle_sleep: float = 0.0005):
        """Real-time replay of `requests` (arrival times in seconds from start)."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        for eng in self.engines.values():
            eng.sync()
        self.t0 = time.perf_counter()
        for eng in self.engines.values():
            eng.set_origin(0.0)
        last_arrival = pending[-1].arrival if pending else 0.0
        while pending or self.queue or any(self.active.values()):
            now = self.now()
            while pending and pending[0].arrival <= now:
                self.queue.append(pending.popleft())
            self.max_queue = max(self.max_queue, len(self.queue))
            self.admit()
            self.trace.sample(now, len(self.queue), sum(len(a) for a in self.active.values()))
            if not self.step_all():
                # nothing could step (idle, or every engine's queue is full)
                wait = idle_sleep
                if pending and not any(self.active.values()):
                    wait = min(idle_sleep, max(0.0, pending[0].arrival - self.now()))
                time.sleep(wait)
            if now > last_arrival + drain_seconds:
                break
        for key, q in self.inflight.items():
            while q:
                self.engines[key].time_of(q.popleft())
        for r in self.done:
            r.finish = r.engine.time_of(r.handle)
        return self.report(requests)

    def report(self, requests):
        lat = np.array([r.finish - r.arrival for r in self.done if r.finish is not None])
        unfinished = [r for r in requests if r.finish is None and r not in self.rejected]
        end = self.now()
        out = {"requests": len(requests), "completed": int(lat.size),
               "unfinished": len(unfinished), "rejected": len(self.rejected),
               "max_queue": self.max_queue, "queue_depth": self.trace.summary()}
        if lat.size:
            out["p50_ms"] = float(np.percentile(lat, 50) * 1e3)
            out["p99_ms"] = float(np.percentile(lat, 99) * 1e3)
            span = max(r.finish for r in self.done if r.finish is not None) - min(
                r.arrival for r in requests)
            out["req_per_s"] = lat.size / span if span > 0 else None
        if unfinished:
            # censored: their latency is at least end - arrival
            cens = np.array([end - r.arrival for r in unfinished])
            allv = np.concatenate([lat, cens]) if lat.size else cens
            out["p99_ms_lower_bound"] = float(np.percentile(allv, 99) * 1e3)
        per = collections.defaultdict(list)
        for r in self.done:
            if r.finish is not None:
                per[r.key].append(r.finish - r.arrival)
        out["per_geometry"] = {f"{k[0]}x{k[0]}x{k[1]}x{k[2]}": {
            "completed": len(v), "p50_ms": float(np.percentile(v, 50) * 1e3),
            "p99_ms": float(np.percentile(v, 99) * 1e3)} for k, v in per.items()}
        return out

    def close(self):
        for eng in self.engines.values():
            eng.close()
        self.engines.clear()


def serve_one_at_a_time(plans, requests, drain_seconds: float = 60.0):
    """The plain path the batched server is compared with: requests in arrival
    order, one pat_fista_solve each (batch 1) on the geometry's plan, one stream."""
    import torch
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    stream = torch.cuda.current_stream()
    ref = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ref.record(stream)
    last_arrival = pending[-1].arrival if pending else 0.0
    inflight = collections.deque()
    done = []
    trace = QueueTrace()
    while pending:
        now = time.perf_counter() - t0
        if now > last_arrival + drain_seconds:
            break
        # arrived but not yet started (the request being issued counts as started)
        arrived = 0
        for q in pending:          # sorted by arrival
            if q.arrival > now:
                break
            arrived += 1
        trace.sample(now, max(0, arrived - 1) if arrived else 0, 1 if inflight else 0)
        r = pending[0]
        if r.arrival > now and not inflight:
            time.sleep(min(0.0005, r.arrival - now))
            continue
        if r.arrival > now:
            inflight.popleft().synchronize()
            continue
        pending.popleft()
        plan, L = plans[r.key]
        x = torch.empty((plan.nz, plan.ny, plan.nx), dtype=torch.float32, device="cuda")
        plan.fista(r.y, x=x, iters=r.iters, lam=r.lam, L=L)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        r.handle, r.out = ev, x
        inflight.append(ev)
        while len(inflight) > 2:
            inflight.popleft().synchronize()
        done.append(r)
    torch.cuda.synchronize()
    end = time.perf_counter() - t0
    for r in done:
        r.finish = ref.elapsed_time(r.handle) / 1e3
    lat = np.array([r.finish - r.arrival for r in done])
    unfinished = [r for r in requests if r.finish is None]
    out = {"requests": len(requests), "completed": int(lat.size), "unfinished": len(unfinished),
           "queue_depth": trace.summary()}
    if lat.size:
        out["p50_ms"] = float(np.percentile(lat, 50) * 1e3)
        out["p99_ms"] = float(np.percentile(lat, 99) * 1e3)
        span = max(r.finish for r in done) - min(r.arrival for r in requests)
        out["req_per_s"] = lat.size / span if span > 0 else None
    if unfinished:
        cens = np.array([end - r.arrival for r in unfinished])
        allv = np.concatenate([lat, cens]) if lat.size else cens
        out["p99_ms_lower_bound"] = float(np.percentile(allv, 99) * 1e3)
    return out


def poisson_arrivals(rate: float, seconds: float, seed: int = 0):
    """Arrival times of a Poisson process of `rate` per second over `seconds`."""
    g = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate)
        if t >= seconds:
            return out
        out.append(t)
