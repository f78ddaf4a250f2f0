"""Scheduler logic of the continuous-batching server on the CPU: a fake engine
with the same interface runs a per-slot recurrence, so every request's result
can be checked against the same recurrence run alone."""
import time

import numpy as np
import pytest

from paper_2603_28150_gb300.serve import Geometry, Request, Server, poisson_arrivals


class FakeEngine:
    """Slot s holds state x; one step: x <- 0.5 x + (k + 1) y, k = the slot's own
    iteration count. Costs `per_step` seconds of host time per step."""
    created = []
    closed = []
    per_step = 0.0

    def __init__(self, geom, slots, priority=0):
        self.geom, self.slots, self.priority = geom, slots, priority
        self.x = np.zeros((slots, 4))
        self.y = np.zeros((slots, 4))
        self.k = np.zeros(slots, dtype=int)
        self.t0 = time.perf_counter()
        FakeEngine.created.append(geom.key)

    @staticmethod
    def estimate(geom, slots):
        return geom.n * 1000 + slots

    def set_origin(self, host_time):
        self.ref = time.perf_counter() - host_time

    def sync(self):
        pass

    def load(self, slot, req):
        self.x[slot] = 0
        self.y[slot] = req.y
        self.k[slot] = 0

    def move(self, dst, src):
        self.x[dst], self.y[dst], self.k[dst] = self.x[src], self.y[src], self.k[src]

    def step(self, n):
        if self.per_step:
            time.sleep(self.per_step)
        self.x[:n] = 0.5 * self.x[:n] + (self.k[:n, None] + 1) * self.y[:n]
        self.k[:n] += 1
        return time.perf_counter() - self.ref

    def read(self, slot, req):
        req.out = self.x[slot].copy()

    def ready(self, h):
        return True

    def time_of(self, h):
        return h

    def close(self):
        FakeEngine.closed.append(self.geom.key)


def alone(y, iters):
    x = np.zeros(4)
    for k in range(iters):
        x = 0.5 * x + (k + 1) * y
    return x


GA, GB, GC = Geometry(8, 2, 4, 16), Geometry(16, 2, 4, 32), Geometry(32, 2, 4, 64)


def _reqs(arrivals, keys, iters_choices=(3, 5, 8), seed=0):
    g = np.random.default_rng(seed)
    out = []
    for i, (t, key) in enumerate(zip(arrivals, keys)):
        out.append(Request(rid=i, key=key, y=g.normal(size=4), iters=int(g.choice(iters_choices)),
                           lam=0.0, arrival=t))
    return out


def test_every_result_equals_its_request_run_alone():
    FakeEngine.created, FakeEngine.closed = [], []
    arr = poisson_arrivals(400.0, 0.25, seed=1)
    keys = [(GA, GB, GC)[i % 3].key for i in range(len(arr))]
    reqs = _reqs(arr, keys)
    srv = Server([GA, GB, GC], budget_bytes=10 ** 9, slots=3, engine_factory=FakeEngine)
    rep = srv.run(reqs)
    assert rep["completed"] == len(reqs) and rep["unfinished"] == 0
    for r in reqs:
        assert np.allclose(r.out, alone(r.y, r.iters)), r.rid
        assert r.finish >= r.arrival
    assert rep["p99_ms"] >= rep["p50_ms"] >= 0


def test_slots_limit_and_fifo_within_a_geometry():
    FakeEngine.per_step = 0.0005
    reqs = _reqs([0.0] * 6, [GA.key] * 6, iters_choices=(4,))
    srv = Server([GA], budget_bytes=10 ** 9, slots=2, engine_factory=FakeEngine)
    srv.run(reqs)
    FakeEngine.per_step = 0.0
    adm = sorted(reqs, key=lambda r: r.admitted)
    assert [r.rid for r in adm] == list(range(6))  # arrival order
    assert srv.max_queue >= 4


def test_no_head_of_line_blocking_across_geometries():
    # GA has one slot and a long request; a later GB request must not wait for it
    reqs = [Request(0, GA.key, np.ones(4), 2000, 0.0, 0.0), Request(1, GA.key, np.ones(4), 3, 0.0, 0.0),
            Request(2, GB.key, np.ones(4), 3, 0.0, 0.0)]
    srv = Server([GA, GB], budget_bytes=10 ** 9, slots=1, engine_factory=FakeEngine)
    srv.run(reqs)
    assert reqs[2].finish < reqs[0].finish
    assert reqs[1].admitted >= reqs[0].finish - 1e-9 or reqs[1].admitted > reqs[2].admitted


def test_memory_budget_evicts_idle_engines_and_rejects_oversized():
    FakeEngine.created, FakeEngine.closed = [], []
    big = Geometry(10 ** 6, 1, 1, 16)  # estimate 1e9 > budget: never fits
    budget = FakeEngine.estimate(GC, 2) + 10   # one engine at a time
    reqs = [Request(0, GA.key, np.ones(4), 3, 0.0, 0.0), Request(1, GC.key, np.ones(4), 3, 0.0, 0.01),
            Request(2, big.key, np.ones(4), 3, 0.0, 0.02)]
    srv = Server([GA, GC, big], budget_bytes=budget, slots=2, engine_factory=FakeEngine)
    rep = srv.run(reqs)
    assert rep["completed"] == 2 and rep["rejected"] == 1
    assert FakeEngine.created == [GA.key, GC.key] and FakeEngine.closed == [GA.key]
    assert np.allclose(reqs[1].out, alone(np.ones(4), 3))


def test_poisson_arrivals_rate():
    a = poisson_arrivals(20.0, 60.0, seed=0)
    assert 1000 < len(a) < 1400 and all(np.diff(a) > 0)


def test_smaller_geometries_get_more_urgent_streams():
    class PrioEngine(FakeEngine):
        @staticmethod
        def priorities(ranks):
            return list(range(-ranks + 1, 1))   # most urgent (lowest) first

    big = Geometry(24, 2, 4, 48)
    srv = Server([big, GA, GC], budget_bytes=10 ** 9, slots=2, engine_factory=PrioEngine)
    order = sorted([big, GA, GC], key=lambda g: g.n)
    assert [srv.priority[g.key] for g in order] == [-2, -1, 0]
    eng = srv._engine_for(order[0].key)
    assert eng.priority == -2
    srv.close()
