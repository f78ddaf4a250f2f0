"""Continuous batching on the GPU: requests that share a plan's slots, enter at
different times and leave in a different order give the same reconstruction
as each request solved alone (pat_fista_solve, batch 1)."""
import numpy as np
import pytest

from paper_2603_28150_gb300 import Medium, Plan, synth
from paper_2603_28150_gb300.serve import (CudaEngine, Geometry, Request, Server,
                                          poisson_arrivals, serve_one_at_a_time)

pytestmark = pytest.mark.gpu

MED = Medium(1500.0, 50e-6, 50e-6, 50e-6, 10e-9, 64, 1)


def _data(plan, seed):
    import torch
    p0 = torch.tensor(synth.vessel_phantom(plan.nx, plan.nz, seed=seed), dtype=torch.float32,
                      device="cuda")
    d = plan.forward(p0)
    noise = torch.tensor(synth.gaussian_field(tuple(d.shape), seed + 500), dtype=torch.float32,
                         device="cuda")
    return (d + 0.05 * d.pow(2).mean().sqrt() * noise).contiguous()


def _alone(plan, y, iters, lam, L):
    import torch
    x = torch.empty((plan.nz, plan.ny, plan.nx), dtype=torch.float32, device="cuda")
    plan.fista(y, x=x, iters=iters, lam=lam, L=L)
    return x


def _rel(a, b):
    return float((a - b).norm() / b.norm())


def test_slots_staggered_requests_equal_alone():
    import torch
    plan = Plan(16, 16, 8, 32, 32, 32, max_batch=4, medium=MED)
    L = 1.01 * plan.power_norm(torch.ones((8, 16, 16), device="cuda"), 50)
    ys = [_data(plan, s) for s in range(3)]
    lams = [0.0, 1e-3, 0.0]
    iters = [8, 5, 6]
    # A enters, runs 3 steps; B joins, 2 steps; C joins; A leaves after 8 of its own
    plan.slot_load(0, ys[0], lams[0], L)
    for _ in range(3):
        plan.slots_step(1)
    plan.slot_load(1, ys[1], lams[1], L)
    for _ in range(2):
        plan.slots_step(2)
    plan.slot_load(2, ys[2], lams[2], L)
    for _ in range(3):
        plan.slots_step(3)   # A: 8, B: 5, C: 3
    xa, _ = plan.slot_read(0)
    xb, r2b = plan.slot_read(1, resid=True)
    xa, xb = xa.clone(), xb.clone()
    plan.slot_move(0, 2)     # C moves into A's slot; B has finished too
    for _ in range(3):
        plan.slots_step(1)   # C: 6
    xc, _ = plan.slot_read(0)
    for x, y, lam, it in zip((xa, xb, xc), ys, lams, iters):
        ref = _alone(plan, y, it, lam, L)
        assert _rel(x, ref) < 1e-5
    assert r2b > 0


def test_server_mixed_trace_equals_alone():
    import torch
    geoms = [Geometry(16, 8, 32, 32, mz=64), Geometry(32, 8, 48, 64, mz=64)]
    srv = Server(geoms, budget_bytes=8 << 30, slots=4, engine_factory=CudaEngine)
    # engines built up front so every request sees the same L as its alone run
    plans = {}
    for g in geoms:
        eng = srv._engine_for(g.key)
        plans[g.key] = eng
    arr = poisson_arrivals(60.0, 0.6, seed=3)
    reqs = []
    for i, t in enumerate(arr):
        key = geoms[i % 2].key
        eng = plans[key]
        reqs.append(Request(i, key, _data(eng.plan, 100 + i % 5), iters=10 + (i % 3) * 5,
                            lam=0.0, arrival=float(t)))
    torch.cuda.synchronize()
    rep = srv.run(reqs, drain_seconds=30)
    assert rep["completed"] == len(reqs), rep
    for r in reqs:
        eng = plans[r.key]
        ref = _alone(eng.plan, r.y, r.iters, r.lam, eng.L)
        assert _rel(r.out, ref) < 1e-5, r.rid
    assert rep["p99_ms"] >= rep["p50_ms"] > 0
    # the one-at-a-time comparison path runs the same trace
    base = serve_one_at_a_time({k: (e.plan, e.L) for k, e in plans.items()},
                               [Request(r.rid, r.key, r.y, r.iters, r.lam, r.arrival) for r in reqs],
                               drain_seconds=30)
    assert base["completed"] == len(reqs)
    srv.close()
