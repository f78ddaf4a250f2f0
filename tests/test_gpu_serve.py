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


def test_served_tensor_path_equals_alone_and_oracle():
    """Slots on a split-BF16 plan (128 depths, so steps with >= 2 active slots
    contract on the tcgen05 tensor cores, BF16 hi/lo operands): FISTA-50
    requests that enter and leave at different times give, within the
    split-BF16 tolerance of 1e-3, what each gives alone (pat_fista_solve,
    batch 1: the FP32 CUDA-core path) and what the FP64 oracle gives."""
    import torch

    import oracle
    from tests.helpers import MED_50UM, cuda, host
    g = oracle.Grid.square(32, 128, 256)
    med = MED_50UM
    mz = oracle.mz_for(g.nz, g.nt, med)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, max_batch=4, bf16_split=True,
                medium=Medium(med.c, med.dx, med.dy, med.dz, med.dt, mz, 1))
    assert plan.info()["tensor_min_batch"] == 2
    op = oracle.Operator(g, Hf=oracle.table_kspace_closed(g, med, mz))
    L = 1.01 * oracle.power_norm(op, synth.gaussian_field(op.obj_shape, 7), 30)
    ys = []
    for s in range(3):
        clean = op.A(synth.vessel_phantom(g.nx, g.nz, seed=60 + s))
        ys.append(clean + 0.05 * np.sqrt(np.mean(clean ** 2))
                  * synth.gaussian_field(clean.shape, seed=70 + s))
    lams = [0.0, 1e-3 * float(np.abs(op.AT(ys[1])).max()), 0.0]
    yd = [cuda(y) for y in ys]
    # A alone for 5 steps; B joins (20 steps of 2); C joins (25 steps of 3): A done
    plan.slot_load(0, yd[0], lams[0], L)
    for _ in range(5):
        plan.slots_step(1)
    plan.slot_load(1, yd[1], lams[1], L)
    for _ in range(20):
        plan.slots_step(2)
    plan.slot_load(2, yd[2], lams[2], L)
    for _ in range(25):
        plan.slots_step(3)
    xa = plan.slot_read(0)[0].clone()
    plan.slot_move(0, 2)           # C takes A's slot
    for _ in range(5):
        plan.slots_step(2)         # B done (50), C at 30
    xb = plan.slot_read(1)[0].clone()
    for _ in range(20):
        plan.slots_step(1)         # C done
    xc = plan.slot_read(0)[0].clone()
    plan.check()
    torch.cuda.synchronize()
    for x, y, lam in zip((xa, xb, xc), yd, lams):
        alone = _alone(plan, y, 50, lam, L)
        assert _rel(x, alone) < 1e-3
    for x, y, lam in zip((xa, xb, xc), ys, lams):
        ref = oracle.fista(op, y, L, iters=50, lam=lam).x
        assert oracle.rel_l2(host(x), ref) < 1e-3
    # the same three requests as one batched solve on the tensor path
    xs, _ = plan.fista(torch.stack(yd), iters=50, lam=0.0, L=L)
    plan.check()
    for v in (0, 2):
        assert oracle.rel_l2(host(xs[v]), oracle.fista(op, ys[v], L, iters=50).x) < 1e-3
