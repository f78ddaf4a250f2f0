"""The C-ABI boundary on the GPU: plans on caller-owned (torch) workspace,
clean-up after a failed device allocation (host-side fault injection), the
bounded-wait path of the tensor-core kernels (a wait limit of 0 makes every
pipeline wait give up: no device fault involved), and the seeded power
iteration against the oracle started from the same counter-based vector."""
import numpy as np
import pytest

import oracle
from paper_2603_28150_gb300 import Medium, PatError, Plan, pat, synth
from tests.helpers import MED_50UM, cuda, kspace_table

pytestmark = pytest.mark.gpu

G = oracle.Grid.square(24, 12, 40)
MED = Medium(1500.0, 50e-6, 50e-6, 50e-6, 10e-9, 64, 1)


def _ws(nbytes, offset=0):
    import torch
    buf = torch.empty(nbytes + offset + 256, dtype=torch.uint8, device="cuda")
    start = (-buf.data_ptr()) % 256 + offset
    return buf, buf[start:start + nbytes]


@pytest.mark.parametrize("kind", ["kspace", "table"])
def test_workspace_plan_equals_self_allocating_plan(kind):
    import torch
    B = 3
    n = pat.workspace_size(G.nx, G.ny, G.nz, G.nt, G.px, G.py, max_batch=B)
    _, ws = _ws(n)
    src = {"medium": MED} if kind == "kspace" else {"table": kspace_table(G, oracle.Medium(
        c=1500.0, dx=50e-6, dy=50e-6, dz=50e-6, dt=10e-9))[0]}
    base = pat.debug_live_allocations()
    pw = Plan(G.nx, G.ny, G.nz, G.nt, G.px, G.py, max_batch=B, workspace=ws, **src)
    held = pat.debug_live_allocations() - base   # the table side only
    pa = Plan(G.nx, G.ny, G.nz, G.nt, G.px, G.py, max_batch=B, **src)
    assert pw.info()["workspace_external"] == 1 and pa.info()["workspace_external"] == 0
    assert pat.debug_live_allocations() - base == 2 * held + 1  # + the other plan's arena
    xs = cuda(np.stack([synth.blobs(G.nx, G.ny, G.nz, count=3, seed=s) for s in range(B)]))
    ys = cuda(np.stack([synth.gaussian_field((G.nt, G.ny, G.nx), 10 + s) for s in range(B)]))
    for op in ("forward", "adjoint"):
        a = getattr(pw, op)(xs if op == "forward" else ys)
        b = getattr(pa, op)(xs if op == "forward" else ys)
        assert torch.equal(a, b), op
    L = 1.01 * pa.power_norm(torch.ones((G.nz, G.ny, G.nx), device="cuda"), 30)
    xw, _ = pw.fista(ys, iters=12, L=L)
    xa, _ = pa.fista(ys, iters=12, L=L)
    assert torch.equal(xw, xa)
    # host pointers use the staging carved from the caller's workspace
    before = pat.debug_live_allocations()
    dh = pw.forward(xs.cpu())
    assert torch.equal(dh, pa.forward(xs).cpu())
    assert pat.debug_live_allocations() == before
    # slots
    for p in (pw, pa):
        p.slot_load(0, ys[0], 0.0, L)
        p.slot_load(1, ys[1], 0.0, L)
        for _ in range(4):
            p.slots_step(2)
    assert torch.equal(pw.slot_read(1)[0], pa.slot_read(1)[0])
    with pytest.raises(PatError) as e:
        pw.fista(ys[:1], iters=5000, L=L)
    assert e.value.code == pat.PAT_ERR_ARG
    pw.close()
    pa.close()
    assert pat.debug_live_allocations() == base


def test_workspace_rejected_when_too_small_misaligned_or_host():
    import torch
    n = pat.workspace_size(G.nx, G.ny, G.nz, G.nt, G.px, G.py)
    base = pat.debug_live_allocations()
    for ws in (_ws(n - 256)[1], _ws(n, offset=16)[1], torch.empty(n, dtype=torch.uint8)):
        with pytest.raises((PatError, ValueError)) as e:
            Plan(G.nx, G.ny, G.nz, G.nt, G.px, G.py, medium=MED, workspace=ws)
        if isinstance(e.value, PatError):
            assert e.value.code == pat.PAT_ERR_ARG
    assert pat.debug_live_allocations() == base
    Plan(G.nx, G.ny, G.nz, G.nt, G.px, G.py, medium=MED, workspace=_ws(n)[1]).close()


def test_binding_rejects_short_or_mistyped_buffers():
    """Caller-supplied outputs and second inputs of the operator, stage and
    slot calls are checked (element count and type) before the library is
    called; the plan then still computes correctly."""
    import torch
    p = Plan(G.nx, G.ny, G.nz, G.nt, G.px, G.py, medium=MED)
    rho = torch.rand((G.nz, G.ny, G.nx), device="cuda")
    d = torch.rand((G.nt, G.ny, G.nx), device="cuda")
    short_d = torch.empty(G.nt * G.ny * G.nx - 1, device="cuda")
    f64_rho = torch.empty((G.nz, G.ny, G.nx), dtype=torch.float64, device="cuda")
    kp = p.info()["bins_padded"]
    X = torch.zeros((G.nz, kp), dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError, match="out"):
        p.forward(rho, out=short_d)
    with pytest.raises(ValueError, match="out"):
        p.adjoint(d, out=f64_rho)
    with pytest.raises(ValueError, match="y"):
        p.gradient(rho, short_d)
    with pytest.raises(ValueError, match="X"):
        p.stage_contract(X[:-1], torch.zeros((G.nt, kp), dtype=torch.complex64, device="cuda"))
    with pytest.raises(ValueError, match="out"):
        p.stage_contract(X, torch.zeros((G.nt, kp), dtype=torch.complex128, device="cuda"))
    with pytest.raises(ValueError, match="x"):
        p.fista(d, x=short_d, iters=2, L=1.0, warm_start=True)
    out = torch.full((G.nt, G.ny, G.nx), float("nan"), device="cuda")
    p.forward(rho, out=out)
    assert torch.equal(out, p.forward(rho))
    p.close()


@pytest.mark.parametrize("kind", ["kspace", "table_folded", "table_complex", "bf16"])
def test_failed_allocation_cleans_up(monkeypatch, kind):
    """The n-th device allocation of plan creation fails (n = 1, 2, ...): each
    attempt returns PAT_ERR_OOM and leaves no allocation behind, until n passes
    the number of allocations and the plan builds."""
    import torch
    if kind == "bf16":
        g, kw = oracle.Grid.square(16, 128, 128), {"bf16_split": True, "max_batch": 4}
        kw["medium"] = Medium(1500.0, 50e-6, 50e-6, 50e-6, 10e-9,
                              oracle.mz_for(128, 128, MED_50UM), 1)
    else:
        g, kw = G, {}
        if kind == "kspace":
            kw["medium"] = MED
        else:
            h = synth.random_kernels(g.nz, g.nt, g.px, g.py, seed=3, d4=True)
            # a device table (no host staging) and a host table
            kw["table"] = torch.tensor(h, device="cuda") if kind == "table_folded" else h
            kw["force_complex"] = kind == "table_complex"
    base = pat.debug_live_allocations()
    for n in range(1, 80):
        monkeypatch.setenv("PAT_DEBUG_FAIL_ALLOC", str(n))
        try:
            plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, **kw)
        except PatError as e:
            assert e.code == pat.PAT_ERR_OOM, (n, e)
            assert pat.debug_live_allocations() == base, n
            continue
        monkeypatch.delenv("PAT_DEBUG_FAIL_ALLOC")
        assert n >= 3
        info = plan.info()
        assert info["folded"] == (1 if kind in ("kspace", "table_folded", "bf16") else 0)
        plan.close()
        assert pat.debug_live_allocations() == base
        break
    else:
        pytest.fail("plan creation never succeeded")


@pytest.mark.parametrize("fold", [True, False])
def test_tensor_wait_timeout_is_reported_and_recovers(fold):
    """A wait limit of 0 makes every pipeline wait of the tcgen05 contraction
    give up: the kernel drains what it issued, frees its tensor memory and
    returns; pat_plan_check reports PAT_ERR_TIMEOUT once. Back at the default
    limit the next call matches the CUDA-core path."""
    import torch
    g = oracle.Grid.square(16, 128, 256)
    B = 16
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, max_batch=B, bf16_split=True, fold=fold,
                medium=Medium(1500.0, 50e-6, 50e-6, 50e-6, 10e-9,
                              oracle.mz_for(g.nz, g.nt, MED_50UM), 1))
    Kp = plan.info()["bins_padded"]
    gen = torch.Generator(device="cuda").manual_seed(2)
    X = torch.randn((B, g.nz, Kp), dtype=torch.complex64, device="cuda", generator=gen)
    D = torch.randn((B, g.nt, Kp), dtype=torch.complex64, device="cuda", generator=gen)
    Y = torch.zeros((B, g.nt, Kp), dtype=torch.complex64, device="cuda")
    Z = torch.zeros((B, g.nz, Kp), dtype=torch.complex64, device="cuda")
    plan.set_wait_limit(0)
    for adjoint in (False, True):
        if adjoint:
            plan.stage_contract(D, Z, batch=B, adjoint=True)
        else:
            plan.stage_contract(X, Y, batch=B)
        with pytest.raises(PatError) as e:
            plan.check()
        assert e.value.code == pat.PAT_ERR_TIMEOUT
        plan.check()  # the flag was cleared
    # the operator path (batch >= 2 takes the tensor cores) reports it as well
    xs = torch.rand((2, g.nz, g.ny, g.nx), device="cuda")
    plan.forward(xs)
    with pytest.raises(PatError):
        plan.check()
    plan.set_wait_limit(-1)
    K = plan.info()["bins"]
    outs = {}
    for mode in ("tensor", "cuda"):
        plan.set_tensor_batch(2 if mode == "tensor" else 0)
        Y.zero_()
        Z.zero_()
        plan.stage_contract(X, Y, batch=B)
        plan.stage_contract(D, Z, batch=B, adjoint=True)
        plan.check()
        outs[mode] = (Y[..., :K].clone(), Z[..., :K].clone())
    for i in range(2):
        a, b = outs["tensor"][i], outs["cuda"][i]
        assert float((a - b).norm() / b.norm()) < 1e-4


def test_power_norm_seed_matches_oracle():
    """The device start vector is splitmix64 of (seed, index); the oracle runs
    its power iteration from the same sequence drawn on the host."""
    g = oracle.Grid.square(16, 8, 32)
    h = kspace_table(g, oracle.Medium(c=1500.0, dx=100e-6, dy=100e-6, dz=100e-6, dt=20e-9))[0]
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h)
    for seed in (0, 0x5EED, 2 ** 63 + 12345):
        v0 = synth.splitmix_uniform(g.nz * g.ny * g.nx, seed).reshape(g.nz, g.ny, g.nx)
        L_ref = oracle.power_norm(oracle.Operator(g, h=h), v0, 12)
        L_gpu = plan.power_norm_seed(12, seed)
        assert abs(L_gpu - L_ref) / L_ref < 1e-5, seed
        # the same start vector passed explicitly gives the same L
        assert abs(plan.power_norm(cuda(v0), 12) - L_gpu) <= 1e-6 * L_gpu
