"""GPU parity of the measurement operator (Sec. 2.3, Sec. 3.3): S H and
H* S^T through the C ABI against the FP64 oracle's composed pair, FISTA on
scan-grid data, the slots, and the full-size benchmark geometry against the
unsampled GPU operator (the sampled forward keeps exactly the scan positions
of H rho; the sampled adjoint equals H* of the zero-filled data).

Tolerances as for the plain operator: FP32 <= 1e-5 relative l2, FP64 <= 1e-12."""
import numpy as np
import pytest

import oracle
from paper_2603_28150_gb300 import Medium, PatError, Plan, synth
from tests.helpers import MED_50UM, MED_CFG1, cuda, host, kspace_table

pytestmark = pytest.mark.gpu

CFG1 = oracle.Grid.square(32, 16, 64)
RAGGED = oracle.Grid(nx=23, ny=17, nz=5, nt=9, px=64, py=64)
RECT = oracle.Grid(nx=20, ny=9, nz=3, nt=7, px=64, py=32)
PATTERNS = [(2, 2, 0, 0), (2, 2, 1, 1), (3, 2, 1, 0), (2, 3, 0, 2), (5, 1, 4, 0)]


def _table(g, kind, seed):
    if kind == "random":
        return synth.random_kernels(g.nz, g.nt, g.px, g.py, seed=seed)
    return kspace_table(g, MED_CFG1)[0]


@pytest.mark.parametrize("g", [CFG1, RAGGED, RECT], ids=["cfg1", "ragged", "rect"])
@pytest.mark.parametrize("samp", PATTERNS, ids=[str(p) for p in PATTERNS])
@pytest.mark.parametrize("kind,fp64", [("random", False), ("kspace", False), ("random", True)])
def test_sampled_pair_matches_oracle(g, samp, kind, fp64):
    h = _table(g, kind, seed=g.nx + samp[0])
    op = oracle.Operator(g, h=h, sampling=samp)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, fp64=fp64, max_batch=2)
    plan.set_sampling(*samp)
    assert plan.data_shape(1)[1:] == op.data_shape
    rho = synth.blobs(g.nx, g.ny, g.nz, count=6, seed=2) + 0.1 * synth.gaussian_object(g.nx, g.ny, g.nz, 3)
    y = synth.gaussian_field(op.data_shape, seed=4)
    tol = 1e-12 if fp64 else 1e-5
    d = host(plan.forward(cuda(rho, fp64)))
    assert d.shape == op.data_shape
    assert oracle.rel_l2(d, op.A(rho)) < tol
    a = host(plan.adjoint(cuda(y, fp64)))
    assert oracle.rel_l2(a, op.AT(y)) < tol
    # batch of two equals the single volumes
    rho2 = np.stack([rho, synth.blobs(g.nx, g.ny, g.nz, count=4, seed=5)])
    d2 = host(plan.forward(cuda(rho2, fp64)))
    assert np.array_equal(d2[0], d)
    assert oracle.rel_l2(d2[1], op.A(rho2[1])) < tol
    y2 = np.stack([y, synth.gaussian_field(op.data_shape, seed=6)])
    a2 = host(plan.adjoint(cuda(y2, fp64)))
    assert np.array_equal(a2[0], a)
    assert oracle.rel_l2(a2[1], op.AT(y2[1])) < tol


@pytest.mark.parametrize("fp64", [False, True])
def test_sampled_adjoint_identity(fp64):
    g = RAGGED
    h = _table(g, "random", seed=31)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, fp64=fp64)
    plan.set_sampling(3, 2, 2, 1)
    x = cuda(synth.gaussian_field(plan.obj_shape(1)[1:], 7), fp64)
    y = cuda(synth.gaussian_field(plan.data_shape(1)[1:], 8), fp64)
    lhs = plan.dot(plan.forward(x), y)
    rhs = plan.dot(x, plan.adjoint(y))
    assert abs(lhs - rhs) <= (1e-12 if fp64 else 1e-5) * max(abs(lhs), abs(rhs))


def test_sampled_fista_matches_oracle():
    """Sec. 3.3 set-up in miniature: reconstruction grid twice as fine as the
    scan grid, FISTA with positivity and l1 on scan-grid data."""
    g = CFG1
    h = _table(g, "kspace", seed=0)
    op = oracle.Operator(g, h=h, sampling=(2, 2, 0, 0))
    p0 = synth.vessel_phantom(g.nx, g.nz, seed=9)
    clean = op.A(p0)
    y = clean + 0.05 * np.sqrt(np.mean(clean ** 2)) * synth.gaussian_field(clean.shape, 10)
    L = 1.01 * oracle.power_norm(op, synth.gaussian_field(op.obj_shape, 11), 50)
    lam = 1e-3 * float(np.abs(op.AT(y)).max())
    ref = oracle.fista(op, y, L, iters=40, lam=lam, track=True)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h)
    plan.set_sampling(2, 2, 0, 0)
    x, rep = plan.fista(cuda(y), iters=40, lam=lam, L=L)
    assert oracle.rel_l2(host(x), ref.x) < 1e-5
    assert abs(rep["resid2_first"] - ref.resid2[0]) < 1e-5 * ref.resid2[0]
    # power iteration on (S H)* (S H)
    v0 = synth.gaussian_field(op.obj_shape, 12)
    L_gpu = plan.power_norm(cuda(v0), 30)
    L_ref = oracle.power_norm(op, v0, 30)
    assert abs(L_gpu - L_ref) / L_ref < 1e-5


def test_sampled_slots_equal_fista():
    import torch
    g = oracle.Grid.square(16, 8, 32)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, max_batch=3,
                medium=Medium(1500.0, 50e-6, 50e-6, 50e-6, 10e-9, 64, 1))
    plan.set_sampling(2, 2, 1, 0)
    L = 1.01 * plan.power_norm(torch.ones(plan.obj_shape(1)[1:], device="cuda"), 40)
    ys = [plan.forward(cuda(synth.vessel_phantom(g.nx, g.nz, seed=s))).contiguous() for s in (1, 2)]
    plan.slot_load(0, ys[0], 0.0, L)
    plan.slots_step(1)
    plan.slot_load(1, ys[1], 1e-3, L)
    for _ in range(4):
        plan.slots_step(2)
    xa = plan.slot_read(0)[0].clone()
    xb = plan.slot_read(1)[0].clone()
    ra, _ = plan.fista(ys[0], iters=5, lam=0.0, L=L)
    rb, _ = plan.fista(ys[1], iters=4, lam=1e-3, L=L)
    assert float((xa - ra).norm() / ra.norm()) < 1e-5
    assert float((xb - rb).norm() / rb.norm()) < 1e-5


def test_set_sampling_arguments_and_reset():
    g = RECT
    h = _table(g, "random", seed=41)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h)
    for bad in [(0, 1, 0, 0), (1, 0, 0, 0), (1, 1, -1, 0), (1, 1, g.nx, 0), (1, 1, 0, g.ny)]:
        with pytest.raises(PatError):
            plan.set_sampling(*bad)
    rho = cuda(synth.blobs(g.nx, g.ny, g.nz, count=4, seed=42))
    plain = host(plan.forward(rho))
    plan.set_sampling(2, 3, 1, 2)
    assert host(plan.forward(rho)).shape == (g.nt, len(range(2, g.ny, 3)), len(range(1, g.nx, 2)))
    plan.set_sampling(1, 1, 0, 0)
    assert np.array_equal(host(plan.forward(rho)), plain)
    # largest strides: one scan position per axis
    plan.set_sampling(g.nx, g.ny, g.nx - 1, g.ny - 1)
    d = host(plan.forward(rho))
    assert d.shape == (g.nt, 1, 1)
    assert np.array_equal(d[:, 0, 0], plain[:, g.ny - 1, g.nx - 1])


def test_sampled_full_size_against_unsampled_gpu_operator():
    """128^2 reconstruction grid (256^2 padded), 64 depths, 256 samples, table
    generated on the device, scan grid of every second position (Sec. 3.3):
    S H rho is exactly the scan positions of H rho and H* S^T y exactly H* of
    the zero-filled y (the same kernels compute the same values)."""
    import torch
    g = oracle.Grid.square(128, 64, 256)
    med = MED_50UM
    mz = oracle.mz_for(g.nz, g.nt, med)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, max_batch=2,
                medium=Medium(med.c, med.dx, med.dy, med.dz, med.dt, mz, 1))
    rho = cuda(np.stack([synth.vessel_phantom(g.nx, g.nz, seed=s) for s in (0, 1)]))
    full = plan.forward(rho).clone()
    y = cuda(synth.gaussian_field((2, g.nt, 64, 64), 3))
    zf = torch.zeros_like(full)
    zf[:, :, 0::2, 0::2] = y
    a_full = plan.adjoint(zf).clone()
    plan.set_sampling(2, 2, 0, 0)
    assert torch.equal(plan.forward(rho), full[:, :, 0::2, 0::2])
    assert torch.equal(plan.adjoint(y), a_full)


def test_sampled_batched_tensor_path_matches_cuda_core():
    """Measurement operator on the batched tensor-core path (folded tiles,
    spectra in the representative-slot layout) against the single-precision
    CUDA-core path on the same plan, volume by volume."""
    g = oracle.Grid.square(16, 128, 128)
    med = MED_50UM
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, max_batch=4, bf16_split=True,
                medium=Medium(med.c, med.dx, med.dy, med.dz, med.dt,
                              oracle.mz_for(g.nz, g.nt, med), 1))
    assert plan.info()["folded"] == 1 and plan.info()["tensor_min_batch"] == 2
    plan.set_sampling(2, 2, 1, 0)
    xs = cuda(np.stack([synth.vessel_phantom(g.nx, g.nz, seed=s) for s in range(4)]))
    ys = cuda(np.stack([synth.gaussian_field(plan.data_shape(1)[1:], 80 + s) for s in range(4)]))
    d_tc, a_tc = host(plan.forward(xs)), host(plan.adjoint(ys))
    plan.check()
    plan.set_tensor_batch(0)
    d_cc, a_cc = host(plan.forward(xs)), host(plan.adjoint(ys))
    for v in range(4):
        assert oracle.rel_l2(d_tc[v], d_cc[v]) < 1e-4, v
        assert oracle.rel_l2(a_tc[v], a_cc[v]) < 1e-4, v
