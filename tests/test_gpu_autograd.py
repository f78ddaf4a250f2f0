"""torch.autograd wrapper of H with H* as its backward (differentiation row):
FP64 gradcheck, finite differences of 1/2 ||Ax - y||^2 + 1e-3 TV(x) on 32
random directions at 64^2 (padded 128^2) x 32 depths x 128 samples, and the
FP32 gradient against the oracle's H*(Hx - y)."""
import numpy as np
import pytest

import oracle
from paper_2603_28150_gb300 import Plan, apply, synth
from tests.helpers import MED_50UM, cuda, host, kspace_table

pytestmark = pytest.mark.gpu


def _tv(x, eps=1e-3):
    """Isotropic TV with forward differences and replicate boundary (torch)."""
    import torch
    dz = torch.diff(x, dim=-3, append=x[..., -1:, :, :])
    dy = torch.diff(x, dim=-2, append=x[..., :, -1:, :])
    dx = torch.diff(x, dim=-1, append=x[..., :, :, -1:])
    return torch.sqrt(dz * dz + dy * dy + dx * dx + eps * eps).sum()


def test_gradcheck_fp64_small():
    import torch
    g = oracle.Grid(nx=6, ny=5, nz=3, nt=4, px=16, py=16)
    h = synth.random_kernels(g.nz, g.nt, g.px, g.py, seed=1)   # asymmetric: complex path
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, fp64=True, max_batch=2)
    x = torch.tensor(synth.gaussian_field((2, g.nz, g.ny, g.nx), 2), dtype=torch.float64,
                     device="cuda", requires_grad=True)
    # central differences of outputs of magnitude ~10 carry ~1e-9 rounding at eps = 1e-6
    assert torch.autograd.gradcheck(lambda v: apply(plan, v), (x,), eps=1e-6, atol=1e-7, rtol=1e-6)


@pytest.fixture(scope="module")
def cfg4():
    g = oracle.Grid.square(64, 32, 128)
    h, _ = kspace_table(g, MED_50UM)
    op = oracle.Operator(g, h=h)
    x = synth.vessel_phantom(g.nx, g.nz, seed=3)
    y = op.A(synth.vessel_phantom(g.nx, g.nz, seed=4))
    return g, h, op, x, y


def _loss(plan, x, y):
    r = apply(plan, x) - y
    return 0.5 * (r * r).sum() + 1e-3 * _tv(x)


def test_cfg4_finite_differences_fp64(cfg4):
    import torch
    g, h, op, x0, y0 = cfg4
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, fp64=True)
    x = torch.tensor(x0, dtype=torch.float64, device="cuda", requires_grad=True)
    y = torch.tensor(y0, dtype=torch.float64, device="cuda")
    L = _loss(plan, x, y)
    (grad,) = torch.autograd.grad(L, x)
    step = 1e-4
    worst = 0.0
    for k in range(32):
        v = torch.tensor(synth.gaussian_field(x.shape, 100 + k), dtype=torch.float64, device="cuda")
        v /= torch.linalg.norm(v)
        with torch.no_grad():
            fd = (_loss(plan, x + step * v, y) - _loss(plan, x - step * v, y)) / (2 * step)
        an = float((grad * v).sum())
        worst = max(worst, abs(float(fd) - an) / max(abs(an), 1e-30))
    assert worst < 1e-6, worst


@pytest.mark.parametrize("fp64", [False, True])
def test_cfg4_gradient_matches_oracle(cfg4, fp64):
    import torch
    g, h, op, x0, y0 = cfg4
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, fp64=fp64)
    x = cuda(x0, fp64).requires_grad_(True)
    y = cuda(y0, fp64)
    r = apply(plan, x) - y
    (0.5 * (r * r).sum()).backward()
    ref = op.AT(op.A(x0) - y0)  # Eq. 15
    assert oracle.rel_l2(host(x.grad), ref) < (1e-12 if fp64 else 1e-5)
