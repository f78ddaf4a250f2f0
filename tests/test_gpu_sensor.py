"""GPU parity of the sensor-response folding (Sec. 2: the sensors' temporal
impulse response incorporated into the kernels by temporal convolution):
the plan's operator after pat_plan_set_sensor_response against the FP64
oracle's operator on the folded kernels, for k-space (folded and unfolded),
asymmetric and FP64 libraries, the tensor-core path, and at the benchmark
geometry against the time convolution of the unfolded plan's output."""
import numpy as np
import pytest

import oracle
from paper_2603_28150_gb300 import Medium, PatError, Plan, synth
from tests.helpers import MED_50UM, MED_CFG1, cuda, host, kspace_table

pytestmark = pytest.mark.gpu

CFG1 = oracle.Grid.square(32, 16, 64)
RAGGED = oracle.Grid(nx=23, ny=17, nz=5, nt=9, px=64, py=64)


def _response(nr, seed):
    # a damped oscillation with noise: band-limited like a real sensor
    t = np.arange(nr)
    return np.exp(-t / 4.0) * np.cos(0.9 * t) + 0.05 * synth.gaussian_field((nr,), seed)


@pytest.mark.parametrize("g,kind,fp64,fold", [(CFG1, "kspace", False, True),
                                              (CFG1, "kspace", False, False),
                                              (RAGGED, "random", False, False),
                                              (RAGGED, "random", True, False)])
def test_folded_response_matches_oracle(g, kind, fp64, fold):
    h = (kspace_table(g, MED_CFG1)[0] if kind == "kspace"
         else synth.random_kernels(g.nz, g.nt, g.px, g.py, seed=3))
    r = _response(7, 1)
    op = oracle.Operator(g, h=oracle.apply_sensor_response(h, r))
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, fp64=fp64, fold=fold)
    assert plan.info()["folded"] == (1 if (fold and kind == "kspace" and not fp64) else 0)
    plan.set_sensor_response(r)
    x = synth.blobs(g.nx, g.ny, g.nz, count=6, seed=4)
    y = synth.gaussian_field(op.data_shape, seed=5)
    tol = 1e-12 if fp64 else 1e-5
    assert oracle.rel_l2(host(plan.forward(cuda(x, fp64))), op.A(x)) < tol
    assert oracle.rel_l2(host(plan.adjoint(cuda(y, fp64))), op.AT(y)) < tol
    # a second call folds the convolution of both responses
    r2 = _response(3, 2)
    plan.set_sensor_response(r2)
    op2 = oracle.Operator(g, h=oracle.apply_sensor_response(h, np.convolve(r, r2)))
    assert oracle.rel_l2(host(plan.forward(cuda(x, fp64))), op2.A(x)) < tol


def test_response_on_tensor_path_matches_cuda_core():
    g = oracle.Grid.square(16, 128, 128)
    med = MED_50UM
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, max_batch=4, bf16_split=True,
                medium=Medium(med.c, med.dx, med.dy, med.dz, med.dt,
                              oracle.mz_for(g.nz, g.nt, med), 1))
    plan.set_sensor_response(_response(12, 3))
    xs = cuda(np.stack([synth.vessel_phantom(g.nx, g.nz, seed=s) for s in range(4)]))
    d_tc = host(plan.forward(xs))
    plan.check()
    plan.set_tensor_batch(0)
    d_cc = host(plan.forward(xs))
    for v in range(4):
        assert oracle.rel_l2(d_tc[v], d_cc[v]) < 1e-4, v


def test_response_full_size_equals_time_convolution():
    """128^2 -> 256^2, 64 depths, 256 samples (the benchmark geometry): H' x
    equals H x convolved along time with r (torch conv1d on the device)."""
    import torch
    g = oracle.Grid.square(128, 64, 256)
    med = MED_50UM
    mz = oracle.mz_for(g.nz, g.nt, med)
    medium = Medium(med.c, med.dx, med.dy, med.dz, med.dt, mz, 1)
    plain = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, medium=medium)
    folded = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, medium=medium)
    r = _response(16, 4)
    folded.set_sensor_response(r)
    x = cuda(synth.vessel_phantom(g.nx, g.nz, seed=0))
    d = plain.forward(x).double()  # [nt][ny][nx]
    seq = d.permute(1, 2, 0).reshape(-1, 1, g.nt)
    w = torch.tensor(r[::-1].copy(), dtype=torch.float64, device="cuda").view(1, 1, -1)
    ref = torch.nn.functional.conv1d(torch.nn.functional.pad(seq, (len(r) - 1, 0)), w)
    ref = ref.reshape(g.ny, g.nx, g.nt).permute(2, 0, 1)
    got = folded.forward(x).double()
    assert float((got - ref).norm() / ref.norm()) < 1e-5


def test_response_arguments():
    g = RAGGED
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py,
                table=synth.random_kernels(g.nz, g.nt, g.px, g.py, seed=9))
    with pytest.raises(PatError):
        plan.set_sensor_response([])
    x = cuda(synth.blobs(g.nx, g.ny, g.nz, count=3, seed=1))
    before = host(plan.forward(x))
    plan.set_sensor_response([1.0])  # unit response: unchanged
    assert oracle.rel_l2(host(plan.forward(x)), before) < 1e-7
