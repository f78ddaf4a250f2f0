"""Batched split-BF16 contraction on tcgen05 (precision + batching row): the
tensor-core path against the single-precision CUDA-core path on identical
inputs, and the whole operator against the FP64 oracle per volume (target
<= 1e-3 relative; FFTs stay FP32)."""
import numpy as np
import pytest

import oracle
from paper_2603_28150_gb300 import Medium, PatError, Plan, synth
from tests.helpers import MED_50UM, cuda, host

pytestmark = pytest.mark.gpu


def _medium(g, med):
    return Medium(med.c, med.dx, med.dy, med.dz, med.dt, oracle.mz_for(g.nz, g.nt, med), 1)


@pytest.mark.parametrize("n,nt,fold", [(16, 128, True), (24, 256, True), (32, 512, True),
                                        (24, 256, False)])
@pytest.mark.parametrize("batch", [16, 5, 20])
def test_tensor_contraction_matches_cuda_core(n, nt, fold, batch):
    """Folded plans run one tile set per representative (N = 4 bins x 32
    columns per MMA); unfolded plans one per bin."""
    import torch
    g = oracle.Grid.square(n, 128, nt)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, max_batch=batch,
                medium=_medium(g, MED_50UM), bf16_split=True, fold=fold)
    info = plan.info()
    assert info["real_table"] == 1 and info["tensor_min_batch"] == 2
    assert info["folded"] == (1 if fold else 0)
    # hi + lo BF16 per (table row, t, z), one copy per direction
    assert info["tensor_table_bytes"] == 2 * info["table_rows"] * g.nt * g.nz * 4
    Kp = info["bins_padded"]
    gen = torch.Generator(device="cuda").manual_seed(1)
    X = torch.randn((batch, g.nz, Kp), dtype=torch.complex64, device="cuda", generator=gen)
    D = torch.randn((batch, g.nt, Kp), dtype=torch.complex64, device="cuda", generator=gen)
    K = info["bins"]
    outs = {}
    for mode in ("tensor", "cuda"):
        plan.set_tensor_batch(2 if mode == "tensor" else 0)
        Y = torch.zeros((batch, g.nt, Kp), dtype=torch.complex64, device="cuda")
        Z = torch.zeros((batch, g.nz, Kp), dtype=torch.complex64, device="cuda")
        plan.stage_contract(X, Y, batch=batch)
        plan.stage_contract(D, Z, batch=batch, adjoint=True)
        plan.check()
        outs[mode] = (Y[..., :K].cpu().numpy(), Z[..., :K].cpu().numpy())
    for i in range(2):
        a, b = outs["tensor"][i], outs["cuda"][i]
        for v in range(batch):
            err = np.linalg.norm(a[v] - b[v]) / np.linalg.norm(b[v])
            assert err < 1e-4, (i, v, err)


def test_batched_operator_matches_fp64_oracle_per_volume():
    g = oracle.Grid.square(16, 128, 256)
    med = MED_50UM
    mz = oracle.mz_for(g.nz, g.nt, med)
    h = oracle.table_kspace_solve(g, med, mz)
    A = oracle.Operator(g, h=h)
    B = 16
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, max_batch=B, table=h, bf16_split=True)
    xs = np.stack([synth.vessel_phantom(g.nx, g.nz, seed=s) for s in range(B)])
    ys = np.stack([synth.gaussian_field((g.nt, g.ny, g.nx), 50 + s) for s in range(B)])
    d = host(plan.forward(cuda(xs)))
    a = host(plan.adjoint(cuda(ys)))
    plan.check()
    ef = [oracle.rel_l2(d[v], A.A(xs[v])) for v in range(B)]
    ea = [oracle.rel_l2(a[v], A.AT(ys[v])) for v in range(B)]
    assert max(ef) < 1e-3 and max(ea) < 1e-3, (max(ef), max(ea))
    # the split product is far better than plain BF16 (~4e-3): expect ~1e-5
    assert max(ef) < 1e-4 and max(ea) < 1e-4, (max(ef), max(ea))


def test_cfg3_sampled_outputs_full_size():
    """16 volumes, 128^2 -> 256^2, 128 depths, 512 samples, library generated on
    the device: sampled time samples of H rho and one depth of H* d for every
    volume against the oracle's closed-form library for those samples."""
    g = oracle.Grid.square(128, 128, 512)
    med = MED_50UM
    mz = oracle.mz_for(g.nz, g.nt, med)
    B = 16
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, max_batch=B,
                medium=Medium(med.c, med.dx, med.dy, med.dz, med.dt, mz, 1), bf16_split=True)
    xs = np.stack([synth.vessel_phantom(g.nx, g.nz, seed=s) for s in range(B)])
    d = host(plan.forward(cuda(xs)))
    plan.check()
    gt = oracle.Grid(g.nx, g.ny, g.nz, 1, g.px, g.py)
    for t in (150, 400):
        Hf = oracle.table_kspace_closed(g, med, mz, t_idx=[t])
        for v in (0, 7, 15):
            ref = oracle.forward_fft(Hf, xs[v], gt)[0]
            assert oracle.rel_l2(d[v, t], ref) < 1e-3, (t, v)
    ys = np.stack([synth.gaussian_field((g.nt, g.ny, g.nx), 70 + s) for s in range(B)])
    a = host(plan.adjoint(cuda(ys)))
    plan.check()
    Hf = oracle.table_kspace_closed(g, med, mz, z_idx=[40])
    gz = oracle.Grid(g.nx, g.ny, 1, g.nt, g.px, g.py)
    for v in (0, 15):
        ref = oracle.adjoint_fft(Hf, ys[v], gz)[0]
        assert oracle.rel_l2(a[v, 40], ref) < 1e-3, v


def test_contract_slots_equals_converting_stage():
    """pat_stage_contract_slots on spectra placed in the representative-slot
    layout (bin k at 4 u + i) gives, bit for bit, what pat_stage_contract
    gives on the bin layout (which converts to that layout and back)."""
    import torch

    from paper_2603_28150_gb300 import pat
    g = oracle.Grid.square(16, 128, 256)
    B = 16
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, max_batch=B, medium=_medium(g, MED_50UM),
                bf16_split=True)
    info = plan.info()
    assert info["folded"] == 1
    # with one rank the depth-side map is the slot position itself
    sinfo, slot, _, _ = pat.shard_layout(g.nx, g.ny, g.nz, g.nt, g.px, g.py, True, 0, 1)
    srow = sinfo["slot_width"]
    assert srow == 4 * ((info["table_rows"] + 31) // 32 * 32)
    slot = torch.tensor(slot, dtype=torch.long, device="cuda")
    K, Kp = info["bins"], info["bins_padded"]
    gen = torch.Generator(device="cuda").manual_seed(3)
    for adjoint, rin, rout in ((False, g.nz, g.nt), (True, g.nt, g.nz)):
        X = torch.randn((B, rin, Kp), dtype=torch.complex64, device="cuda", generator=gen)
        Y = plan.stage_contract(X, torch.zeros((B, rout, Kp), dtype=torch.complex64, device="cuda"),
                                batch=B, adjoint=adjoint)
        Xs = torch.zeros((B, rin, srow), dtype=torch.complex64, device="cuda")
        Xs[:, :, slot] = X[:, :, :K]
        Ys = plan.stage_contract_slots(Xs, torch.zeros((B, rout, srow), dtype=torch.complex64,
                                                       device="cuda"), B, adjoint=adjoint)
        plan.check()
        assert torch.equal(Ys[:, :, slot], Y[:, :, :K])
    with pytest.raises(PatError):
        plan.stage_contract_slots(Xs, Ys, 1)   # below the tensor batch: no slot layout
