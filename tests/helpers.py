"""Shared test helpers: torch/numpy conversion and the standard test grids.
Inputs come from paper_2603_28150_gb300.synth; expected values from oracle/."""
import numpy as np

import oracle

MED_CFG1 = oracle.Medium(c=1500.0, dx=100e-6, dy=100e-6, dz=100e-6, dt=20e-9)
MED_50UM = oracle.Medium(c=1500.0, dx=50e-6, dy=50e-6, dz=50e-6, dt=10e-9)


def cuda(a, fp64=False):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64 if fp64 else torch.float32,
                        device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def kspace_table(g, med, z0=1):
    """Spatial library from the oracle's one-solve construction."""
    mz = oracle.mz_for(g.nz, g.nt, med, z0)
    return oracle.table_kspace_solve(g, med, mz, z0=z0), mz
