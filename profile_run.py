"""A short, fixed run of the operator for kernel profilers (few launches, small
device footprint): builds a plan with a device-generated real library and
applies `--pairs` gradients H*(H x - y) (one forward and one adjoint each).

  python profile_run.py [--n 128] [--nz 64] [--nt 256]
         [--pairs 3] [--fista 0] [--batch 1] [--no-fold] [--no-radial] [--complex] [--tensor]

The data y = H x come first (4 FFT launches, 1 contraction). Each pair then
launches, in order: stage i over depths (row, column FFT), the depth
contraction, stage iii over time samples (column, row inverse FFT), stage i
over time samples, the time contraction, stage iii over depths; so a profiler
skipping 12 FFT launches (or 3 contractions) starts at the second pair.
With --fista N a power iteration (5 pairs) and an N-iteration FISTA solve
follow (one CUDA graph of 8 kernels per iteration).
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import torch  # noqa: E402

from paper_2603_28150_gb300 import Medium, Plan, synth  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--nz", type=int, default=64)
    ap.add_argument("--nt", type=int, default=256)
    ap.add_argument("--pairs", type=int, default=3)
    ap.add_argument("--fista", type=int, default=0, help="FISTA iterations after the pairs")
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--no-fold", action="store_true")
    ap.add_argument("--no-radial", action="store_true",
                    help="one stored row per D4 representative (no radial sharing)")
    ap.add_argument("--complex", action="store_true", help="store the complex table")
    ap.add_argument("--tensor", action="store_true", help="split-BF16 tensor-core tables")
    a = ap.parse_args(argv)
    p = 1
    while p < 2 * a.n:
        p *= 2
    mz = 1
    while mz < 1 + a.nz + a.nt * 1500.0 * 10e-9 / 50e-6 + 1:
        mz *= 2
    plan = Plan(a.n, a.n, a.nz, a.nt, p, p, max_batch=a.batch, fold=not a.no_fold,
                radial=not a.no_radial,
                force_complex=a.complex, bf16_split=a.tensor,
                medium=Medium(1500.0, 50e-6, 50e-6, 50e-6, 10e-9, mz, 1))
    dev = torch.device("cuda")
    x = torch.tensor(synth.vessel_phantom(a.n, a.nz, seed=0), dtype=torch.float32,
                     device=dev).expand(a.batch, -1, -1, -1).contiguous()
    y = plan.forward(x).contiguous()
    g = torch.empty_like(x)
    for _ in range(a.pairs):
        plan.gradient(x, y, out=g, resid=False)
    if a.fista:
        L = 1.01 * plan.power_norm(torch.ones_like(x[0]), 5)
        plan.fista(y[0], iters=a.fista, L=L)
    torch.cuda.synchronize()
    plan.check()
    info = plan.info()
    print(f"pairs={a.pairs} batch={a.batch} folded={info['folded']} radial={info['radial']} "
          f"real={info['real_table']} "
          f"table_gb={info['table_bytes'] / 1e9:.3f}")


if __name__ == "__main__":
    main()
