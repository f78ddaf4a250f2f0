"""Frequency shards on the GPU: R shard plans (each holding 1/R of the
table's rows) run the real ShardedOperator as R threads of one process on
one GPU, exchanging through host barriers (no kernel waits on another
rank). Sharded H, H*, gradient and FISTA equal the unsharded plan."""
import threading

import numpy as np
import pytest

import oracle
from paper_2603_28150_gb300 import Medium, PatError, Plan, pat, synth
from paper_2603_28150_gb300.shard import ShardedOperator
from tests.helpers import MED_50UM, cuda

pytestmark = pytest.mark.gpu


class LocalExchange:
    """all_to_all / sum among R ranks that are threads of this process."""

    def __init__(self, world):
        self.world = world
        self.box = [None] * world
        self.bar = threading.Barrier(world, timeout=120)

    def rank(self, r):
        ex = self

        class View:
            def all_to_all(self, send):
                import torch
                torch.cuda.synchronize()
                ex.box[r] = send
                ex.bar.wait()
                recv = torch.stack([ex.box[q][r] for q in range(ex.world)])
                torch.cuda.synchronize()
                ex.bar.wait()
                return recv

            def sum(self, value, device):
                ex.box[r] = value
                ex.bar.wait()
                s = 0.0
                for q in range(ex.world):  # rank order: the same sum on every rank
                    s += ex.box[q]
                ex.bar.wait()
                return s
        return View()


def run_ranks(world, fn):
    """fn(rank) on `world` threads; returns their results, re-raises failures."""
    out, err = [None] * world, []

    def body(r):
        try:
            out[r] = fn(r)
        except BaseException as e:  # noqa: BLE001
            err.append(e)
    th = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if err:
        raise err[0]
    return out


def _medium(g):
    return Medium(MED_50UM.c, MED_50UM.dx, MED_50UM.dy, MED_50UM.dz, MED_50UM.dt,
                  oracle.mz_for(g.nz, g.nt, MED_50UM), 1)


@pytest.mark.parametrize("world", [1, 2, 4])
@pytest.mark.parametrize("fold", [True, False])
def test_sharded_operator_equals_plan(world, fold):
    import torch
    g = oracle.Grid.square(32, 16, 64)
    med = _medium(g)
    full = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, medium=med, fold=fold)
    shards = [Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, medium=med, fold=fold, shard=(r, world))
              for r in range(world)]
    info = shards[0].shard_info()
    assert info["folded"] == (1 if fold else 0) and info["world"] == world
    assert sum(p.shard_info()["rows"] for p in shards) == info["rows_total"]
    # each shard holds its share of the rows: rows_per_rank (a multiple of 32,
    # at most 31 above an even split), stored one per representative or bin,
    # or (folded) one per radius among its representatives
    rpr = info["rows_per_rank"]
    assert rpr % 32 == 0 and rpr * world >= info["rows_total"] and rpr < info["rows_total"] / world + 32
    for p in shards:
        pi = p.info()
        assert pi["table_bytes"] == pi["stored_rows"] * g.nt * g.nz * 4
        assert pi["stored_rows"] <= rpr and pi["radial"] == (1 if pi["stored_rows"] < 32 * (
            (p.shard_info()["rows"] + 31) // 32) else 0)
    with pytest.raises(PatError):
        shards[0].forward(torch.zeros((g.nz, g.ny, g.nx), device="cuda"))
    ex = LocalExchange(world)
    zr, tr = g.nz // world, g.nt // world
    rho = cuda(synth.blobs(g.nx, g.ny, g.nz, count=5, seed=1))
    y = cuda(synth.gaussian_field((g.nt, g.ny, g.nx), seed=2))
    meas = full.forward(cuda(synth.blobs(g.nx, g.ny, g.nz, count=4, seed=3)))
    L = 1.01 * full.power_norm(torch.ones((g.nz, g.ny, g.nx), device="cuda"), 40)

    def rank(r):
        sop = ShardedOperator(shards[r], ex.rank(r))
        zs, ts = slice(r * zr, (r + 1) * zr), slice(r * tr, (r + 1) * tr)
        d = sop.forward(rho[zs].contiguous())
        a = sop.adjoint(y[ts].contiguous())
        gr, r2 = sop.gradient(rho[zs].contiguous(), meas[ts].contiguous())
        x, _ = sop.fista(meas[ts].contiguous(), L, iters=20)
        Ls = sop.power_norm(torch.ones((zr, g.ny, g.nx), device="cuda"), 40)
        return d, a, gr, r2, x, Ls

    res = run_ranks(world, rank)
    cat = lambda i: torch.cat([res[r][i] for r in range(world)])  # noqa: E731
    rel = lambda a, b: float((a - b).norm() / b.norm())  # noqa: E731
    assert rel(cat(0), full.forward(rho)) < 1e-6
    assert rel(cat(1), full.adjoint(y)) < 1e-6
    gref, r2ref = full.gradient(rho, meas)
    assert rel(cat(2), gref) < 1e-6
    assert abs(res[0][3] - r2ref) < 1e-5 * r2ref
    xref, _ = full.fista(meas, iters=20, L=L)
    assert rel(cat(4), xref) < 1e-5
    assert all(abs(res[r][5] - L / 1.01) < 1e-5 * L for r in range(world))


def test_sharded_benchmark_geometry():
    """128^2 -> 256^2, 64 depths, 256 samples on 2 shards: H and H* equal the
    unsharded plan, each shard storing half of the representatives' rows."""
    import torch
    g = oracle.Grid.square(128, 64, 256)
    med = _medium(g)
    full = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, medium=med)
    world = 2
    shards = [Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, medium=med, shard=(r, world))
              for r in range(world)]
    info = shards[0].shard_info()
    rpr = info["rows_per_rank"]
    assert info["rows_total"] == 129 * 130 // 2 and rpr == (info["rows_total"] + 63) // 64 * 32
    # radial sharing among each shard's representatives: together the shards
    # store fewer rows than one per representative
    stored = [p.info()["stored_rows"] for p in shards]
    assert all(p.info()["radial"] == 1 for p in shards) and sum(stored) < info["rows_total"]
    assert all(p.info()["table_bytes"] == r * 256 * 64 * 4 for p, r in zip(shards, stored))
    # a shard's workspace: no spectra, object or data buffers, and an FFT
    # intermediate of its own 128 time samples (the full plan's holds 256)
    ws = [p.info()["workspace_bytes"] for p in shards]
    assert max(ws) < full.info()["workspace_bytes"] // 4
    ex = LocalExchange(world)
    rho = cuda(synth.vessel_phantom(g.nx, g.nz, seed=0))
    y = cuda(synth.gaussian_field((g.nt, g.ny, g.nx), seed=1))

    def rank(r):
        sop = ShardedOperator(shards[r], ex.rank(r))
        return (sop.forward(rho[r * 32:(r + 1) * 32].contiguous()),
                sop.adjoint(y[r * 128:(r + 1) * 128].contiguous()))
    res = run_ranks(world, rank)
    d = torch.cat([res[r][0] for r in range(world)])
    a = torch.cat([res[r][1] for r in range(world)])
    for got, ref in ((d, full.forward(rho)), (a, full.adjoint(y))):
        assert float((got - ref).norm() / ref.norm()) < 1e-6
