"""Frequency sharding across ranks on the CPU (gloo): ShardedOperator with
DistExchange on 2 and 4 processes. Each rank's stages are a stand-in that
follows the shard stage definitions of include/pat.h with the FP64 oracle's
library and FFTs, laid out by the library's own host partition
(pat_shard_layout); the sharded H, H*, gradient and FISTA must equal the
oracle's unsharded operator."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2603_28150_gb300 import pat, synth
from tests.helpers import MED_50UM


class OracleShardStages:
    """The shard stages of one rank in FP64 (complex128 / float64 torch tensors)."""

    def __init__(self, g, Hf, rank, world, fold):
        self.g, self.Hf = g, Hf
        self.info, self.zmap, self.tmap, _ = pat.shard_layout(
            g.nx, g.ny, g.nz, g.nt, g.px, g.py, fold, rank, world)
        i = self.info
        W = i["slot_width"]
        # bins of this rank's slots: invert the depth-side map on the owner's chunk
        own = self.zmap // (i["nz_local"] * W) == rank
        k = np.nonzero(own)[0]
        self.slot = self.zmap[k] - rank * i["nz_local"] * W
        self.kx, self.ky = k // g.py, k % g.py
        assert np.unique(self.slot).size == self.slot.size and (self.slot < W).all()

    def shard_info(self):
        return dict(self.info)

    def shard_spectrum(self, side, x):
        import torch
        g, i = self.g, self.info
        n, W = (i["nt_local"] if side else i["nz_local"]), i["slot_width"]
        m = self.tmap if side else self.zmap
        send = np.zeros(i["world"] * n * W, np.complex128)
        kx, ky = np.arange(g.px // 2 + 1)[:, None], np.arange(g.py)[None, :]
        for j in range(n):
            pad = np.zeros((g.py, g.px))
            pad[:g.ny, :g.nx] = x[j].numpy()
            F = np.fft.fft2(pad)                      # F[ky, kx], exp(-2 pi i k.n / P)
            send[j * W + m] = F[ky, kx].ravel()      # bin k = kx * py + ky
        return torch.from_numpy(send.reshape(i["world"], n, W))

    def shard_contract(self, X, adjoint=False):
        import torch
        g, W = self.g, self.info["slot_width"]
        H = self.Hf[:, :, self.ky, self.kx] / (g.px * g.py)   # [nz][nt][slots], 1/(px py) folded in
        Xn = X.numpy()
        out = np.zeros((g.nz if adjoint else g.nt, W), np.complex128)
        if adjoint:
            out[:, self.slot] = np.einsum("zts,ts->zs", np.conj(H), Xn[:, self.slot])
        else:
            out[:, self.slot] = np.einsum("zts,zs->ts", H, Xn[:, self.slot])
        return torch.from_numpy(out)

    def shard_image(self, side, recv, sub=None, resid=False):
        import torch
        g, i = self.g, self.info
        n, W = (i["nt_local"] if side else i["nz_local"]), i["slot_width"]
        m = self.tmap if side else self.zmap
        flat = recv.numpy().ravel()
        out = np.zeros((n, g.ny, g.nx))
        for j in range(n):
            half = flat[j * W + m].reshape(g.px // 2 + 1, g.py)   # [kx][ky]
            F = np.zeros((g.py, g.px), np.complex128)
            F[:, :g.px // 2 + 1] = half.T
            for kx in range(g.px // 2 + 1, g.px):                  # Hermitian extension
                F[:, kx] = np.conj(half[g.px - kx][(-np.arange(g.py)) % g.py])
            out[j] = np.real(np.fft.ifft2(F))[:g.ny, :g.nx] * (g.px * g.py)
        r2 = None
        if sub is not None:
            out = out - sub.numpy()
            r2 = float(np.sum(out * out))
        return torch.from_numpy(out), (r2 if resid else None)

    def dot(self, a, b):
        return float(np.dot(a.numpy().ravel(), b.numpy().ravel()))

    def axpby(self, y, x, a, b):
        y.copy_(__import__("torch").from_numpy(a * x.numpy() + b * y.numpy()))

    def fista_step(self, y, xprev, grad, invL, lamL, beta):
        x = np.maximum(y.numpy() - grad.numpy() * invL - lamL, 0.0)
        y.copy_(__import__("torch").from_numpy(x + beta * (x - xprev.numpy())))
        xprev.copy_(__import__("torch").from_numpy(x))


def _rank_main(rank, world, port, fold):
    import torch
    import torch.distributed as dist

    from paper_2603_28150_gb300.shard import DistExchange, ShardedOperator
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = oracle.Grid.square(8, 8, 8)          # 8^2 -> 16^2, 8 depths, 8 samples
        mz = oracle.mz_for(g.nz, g.nt, MED_50UM)
        Hf = oracle.table_kspace_closed(g, MED_50UM, mz)
        op = oracle.Operator(g, Hf=Hf)
        sop = ShardedOperator(OracleShardStages(g, Hf, rank, world, fold), DistExchange())
        zr, tr = g.nz // world, g.nt // world
        zs, ts = slice(rank * zr, (rank + 1) * zr), slice(rank * tr, (rank + 1) * tr)
        rho = synth.blobs(g.nx, g.ny, g.nz, count=3, seed=1)
        y = synth.gaussian_field((g.nt, g.ny, g.nx), seed=2)
        d = sop.forward(torch.from_numpy(rho[zs].copy())).numpy()
        ref = op.A(rho)
        assert np.abs(d - ref[ts]).max() <= 1e-12 * np.abs(ref).max()
        a = sop.adjoint(torch.from_numpy(y[ts].copy())).numpy()
        ref = op.AT(y)
        assert np.abs(a - ref[zs]).max() <= 1e-12 * np.abs(ref).max()
        meas = op.A(synth.blobs(g.nx, g.ny, g.nz, count=3, seed=3))
        grad, r2 = sop.gradient(torch.from_numpy(rho[zs].copy()), torch.from_numpy(meas[ts].copy()))
        res = op.A(rho) - meas
        assert abs(r2 - float(np.sum(res * res))) <= 1e-12 * float(np.sum(res * res))
        ref = op.AT(res)
        assert np.abs(grad.numpy() - ref[zs]).max() <= 1e-12 * np.abs(ref).max()
        v0 = synth.gaussian_field(op.obj_shape, 4)
        L_ref = oracle.power_norm(op, v0, 40)
        assert abs(sop.power_norm(torch.from_numpy(v0[zs].copy()), 40) - L_ref) <= 1e-12 * L_ref
        L = 1.01 * L_ref
        lam = 1e-3 * float(np.abs(op.AT(meas)).max())
        x, hist = sop.fista(torch.from_numpy(meas[ts].copy()), L, iters=12, lam=lam)
        ref = oracle.fista(op, meas, L, iters=12, lam=lam, track=True)
        assert np.abs(x.numpy() - ref.x[zs]).max() <= 1e-10 * np.abs(ref.x).max()
        assert np.allclose(hist, ref.resid2, rtol=1e-10)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("fold", [True, False])
def test_sharded_operator_on_gloo_ranks(world, fold):
    import torch.multiprocessing as mp
    pat.lib()       # build once here, not in every rank
    oracle.lib()
    mp.spawn(_rank_main, args=(world, _free_port(), fold), nprocs=world, join=True)


def test_shard_layout_partitions_every_bin():
    """Every bin has exactly one owner and slot; ranks hold equal 32-aligned
    row ranges covering all rows; the two maps differ only in slice counts."""
    g = oracle.Grid.square(128, 64, 256)
    for fold in (True, False):
        for world in (1, 2, 3, 8):
            if g.nz % world or g.nt % world:
                with pytest.raises(pat.PatError):
                    pat.shard_layout(g.nx, g.ny, g.nz, g.nt, g.px, g.py, fold, 0, world)
                continue
            infos = []
            seen = {}
            for r in range(world):
                info, z, t, mem = pat.shard_layout(g.nx, g.ny, g.nz, g.nt, g.px, g.py, fold, r, world)
                infos.append(info)
                W, nzr, ntr = info["slot_width"], info["nz_local"], info["nt_local"]
                assert info["rows_per_rank"] % 32 == 0 and W == (4 if fold else 1) * info["rows_per_rank"]
                q = z // (nzr * W)
                assert np.array_equal(q, t // (ntr * W))
                assert np.array_equal(z - q * nzr * W, t - q * ntr * W)
                mine = np.nonzero(q == r)[0]
                slots = z[mine] - r * nzr * W
                assert np.unique(slots).size == slots.size
                if fold:
                    assert set(mem[mem >= 0].tolist()) == set(slots.tolist())
                seen[r] = mine
            allk = np.concatenate(list(seen.values()))
            assert np.array_equal(np.sort(allk), np.arange(infos[0]["bins"]))
            assert sum(i["rows"] for i in infos) == infos[0]["rows_total"]
