"""Frequency-sharded operator over ranks: H, H*, the gradient of Eq. 15 and
FISTA (Eq. 12-14) with the table's rows split across `world` ranks.

Every rank holds an equal share of the stored operator (its rows of the
table: D4 representatives of a folded library, else bins), the depth slices
[r nz/world, (r+1) nz/world) of objects and the time samples
[r nt/world, (r+1) nt/world) of data. One application of H is
  stage i of the rank's depth slices -> all-to-all -> stage ii on the rank's
  rows -> all-to-all -> stage iii of the rank's time samples,
and H* the mirror image. The arithmetic runs in the library's shard stages
(pat_shard_*); this module only moves buffers between them through an
exchange object (torch.distributed all_to_all_single: NCCL across GPUs, gloo
on CPU) and sums the FP64 residual norms of the ranks.
"""
from __future__ import annotations

import math


class DistExchange:
    """All-to-all of equal chunks and scalar sums over a torch.distributed group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group

    def all_to_all(self, send):
        """send: contiguous [world][...]; returns recv with recv[q] = rank q's send[me]."""
        import torch
        recv = torch.empty_like(send)
        s = torch.view_as_real(send) if send.is_complex() else send
        r = torch.view_as_real(recv) if recv.is_complex() else recv
        self.dist.all_to_all_single(r, s.contiguous(), group=self.group)
        return recv

    def sum(self, value: float, device) -> float:
        import torch
        t = torch.tensor([value], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, group=self.group)
        return float(t.item())


class ShardedOperator:
    """H / H* / gradient / FISTA of one rank. `stages` is the rank's shard plan
    (paper_2603_28150_gb300.Plan(..., medium=..., shard=(rank, world))) or any
    object with the same shard_* methods and fista_step."""

    def __init__(self, stages, exchange):
        self.st = stages
        self.ex = exchange
        info = stages.shard_info()
        self.world = info["world"]
        self.rank = info["rank"]
        self.nz_r = info["nz_local"]
        self.nt_r = info["nt_local"]
        self.W = info["slot_width"]
        self.nz = self.nz_r * self.world
        self.nt = self.nt_r * self.world

    # stage ii between two exchanges: slices of this rank -> slices of this rank
    def _through(self, send, adjoint: bool):
        rows_in = self.nt if adjoint else self.nz
        rows_out_r = self.nz_r if adjoint else self.nt_r
        X = self.ex.all_to_all(send).reshape(rows_in, self.W)     # this rank's slots, all slices
        Y = self.st.shard_contract(X, adjoint=adjoint)              # [rows_out][W]
        return self.ex.all_to_all(Y.reshape(self.world, rows_out_r, self.W))

    def forward(self, rho_local):
        """d = H rho (Eq. 7-8) on this rank's slices: rho [nz/world][ny][nx] ->
        d [nt/world][ny][nx]."""
        recv = self._through(self.st.shard_spectrum(0, rho_local), adjoint=False)
        return self.st.shard_image(1, recv)[0]

    def adjoint(self, d_local):
        """rho = H* d (Eq. 11): d [nt/world][ny][nx] -> rho [nz/world][ny][nx]."""
        recv = self._through(self.st.shard_spectrum(1, d_local), adjoint=True)
        return self.st.shard_image(0, recv)[0]

    def gradient(self, x_local, y_local):
        """(H*(H x - y) of this rank's depth slices, ||H x - y||^2 over all ranks)
        (Eq. 15); the residual stays on this rank's time samples."""
        recv = self._through(self.st.shard_spectrum(0, x_local), adjoint=False)
        r, r2 = self.st.shard_image(1, recv, sub=y_local, resid=True)
        r2 = self.ex.sum(r2, device=r.device)
        recv = self._through(self.st.shard_spectrum(1, r), adjoint=True)
        return self.st.shard_image(0, recv)[0], r2

    def dot(self, a_local, b_local) -> float:
        """<a, b> over all ranks (FP64 products and sums on each rank)."""
        return self.ex.sum(self.st.dot(a_local, b_local), device=a_local.device)

    def power_norm(self, v0_local, iters: int) -> float:
        """L = ||H*H|| by power iteration from v0 (this rank's depth slices of
        the start vector): v <- H*H v / ||H*H v||, norms over all ranks."""
        v = v0_local.clone()
        self.st.axpby(v, v, 1.0 / math.sqrt(self.dot(v, v)), 0.0)
        L = 0.0
        for _ in range(iters):
            w = self.adjoint(self.forward(v))
            L = math.sqrt(self.dot(w, w))
            self.st.axpby(w, w, 1.0 / L, 0.0)
            v = w
        return L

    def fista(self, y_local, L: float, iters: int, lam: float = 0.0, x0=None):
        """FISTA with constant step 1/L (Eq. 12-14, Beck & Teboulle): y_1 = x_0,
        t_1 = 1; x_k = max(y_k - grad/L - lam/L, 0); t_{k+1} = (1 + sqrt(1 +
        4 t_k^2)) / 2; y_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1}).
        Returns (x_iters of this rank's depth slices, residual norms ||H y_k - y||^2)."""
        import torch
        shape = (self.nz_r,) + tuple(y_local.shape[1:])
        xprev = (torch.zeros(shape, dtype=y_local.dtype, device=y_local.device) if x0 is None
                 else x0.clone())
        yk = xprev.clone()
        t, hist = 1.0, []
        for _ in range(iters):
            g, r2 = self.gradient(yk, y_local)
            hist.append(r2)
            t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
            self.st.fista_step(yk, xprev, g, 1.0 / L, lam / L, (t - 1.0) / t_next)
            t = t_next
        return xprev, hist
