"""Iterative parts of the oracle, in plain numpy FP64 (TEST INFRASTRUCTURE ONLY).

- ``fista``: Beck & Teboulle's FISTA with constant step 1/L for Eq. 12
  (f + g, f of Eq. 13, g of Eq. 14), gradient of Eq. 15.
- ``power_norm``: power iteration for L = ||H*H||_2, the Lipschitz constant of
  the gradient of f (not printed in the paper; FISTA needs it).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


class Operator:
    """H and H* of one geometry, from the oracle's FFT form (default) or the
    direct spatial form of Eq. 7 / Eq. 11. With ``sampling = (sx, sy, ox, oy)``
    the pair is S H and H* S^T, S the measurement operator that keeps the scan
    positions (Sec. 2.3, Sec. 3.3)."""

    def __init__(self, grid, Hf=None, h=None, form: str = "fft", sampling=None):
        from . import adjoint_fft, adjoint_spatial, forward_fft, forward_spatial, table_spectrum
        self.g = grid
        if form == "fft":
            Hf = table_spectrum(h) if Hf is None else Hf
            self._A = lambda x: forward_fft(Hf, x, grid)
            self._AT = lambda y: adjoint_fft(Hf, y, grid)
        elif form == "spatial":
            assert h is not None, "the spatial form needs the spatial table"
            self._A = lambda x: forward_spatial(h, x, grid)
            self._AT = lambda y: adjoint_spatial(h, y, grid)
        else:
            raise ValueError(form)
        self.sampling = tuple(sampling) if sampling is not None else None

    @property
    def obj_shape(self):
        return (self.g.nz, self.g.ny, self.g.nx)

    @property
    def data_shape(self):
        if self.sampling is None:
            return (self.g.nt, self.g.ny, self.g.nx)
        from . import scan_positions
        sx, sy, ox, oy = self.sampling
        return (self.g.nt, len(scan_positions(self.g.ny, sy, oy)),
                len(scan_positions(self.g.nx, sx, ox)))

    def A(self, x):
        d = self._A(x)
        if self.sampling is None:
            return d
        from . import sample_scan
        return sample_scan(d, *self.sampling)

    def AT(self, y):
        if self.sampling is not None:
            from . import zero_fill
            y = zero_fill(y, self.g.ny, self.g.nx, *self.sampling)
        return self._AT(y)


def power_norm(op: Operator, v0, iters: int) -> float:
    """Power iteration on H*H from the start vector v0 (normalised first):
    v <- H*H v / ||H*H v||; returns ||H*H v|| of the last step."""
    v = np.asarray(v0, np.float64)
    v = v / np.linalg.norm(v.ravel())
    L = 0.0
    for _ in range(iters):
        w = op.AT(op.A(v))
        L = float(np.linalg.norm(w.ravel()))
        v = w / L
    return L


@dataclass
class FistaResult:
    x: np.ndarray
    objective: list = field(default_factory=list)   # F(x_k) = f(x_k) + g(x_k)
    resid2: list = field(default_factory=list)      # ||H y_k - d||^2 of each gradient step
    t: list = field(default_factory=list)           # t_1, t_2, ... of the momentum recurrence


def prox_g(v, step: float, lam: float):
    """prox of step * g with g = lam ||.||_1 + indicator(x >= 0) (Eq. 14):
    the minimiser of ||x - v||^2 / 2 + step lam ||x||_1 over x >= 0 is
    max(v - step lam, 0) componentwise."""
    return np.maximum(v - step * lam, 0.0)


def next_t(t: float) -> float:
    """Beck & Teboulle's momentum parameter: t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2."""
    return (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0


def momentum(t: float, t_next: float) -> float:
    """Extrapolation weight of y_{k+1} = x_k + beta_k (x_k - x_{k-1}):
    beta_k = (t_k - 1) / t_{k+1}."""
    return (t - 1.0) / t_next


def fista(op: Operator, d, L: float, iters: int, lam: float = 0.0, x0=None,
          track: bool = False) -> FistaResult:
    """FISTA with constant step 1/L (Beck & Teboulle 2009):
        y_1 = x_0, t_1 = 1
        x_k     = prox_{g/L}(y_k - grad f(y_k) / L),  grad f = H*(H y - d)   (Eq. 15)
        t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
        y_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1})
    x_0 = 0 unless given. Returns x_iters (and, with track, F(x_k) and the
    residual norms of the gradient steps and t_1 .. t_{iters+1})."""
    d = np.asarray(d, np.float64)
    x_prev = np.zeros(op.obj_shape) if x0 is None else np.asarray(x0, np.float64).copy()
    y = x_prev.copy()
    t = 1.0
    out = FistaResult(x=x_prev)
    if track:
        out.t.append(t)
    for _ in range(iters):
        r = op.A(y) - d
        grad = op.AT(r)
        x = prox_g(y - grad / L, 1.0 / L, lam)
        t_next = next_t(t)
        y = x + momentum(t, t_next) * (x - x_prev)
        if track:
            out.t.append(float(t_next))
            out.resid2.append(float(np.dot(r.ravel(), r.ravel())))
            rx = op.A(x) - d
            out.objective.append(0.5 * float(np.dot(rx.ravel(), rx.ravel()))
                                 + lam * float(np.abs(x).sum()))
        x_prev, t = x, t_next
    out.x = x_prev
    return out
