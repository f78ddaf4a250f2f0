"""Seeded synthetic inputs: phantoms, noise, random kernels, start vectors.

This module holds none of the operator's arithmetic. It only draws numbers
(numpy ``default_rng``) and rasterises simple shapes, so the CPU oracle and the
CUDA path can be fed identical inputs. Shapes follow the paper's datasets:
sparse point-like absorbers (bead phantoms) and tubular vessels (wire phantom,
forearm vasculature) on isotropic voxels, a few tens of depths (Sec. 3.3-3.4).

Arrays are float64, row-major with x fastest: objects [nz][ny][nx].
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def _add_gaussian(vol: np.ndarray, centre, sigma: float, amp: float) -> None:
    nz, ny, nx = vol.shape
    r = int(np.ceil(4 * sigma))
    cz, cy, cx = centre
    z0, z1 = max(0, int(cz) - r), min(nz, int(cz) + r + 2)
    y0, y1 = max(0, int(cy) - r), min(ny, int(cy) + r + 2)
    x0, x1 = max(0, int(cx) - r), min(nx, int(cx) + r + 2)
    if z0 >= z1 or y0 >= y1 or x0 >= x1:
        return
    zz, yy, xx = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1),
                             indexing="ij")
    d2 = (zz - cz) ** 2 + (yy - cy) ** 2 + (xx - cx) ** 2
    vol[z0:z1, y0:y1, x0:x1] += amp * np.exp(-d2 / (2.0 * sigma * sigma))


def blobs(nx: int, ny: int, nz: int, count: int, seed: int = 0) -> np.ndarray:
    """Sum of `count` isotropic Gaussians: sigma ~ U[1, 3] voxels, amplitude
    ~ U[0.5, 1], centres uniform at least 3 sigma inside the volume where the
    volume allows it (else uniform over the volume)."""
    g = rng(seed)
    vol = np.zeros((nz, ny, nx))
    for _ in range(count):
        sigma = g.uniform(1.0, 3.0)
        amp = g.uniform(0.5, 1.0)
        c = []
        for n in (nz, ny, nx):
            m = 3.0 * sigma
            lo, hi = (m, n - 1 - m) if n - 1 - 2 * m > 0 else (0.0, n - 1.0)
            c.append(g.uniform(lo, hi))
        _add_gaussian(vol, c, sigma, amp)
    return vol


def vessels(nx: int, ny: int, nz: int, tubes: int, seed: int = 0, steps: int | None = None,
            blob_count: int = 0) -> np.ndarray:
    """Random-walk tubes plus optional blobs. Each tube starts uniformly in the
    volume and takes `steps` (default 4 max(nx, ny)) unit steps; the direction
    keeps its persistence by adding N(0, 0.15^2) per component and
    renormalising. Radius ~ U{1..4} voxels, amplitude ~ U[0.5, 1]; a voxel takes
    the maximum over tubes. Walks are clipped to the volume."""
    g = rng(seed)
    steps = 4 * max(nx, ny) if steps is None else steps
    vol = np.zeros((nz, ny, nx))
    dims = np.array([nz, ny, nx], dtype=np.float64)
    for _ in range(tubes):
        p = g.uniform(0.0, 1.0, 3) * (dims - 1)
        v = g.normal(0.0, 1.0, 3)
        v /= np.linalg.norm(v)
        rad = int(g.integers(1, 5))
        amp = g.uniform(0.5, 1.0)
        for _ in range(steps):
            lo = np.maximum(np.floor(p - rad).astype(int), 0)
            hi = np.minimum(np.ceil(p + rad).astype(int) + 1, dims.astype(int))
            if np.all(hi > lo):
                zz, yy, xx = np.meshgrid(np.arange(lo[0], hi[0]), np.arange(lo[1], hi[1]),
                                         np.arange(lo[2], hi[2]), indexing="ij")
                inside = (zz - p[0]) ** 2 + (yy - p[1]) ** 2 + (xx - p[2]) ** 2 <= rad * rad
                sub = vol[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
                np.maximum(sub, np.where(inside, amp, 0.0), out=sub)
            v = v + g.normal(0.0, 0.15, 3)
            v /= np.linalg.norm(v)
            p = np.clip(p + v, 0.0, dims - 1)
    if blob_count:
        vol += blobs(nx, ny, nz, blob_count, seed=seed + 7919)
    return vol


def vessel_phantom(n: int, nz: int, seed: int = 0) -> np.ndarray:
    """The headline phantom: n/16 tubes + n/16 blobs on an n x n x nz grid."""
    k = max(1, n // 16)
    return vessels(n, n, nz, tubes=k, seed=seed, blob_count=k)


def gaussian_object(nx: int, ny: int, nz: int, seed: int = 0) -> np.ndarray:
    """I.i.d. N(0, 1) voxels: the random test objects of the forward-model check."""
    return rng(seed).normal(0.0, 1.0, (nz, ny, nx))


def gaussian_field(shape, seed: int = 0) -> np.ndarray:
    """I.i.d. N(0, 1) array of any shape (noise, start vectors, adjoint tests)."""
    return rng(seed).normal(0.0, 1.0, shape)


def random_kernels(nz: int, nt: int, px: int, py: int, seed: int = 0,
                   even: bool = False, d4: bool = False) -> np.ndarray:
    """A random spatial kernel library h[nz][nt][py][px] (wrapped origin),
    U[-1, 1]. With even=True every plane satisfies h(-u) = h(u) (index
    negation modulo the padded size), i.e. its spectrum is real. With d4=True
    (px == py) every plane is the average of its 8 images under the square's
    symmetries (ux -> -ux, uy -> -uy, ux <-> uy), like a radially symmetric
    kernel: its spectrum is real and depends on {|kx|, |ky|} only."""
    h = rng(seed).uniform(-1.0, 1.0, (nz, nt, py, px))
    if even or d4:
        iy = (-np.arange(py)) % py
        ix = (-np.arange(px)) % px
        h = 0.5 * (h + h[:, :, iy][:, :, :, ix])
    if d4:
        assert px == py, "the square's symmetries need px == py"
        h = 0.5 * (h + h[:, :, iy])            # uy -> -uy
        h = 0.5 * (h + np.swapaxes(h, 2, 3))   # ux <-> uy
    return h


def timing_spectra(nz: int, nt: int, py: int, px: int, seed: int = 0) -> np.ndarray:
    """A complex128 [nz][nt][py][px] array filled quickly (a random plane scaled
    by a random factor per (j, t)): shape-correct filler for timing runs whose
    cost does not depend on the values."""
    g = rng(seed)
    base = g.uniform(-1, 1, (py, px)) + 1j * g.uniform(-1, 1, (py, px))
    scale = g.uniform(0.5, 1.0, (nz, nt))
    out = np.empty((nz, nt, py, px), dtype=np.complex128)
    for j in range(nz):
        np.multiply(scale[j][:, None, None], base[None], out=out[j])
    return out


def splitmix_uniform(n: int, seed: int) -> np.ndarray:
    """n values 2 u_i - 1 in [-1, 1), u_i = (splitmix64(seed + (i + 1) * gamma) >> 11) * 2^-53,
    gamma = 0x9E3779B97F4A7C15: the counter-based generator of Steele, Lea &
    Flood ("Fast splittable pseudorandom number generators", 2014), written
    from its published definition (the device fills the power iteration's
    seeded start vector with the same sequence)."""
    m64 = np.uint64(0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        z = (np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
             + np.uint64(0x9E3779B97F4A7C15) * np.arange(1, n + 1, dtype=np.uint64)) & m64
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0) * 2.0 - 1.0
