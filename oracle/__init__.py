"""CPU oracle for the planar PAT operator (FP64).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the product package. It shares no
code with the CUDA path.

The heavy operators are plain C++ (``pat_oracle.cpp``); this module marshals
numpy arrays to them and adds the iterative parts written in numpy:
  - FISTA (Beck & Teboulle) for Eq. 12-14 with the gradient of Eq. 15,
  - power iteration for the Lipschitz constant ||H*H||,
  - the paper's relative l2 / l-infinity error metrics (Sec. 3.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pat_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "libpat_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C++ oracle into oracle/_build/libpat_oracle.so (g++ -O2)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    newer = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pat_oracle.h")))
    if force or not newer:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                        _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Medium(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("dt", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L, D, P = ctypes.c_long, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long)
        I = ctypes.c_int
        sig = {
            "orc_fft1d": [D, L, I], "orc_dft1d": [D, D, L, I],
            "orc_fft2d": [D, L, L, I], "orc_fft3d": [D, L, L, L, I],
            "orc_forward_spatial": [D, D, D, L, L, L, L, L, L],
            "orc_adjoint_spatial": [D, D, D, L, L, L, L, L, L],
            "orc_table_spectrum": [D, D, L, L, L, L],
            "orc_forward_fft": [D, D, D, L, L, L, L, L, L],
            "orc_adjoint_fft": [D, D, D, L, L, L, L, L, L],
            "orc_kspace_solve": [D, L, L, L, _Medium, L, I, P, L, D],
            "orc_table_kspace_solve": [L, L, L, _Medium, L, L, L, L, I, D],
            "orc_table_kspace_closed": [L, L, L, _Medium, L, P, L, P, L, D],
        }
        for name, args in sig.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _lib.orc_set_threads.argtypes = [I]
        _lib.orc_get_threads.restype = I
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "need C-contiguous float64"
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------- FFT
def fft1d(x, inverse: bool = False) -> np.ndarray:
    a = _c128(x).copy()
    _check(lib().orc_fft1d(_dptr(a.view(np.float64)), a.size, int(inverse)), "fft1d")
    return a


def dft1d(x, inverse: bool = False) -> np.ndarray:
    a = _c128(x)
    out = np.empty_like(a)
    _check(lib().orc_dft1d(_dptr(a.view(np.float64)), _dptr(out.view(np.float64)),
                           a.size, int(inverse)), "dft1d")
    return out


def fft2d(x, inverse: bool = False) -> np.ndarray:
    a = _c128(x).copy()
    _check(lib().orc_fft2d(_dptr(a.view(np.float64)), a.shape[0], a.shape[1],
                           int(inverse)), "fft2d")
    return a


def fft3d(x, inverse: bool = False) -> np.ndarray:
    a = _c128(x).copy()
    _check(lib().orc_fft3d(_dptr(a.view(np.float64)), *a.shape, int(inverse)), "fft3d")
    return a


# ----------------------------------------------------------------------------- operator
@dataclass(frozen=True)
class Grid:
    """Transverse grid n x n (nx, ny), padded grid px x py, depths nz, samples nt."""
    nx: int
    ny: int
    nz: int
    nt: int
    px: int
    py: int

    @staticmethod
    def square(n: int, nz: int, nt: int, pad: int | None = None) -> "Grid":
        """Square grid; the padded size defaults to the power of two >= 2n."""
        p = pad
        if p is None:
            p = 1
            while p < 2 * n:
                p *= 2
        return Grid(n, n, nz, nt, p, p)

    def dims(self):
        return (self.nx, self.ny, self.nz, self.nt, self.px, self.py)


def forward_spatial(h, rho, g: Grid) -> np.ndarray:
    """Eq. 7 as written: d[t] = sum_j h[j][t] (*) rho[j] (transverse convolution)."""
    h, rho = _f64(h), _f64(rho)
    assert h.shape == (g.nz, g.nt, g.py, g.px) and rho.shape == (g.nz, g.ny, g.nx)
    d = np.empty((g.nt, g.ny, g.nx))
    _check(lib().orc_forward_spatial(_dptr(h), _dptr(rho), _dptr(d), *g.dims()), "forward_spatial")
    return d


def adjoint_spatial(h, d, g: Grid) -> np.ndarray:
    """Eq. 11 as written: rho[j] = sum_t h[j][t] (correlated with) d[t]."""
    h, d = _f64(h), _f64(d)
    assert h.shape == (g.nz, g.nt, g.py, g.px) and d.shape == (g.nt, g.ny, g.nx)
    rho = np.empty((g.nz, g.ny, g.nx))
    _check(lib().orc_adjoint_spatial(_dptr(h), _dptr(d), _dptr(rho), *g.dims()), "adjoint_spatial")
    return rho


def table_spectrum(h) -> np.ndarray:
    """Full-plane spectra Hf[j][t] = DFT2(h[j][t]), complex128 [nz][nt][py][px]."""
    h = _f64(h)
    Hf = np.empty(h.shape, dtype=np.complex128)
    _check(lib().orc_table_spectrum(_dptr(h), _dptr(Hf.view(np.float64)), *h.shape[:2],
                                    h.shape[3], h.shape[2]), "table_spectrum")
    return Hf


def forward_fft(Hf, rho, g: Grid) -> np.ndarray:
    """Zero-padded FFT realisation of Eq. 7."""
    Hf, rho = _c128(Hf), _f64(rho)
    assert Hf.shape == (g.nz, g.nt, g.py, g.px) and rho.shape == (g.nz, g.ny, g.nx)
    d = np.empty((g.nt, g.ny, g.nx))
    _check(lib().orc_forward_fft(_dptr(Hf.view(np.float64)), _dptr(rho), _dptr(d), *g.dims()),
           "forward_fft")
    return d


def adjoint_fft(Hf, d, g: Grid) -> np.ndarray:
    """Zero-padded FFT realisation of Eq. 11."""
    Hf, d = _c128(Hf), _f64(d)
    assert Hf.shape == (g.nz, g.nt, g.py, g.px) and d.shape == (g.nt, g.ny, g.nx)
    rho = np.empty((g.nz, g.ny, g.nx))
    _check(lib().orc_adjoint_fft(_dptr(Hf.view(np.float64)), _dptr(d), _dptr(rho), *g.dims()),
           "adjoint_fft")
    return rho


# ----------------------------------------------------------------------------- sensor response
def apply_sensor_response(h, r) -> np.ndarray:
    """Kernels with the sensors' temporal impulse response folded in (Sec. 2:
    identical, spatially invariant sensor responses incorporated into the
    kernels by temporal convolution): h'[z][t] = sum_{tau <= t} r[tau] h[z][t - tau]
    over the recorded samples t < nt (causal, r[0] at lag 0), for every
    transverse position. h: [nz][nt][py][px]."""
    h, r = _f64(h), _f64(r).ravel()
    nt = h.shape[1]
    out = np.zeros_like(h)
    for t in range(nt):
        for tau in range(min(len(r), t + 1)):
            out[:, t] += r[tau] * h[:, t - tau]
    return out


# ----------------------------------------------------------------------------- measurement
def scan_positions(n: int, step: int, offset: int) -> list:
    """Sensor-grid indices of one scan axis: offset, offset + step, ... < n
    (Sec. 3.3: the scan grid is coarser than the reconstruction grid)."""
    assert step >= 1 and 0 <= offset < n
    out, c = [], offset
    while c < n:
        out.append(c)
        c += step
    return out


def sample_scan(d, sx: int, sy: int, ox: int, oy: int) -> np.ndarray:
    """S of the measurement operator composed with H (Sec. 2.3, Sec. 3.3):
    keeps the samples at the scan positions x = ox + sx i, y = oy + sy j of
    every [ny][nx] plane of d (leading axes untouched)."""
    d = _f64(d)
    xs = scan_positions(d.shape[-1], sx, ox)
    ys = scan_positions(d.shape[-2], sy, oy)
    out = np.empty(d.shape[:-2] + (len(ys), len(xs)))
    for j, y in enumerate(ys):
        for i, x in enumerate(xs):
            out[..., j, i] = d[..., y, x]
    return out


def zero_fill(ds, ny: int, nx: int, sx: int, sy: int, ox: int, oy: int) -> np.ndarray:
    """S^T: places scan-grid samples ds[..., my, mx] at their sensor positions
    of an [ny][nx] plane and zeros everywhere else."""
    ds = _f64(ds)
    xs = scan_positions(nx, sx, ox)
    ys = scan_positions(ny, sy, oy)
    assert ds.shape[-2:] == (len(ys), len(xs))
    out = np.zeros(ds.shape[:-2] + (ny, nx))
    for j, y in enumerate(ys):
        for i, x in enumerate(xs):
            out[..., y, x] = ds[..., j, i]
    return out


# ----------------------------------------------------------------------------- physics
@dataclass(frozen=True)
class Medium:
    c: float = 1500.0
    dx: float = 100e-6
    dy: float = 100e-6
    dz: float = 100e-6
    dt: float = 20e-9

    def _c(self) -> _Medium:
        return _Medium(self.c, self.dx, self.dy, self.dz, self.dt)


def mz_for(nz: int, nt: int, med: Medium, z0: int = 1) -> int:
    """Depth extent of the periodic solve: the next power of two holding the
    object depths plus the distance sound travels in nt samples (wrap-free)."""
    need = z0 + nz + int(np.ceil(med.c * nt * med.dt / med.dz)) + 1
    m = 1
    while m < need:
        m *= 2
    return m


def kspace_solve(p0, med: Medium, nt: int, planes, closed_form: bool = False) -> np.ndarray:
    """Eq. 1-2 on the periodic grid of p0 [mz][py][px]; records [len(planes)][nt][py][px]."""
    p0 = _f64(p0)
    planes = np.ascontiguousarray(planes, dtype=np.int64)
    mz, py, px = p0.shape
    rec = np.empty((planes.size, nt, py, px))
    _check(lib().orc_kspace_solve(_dptr(p0), px, py, mz, med._c(), nt, int(closed_form),
                                  _lptr(planes), planes.size, _dptr(rec)), "kspace_solve")
    return rec


def table_kspace_solve(g: Grid, med: Medium, mz: int, z0: int = 1, src_plane: int = 0,
                       sign: int = 1) -> np.ndarray:
    """Spatial library h[nz][nt][py][px] from one point-source solve (reciprocity)."""
    h = np.empty((g.nz, g.nt, g.py, g.px))
    _check(lib().orc_table_kspace_solve(g.px, g.py, mz, med._c(), g.nt, g.nz, z0, src_plane,
                                        sign, _dptr(h)), "table_kspace_solve")
    return h


def table_kspace_closed(g: Grid, med: Medium, mz: int, z0: int = 1, t_idx=None,
                        z_idx=None) -> np.ndarray:
    """Closed-form spectrum of the same library for the listed (t, j) (default: all)."""
    t_idx = np.arange(g.nt) if t_idx is None else np.asarray(t_idx)
    z_idx = np.arange(g.nz) if z_idx is None else np.asarray(z_idx)
    t_idx = np.ascontiguousarray(t_idx, dtype=np.int64)
    z_idx = np.ascontiguousarray(z_idx, dtype=np.int64)
    Hf = np.empty((z_idx.size, t_idx.size, g.py, g.px), dtype=np.complex128)
    _check(lib().orc_table_kspace_closed(g.px, g.py, mz, med._c(), z0, _lptr(t_idx), t_idx.size,
                                         _lptr(z_idx), z_idx.size, _dptr(Hf.view(np.float64))),
           "table_kspace_closed")
    return Hf


# ----------------------------------------------------------------------------- metrics
def rel_l2(a, b) -> float:
    """||a - b||_2 / ||b||_2 (Sec. 3.1), in FP64."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def rel_linf(a, b) -> float:
    """||a - b||_inf / ||b||_inf (Sec. 3.1), in FP64."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


from .solvers import Operator, fista, power_norm  # noqa: E402,F401
