"""Python binding of libpat (include/pat.h): argument marshalling only.

Every computation runs in the CUDA kernels of libpat.so; this module passes
pointers, sizes and the current torch CUDA stream through ctypes. There is no
CPU fallback: if the library or a GPU is missing, the calls raise.

Arrays are torch tensors: CUDA tensors are used in place (asynchronous on the
current stream); CPU tensors / numpy arrays are host buffers that the library
stages through the device (synchronous). Shapes, x fastest:
  object rho [batch][nz][ny][nx] (or [nz][ny][nx]); data d [batch][nt][ny][nx].
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

PAT_OK = 0
PAT_ERR_ARG = -1
PAT_ERR_OOM = -2
PAT_ERR_CUDA = -3
PAT_ERR_TIMEOUT = -4
PAT_ERR_UNSUPPORTED = -5

FLAG_FP64 = 1
FLAG_FORCE_COMPLEX = 2
FLAG_BF16_SPLIT = 4
FLAG_NO_FOLD = 8
FLAG_NO_RADIAL = 16

TABLE_SPATIAL_F64 = 0
TABLE_SPATIAL_F32 = 1
TABLE_SPECTRAL_C128 = 2
TABLE_SPECTRAL_C64 = 3

# Every symbol include/pat.h declares.
EXPORTS = (
    "pat_plan_create", "pat_plan_create_kspace", "pat_plan_destroy", "pat_plan_info",
    "pat_last_error", "pat_forward", "pat_adjoint", "pat_gradient", "pat_power_norm",
    "pat_fista_solve", "pat_dot_f64", "pat_stage_spectrum", "pat_stage_image",
    "pat_stage_contract", "pat_spectrum_noalloc", "pat_plan_estimate", "pat_slot_load",
    "pat_slot_move", "pat_slots_step", "pat_slot_read", "pat_plan_set_tensor_batch",
    "pat_plan_check", "pat_plan_set_sampling", "pat_plan_set_sensor_response",
    "pat_workspace_size", "pat_plan_create_with_workspace", "pat_plan_create_kspace_with_workspace",
    "pat_plan_set_wait_limit", "pat_debug_live_allocations", "pat_power_norm_seed",
    "pat_shard_layout", "pat_plan_create_kspace_shard", "pat_plan_shard_info",
    "pat_shard_spectrum", "pat_shard_contract", "pat_shard_image", "pat_fista_step",
    "pat_axpby", "pat_stage_contract_slots", "pat_fold_blocks",
)

WAIT_LIMIT_DEFAULT = 4194304


class PatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libpat error {code}: {msg}")
        self.code = code


class Geometry(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("nt", ctypes.c_int32), ("px", ctypes.c_int32), ("py", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("flags", ctypes.c_int32)]


class MediumC(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("dt", ctypes.c_double), ("mz", ctypes.c_int32),
                ("z0", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("real_table", ctypes.c_int32), ("fp64", ctypes.c_int32),
                ("bins", ctypes.c_int64), ("bins_padded", ctypes.c_int64),
                ("table_bytes", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64), ("table_max_abs", ctypes.c_double),
                ("table_max_imag", ctypes.c_double), ("tensor_table_bytes", ctypes.c_int64),
                ("tensor_min_batch", ctypes.c_int32), ("folded", ctypes.c_int32),
                ("table_rows", ctypes.c_int64), ("workspace_external", ctypes.c_int32),
                ("radial", ctypes.c_int32), ("stored_rows", ctypes.c_int64)]


class ShardInfo(ctypes.Structure):
    _fields_ = [("world", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("nz_local", ctypes.c_int32), ("nt_local", ctypes.c_int32),
                ("folded", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rows_total", ctypes.c_int64), ("rows_per_rank", ctypes.c_int64),
                ("row0", ctypes.c_int64), ("rows", ctypes.c_int64),
                ("slot_width", ctypes.c_int64), ("bins", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class FistaParams(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("power_iters", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("lam", ctypes.c_double), ("L", ctypes.c_double)]


class FistaReport(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("resid2_first", ctypes.c_double),
                ("resid2_last", ctypes.c_double), ("iters", ctypes.c_int32),
                ("kernels_per_iter", ctypes.c_int32)]


_lib = None


def lib(build_if_missing: bool = True):
    """Loads libpat.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libpat.so not found at {path}; run paper_2603_28150_gb300/build.py")
    L = ctypes.CDLL(path)
    P, I, V, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    sig = {
        "pat_plan_create": ([ctypes.POINTER(Geometry), V, I, P, ctypes.POINTER(P)], I),
        "pat_plan_create_kspace": ([ctypes.POINTER(Geometry), ctypes.POINTER(MediumC), P,
                                    ctypes.POINTER(P)], I),
        "pat_plan_destroy": ([P], I),
        "pat_plan_info": ([P, ctypes.POINTER(PlanInfo)], I),
        "pat_last_error": ([], ctypes.c_char_p),
        "pat_forward": ([P, V, V, I, P], I),
        "pat_adjoint": ([P, V, V, I, P], I),
        "pat_gradient": ([P, V, V, V, I, D, P], I),
        "pat_power_norm": ([P, V, I, D, P], I),
        "pat_fista_solve": ([P, V, V, I, ctypes.POINTER(FistaParams), ctypes.POINTER(FistaReport),
                             P], I),
        "pat_dot_f64": ([P, V, V, ctypes.c_int64, D, P], I),
        "pat_stage_spectrum": ([P, V, V, I, P], I),
        "pat_stage_image": ([P, V, V, I, P], I),
        "pat_stage_contract": ([P, V, V, I, I, P], I),
        "pat_spectrum_noalloc": ([V, I, I, I, I, I, V, P], I),
        "pat_plan_estimate": ([ctypes.POINTER(Geometry), I, ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int64)], I),
        "pat_slot_load": ([P, I, V, ctypes.c_double, ctypes.c_double, P], I),
        "pat_slot_move": ([P, I, I, P], I),
        "pat_slots_step": ([P, I, ctypes.POINTER(ctypes.c_int), P], I),
        "pat_slot_read": ([P, I, V, D, P], I),
        "pat_plan_set_tensor_batch": ([P, I], I),
        "pat_plan_check": ([P], I),
        "pat_plan_set_sampling": ([P, I, I, I, I], I),
        "pat_plan_set_sensor_response": ([P, D, I, P], I),
        "pat_workspace_size": ([ctypes.POINTER(Geometry)], ctypes.c_int64),
        "pat_plan_create_with_workspace": ([ctypes.POINTER(Geometry), V, I, V, ctypes.c_size_t, P,
                                            ctypes.POINTER(P)], I),
        "pat_plan_create_kspace_with_workspace": ([ctypes.POINTER(Geometry), ctypes.POINTER(MediumC),
                                                   V, ctypes.c_size_t, P, ctypes.POINTER(P)], I),
        "pat_plan_set_wait_limit": ([P, ctypes.c_int64], I),
        "pat_debug_live_allocations": ([], ctypes.c_int64),
        "pat_power_norm_seed": ([P, I, ctypes.c_uint64, D, P], I),
        "pat_shard_layout": ([ctypes.POINTER(Geometry), I, I, I, ctypes.POINTER(ShardInfo), V, V, V], I),
        "pat_fold_blocks": ([I, I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                             V, V, V, V], I),
        "pat_plan_create_kspace_shard": ([ctypes.POINTER(Geometry), ctypes.POINTER(MediumC), I, I, P,
                                          ctypes.POINTER(P)], I),
        "pat_plan_shard_info": ([P, ctypes.POINTER(ShardInfo)], I),
        "pat_shard_spectrum": ([P, I, V, V, P], I),
        "pat_shard_contract": ([P, I, V, V, P], I),
        "pat_shard_image": ([P, I, V, V, V, D, P], I),
        "pat_fista_step": ([V, V, V, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, P], I),
        "pat_axpby": ([V, V, ctypes.c_int64, ctypes.c_double, ctypes.c_double, P], I),
        "pat_stage_contract_slots": ([P, V, V, I, I, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(rc: int) -> None:
    if rc != PAT_OK:
        raise PatError(rc, lib().pat_last_error().decode())


def _torch():
    import torch
    return torch


def _stream(stream=None) -> int:
    torch = _torch()
    if stream is not None:
        return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
    if torch.cuda.is_available():
        return int(torch.cuda.current_stream().cuda_stream)
    return 0


def _need(a, n: int, dtype, what: str) -> None:
    """Raises ValueError unless `a` holds exactly n elements of numpy dtype
    `dtype`: the C ABI takes raw pointers and sizes, so a short or wrongly
    typed buffer would be read or written past its end."""
    m = int(np.prod(a.shape))
    dt = a.dtype if isinstance(a, np.ndarray) else _np_dtype(a.dtype)
    if m != n or dt != np.dtype(dtype):
        raise ValueError(f"{what}: expected {n} elements of {np.dtype(dtype).name}, "
                         f"got {m} of {dt}")


def _ptr(a) -> int:
    """Data pointer of a contiguous torch tensor or numpy array."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "numpy array must be C-contiguous"
        return a.ctypes.data
    assert a.is_contiguous(), "tensor must be contiguous"
    return a.data_ptr()


@dataclass(frozen=True)
class Medium:
    """Homogeneous medium of a device-generated k-space library (see pat_medium)."""
    c: float = 1500.0
    dx: float = 100e-6
    dy: float = 100e-6
    dz: float = 100e-6
    dt: float = 20e-9
    mz: int = 64
    z0: int = 1

    def c_struct(self) -> MediumC:
        return MediumC(self.c, self.dx, self.dy, self.dz, self.dt, self.mz, self.z0)


class Plan:
    """A resident operator: grid + impulse-response library on the device.

    Build from a table (`table` = spatial h[nz][nt][py][px] real or spectral
    Hh[nz][nt][py][px//2+1] complex; numpy / torch, host or device) or from a
    `medium` (library generated on the device from the k-space solution).
    `workspace`: optional caller-owned CUDA tensor of at least
    workspace_size(...) bytes (e.g. torch.empty(n, dtype=torch.uint8,
    device="cuda")) that holds every per-call buffer of the plan; the plan keeps
    a reference to it and never frees it."""

    def __init__(self, nx: int, ny: int, nz: int, nt: int, px: int | None = None,
                 py: int | None = None, max_batch: int = 1, fp64: bool = False,
                 force_complex: bool = False, table=None, medium: Medium | None = None,
                 bf16_split: bool = False, fold: bool = True, stream=None, workspace=None,
                 shard: tuple | None = None, radial: bool = True):
        L = lib()
        self.nx, self.ny, self.nz, self.nt = nx, ny, nz, nt
        self.mx, self.my = nx, ny          # scan grid of the data (see set_sampling)
        self.sampling = (1, 1, 0, 0)
        self.px = px if px is not None else _pow2_at_least(2 * nx)
        self.py = py if py is not None else _pow2_at_least(2 * ny)
        self.max_batch = max_batch
        self.fp64 = fp64
        flags = ((FLAG_FP64 if fp64 else 0) | (FLAG_FORCE_COMPLEX if force_complex else 0)
                 | (FLAG_BF16_SPLIT if bf16_split else 0) | (0 if fold else FLAG_NO_FOLD)
                 | (0 if radial else FLAG_NO_RADIAL))
        self._geom = Geometry(nx, ny, nz, nt, self.px, self.py, max_batch, flags)
        self._h = ctypes.c_void_p(0)
        self._kp = None      # bins_padded, read once from the plan
        self._sinf = None    # shard layout, read once from the plan
        s = _stream(stream)
        if (table is None) == (medium is None):
            raise ValueError("give exactly one of table= or medium=")
        self._ws = workspace
        ws_ptr, ws_bytes = (None, 0) if workspace is None else (
            workspace.data_ptr(), workspace.numel() * workspace.element_size())
        if workspace is not None and not workspace.is_cuda:
            raise ValueError("workspace must be a CUDA tensor")
        self.shard = shard
        if shard is not None:
            if medium is None or workspace is not None:
                raise ValueError("a frequency shard is built from a medium, on its own workspace")
            rank, world = shard
            _check(L.pat_plan_create_kspace_shard(ctypes.byref(self._geom),
                                                  ctypes.byref(medium.c_struct()), rank, world, s,
                                                  ctypes.byref(self._h)))
        elif medium is not None:
            _check(L.pat_plan_create_kspace_with_workspace(
                ctypes.byref(self._geom), ctypes.byref(medium.c_struct()), ws_ptr, ws_bytes, s,
                ctypes.byref(self._h)))
        else:
            fmt, keep = _table_format(table, self)
            _check(L.pat_plan_create_with_workspace(ctypes.byref(self._geom), _ptr(keep), fmt,
                                                    ws_ptr, ws_bytes, s, ctypes.byref(self._h)))
        self.dtype_name = "float64" if fp64 else "float32"

    # ------------------------------------------------------------------ helpers
    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = PlanInfo()
        _check(lib().pat_plan_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in PlanInfo._fields_}

    def set_tensor_batch(self, min_batch: int) -> None:
        """Batches >= min_batch use the tensor-core contraction (0 = never)."""
        _check(lib().pat_plan_set_tensor_batch(self._h, min_batch))

    def set_sampling(self, sx: int = 1, sy: int = 1, ox: int = 0, oy: int = 0) -> None:
        """Measurement operator (Sec. 2.3, 3.3): data are kept only at the scan
        positions x = ox + sx i, y = oy + sy j of the sensor grid, so forward is
        S H (data [nt][my][mx]) and adjoint H* S^T (zero-filled). (1, 1, 0, 0)
        is the plain operator. Data loaded into slots must be reloaded."""
        _check(lib().pat_plan_set_sampling(self._h, sx, sy, ox, oy))
        self.sampling = (sx, sy, ox, oy)
        self.mx = -(-(self.nx - ox) // sx)
        self.my = -(-(self.ny - oy) // sy)

    def set_sensor_response(self, r, stream=None) -> None:
        """Folds the sensors' temporal impulse response r (causal, r[0] at lag
        0) into the resident library by temporal convolution (Sec. 2)."""
        a = np.ascontiguousarray(np.asarray(r, dtype=np.float64).ravel())
        _check(lib().pat_plan_set_sensor_response(
            self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(a.size),
            _stream(stream)))

    def check(self) -> None:
        """Raises PatError(PAT_ERR_TIMEOUT) if a bounded device wait gave up."""
        _check(lib().pat_plan_check(self._h))

    def set_wait_limit(self, polls: int) -> None:
        """Pipeline wait limit of the tensor-core kernels (tests per wait;
        < 0 restores the default, 0 makes every such wait give up)."""
        _check(lib().pat_plan_set_wait_limit(self._h, int(polls)))

    def close(self) -> None:
        if self._h and self._h.value:
            lib().pat_plan_destroy(self._h)
            self._h = ctypes.c_void_p(0)
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _torch_dtype(self):
        torch = _torch()
        return torch.float64 if self.fp64 else torch.float32

    def obj_shape(self, batch: int = 1):
        return (batch, self.nz, self.ny, self.nx)

    def data_shape(self, batch: int = 1):
        return (batch, self.nt, self.my, self.mx)

    def _batch_of(self, a, per) -> int:
        n = int(np.prod(a.shape))
        if n % per:
            raise ValueError(f"array of {n} elements is not a whole number of {per}-element volumes")
        return n // per

    def _empty_like_device(self, shape, like):
        torch = _torch()
        dev = like.device if hasattr(like, "device") and like.device.type == "cuda" else "cpu"
        return torch.empty(shape, dtype=self._torch_dtype(), device=dev)

    def _rdt(self):
        return np.float64 if self.fp64 else np.float32

    def _cdt(self):
        return np.complex128 if self.fp64 else np.complex64

    def _check_dtype(self, *arrs):
        want = np.float64 if self.fp64 else np.float32
        for a in arrs:
            dt = a.dtype if isinstance(a, np.ndarray) else _np_dtype(a.dtype)
            if dt != want:
                raise TypeError(f"plan works in {self.dtype_name}; got {dt}")

    # ------------------------------------------------------------------ operators
    def forward(self, rho, out=None, stream=None):
        """d = H rho (Eq. 7-8)."""
        self._check_dtype(rho)
        b = self._batch_of(rho, self.nz * self.ny * self.nx)
        if out is None:
            out = self._empty_like_device(self.data_shape(b) if rho.ndim == 4 else
                                          self.data_shape(1)[1:], rho)
        _need(out, b * self.nt * self.my * self.mx, self._rdt(), "out")
        _check(lib().pat_forward(self._h, _ptr(rho), _ptr(out), b, _stream(stream)))
        return out

    def adjoint(self, d, out=None, stream=None):
        """rho = H* d (Eq. 11)."""
        self._check_dtype(d)
        b = self._batch_of(d, self.nt * self.my * self.mx)
        if out is None:
            out = self._empty_like_device(self.obj_shape(b) if d.ndim == 4 else
                                          self.obj_shape(1)[1:], d)
        _need(out, b * self.nz * self.ny * self.nx, self._rdt(), "out")
        _check(lib().pat_adjoint(self._h, _ptr(d), _ptr(out), b, _stream(stream)))
        return out

    def gradient(self, x, y, out=None, resid: bool = True, stream=None):
        """grad = H*(H x - y) (Eq. 15); returns (grad, ||H x - y||^2 or None)."""
        self._check_dtype(x, y)
        b = self._batch_of(x, self.nz * self.ny * self.nx)
        _need(y, b * self.nt * self.my * self.mx, self._rdt(), "y")
        if out is None:
            out = self._empty_like_device(tuple(x.shape), x)
        _need(out, b * self.nz * self.ny * self.nx, self._rdt(), "out")
        r2 = ctypes.c_double(0.0)
        _check(lib().pat_gradient(self._h, _ptr(x), _ptr(y), _ptr(out), b,
                                  ctypes.byref(r2) if resid else None, _stream(stream)))
        return out, (r2.value if resid else None)

    def power_norm(self, v0, iters: int, stream=None) -> float:
        """L = ||H*H|| by power iteration from v0."""
        self._check_dtype(v0)
        _need(v0, self.nz * self.ny * self.nx, self._rdt(), "v0")
        Lout = ctypes.c_double(0.0)
        _check(lib().pat_power_norm(self._h, _ptr(v0), iters, ctypes.byref(Lout), _stream(stream)))
        return Lout.value

    def power_norm_seed(self, iters: int, seed: int, stream=None) -> float:
        """L = ||H*H|| by power iteration from the seeded splitmix64 start vector."""
        Lout = ctypes.c_double(0.0)
        _check(lib().pat_power_norm_seed(self._h, iters, ctypes.c_uint64(seed), ctypes.byref(Lout),
                                         _stream(stream)))
        return Lout.value

    def fista(self, y, x=None, iters: int = 100, lam: float = 0.0, L: float = 0.0,
              power_iters: int = 50, warm_start: bool = False, stream=None):
        """FISTA for Eq. 12-14; returns (x, report dict)."""
        self._check_dtype(y)
        b = self._batch_of(y, self.nt * self.my * self.mx)
        if x is None:
            x = self._empty_like_device(self.obj_shape(b) if y.ndim == 4 else
                                        self.obj_shape(1)[1:], y)
            warm_start = False
        _need(x, b * self.nz * self.ny * self.nx, self._rdt(), "x")
        prm = FistaParams(iters, power_iters, 1 if warm_start else 0, 0, lam, L)
        rep = FistaReport()
        _check(lib().pat_fista_solve(self._h, _ptr(y), _ptr(x), b, ctypes.byref(prm),
                                     ctypes.byref(rep), _stream(stream)))
        return x, {"L": rep.L, "resid2_first": rep.resid2_first, "resid2_last": rep.resid2_last,
                   "iters": rep.iters, "kernels_per_iter": rep.kernels_per_iter}

    def dot(self, a, b, stream=None) -> float:
        """<a, b> with FP64 products and sums (device arrays)."""
        self._check_dtype(a, b)
        out = ctypes.c_double(0.0)
        n = int(np.prod(a.shape))
        assert int(np.prod(b.shape)) == n
        _check(lib().pat_dot_f64(self._h, _ptr(a), _ptr(b), n, ctypes.byref(out), _stream(stream)))
        return out.value

    # ------------------------------------------------------------------ slots
    def slot_load(self, slot: int, y, lam: float, L: float, stream=None) -> None:
        """Loads one FISTA request (data y [nt][my][mx]) into `slot`."""
        self._check_dtype(y)
        _need(y, self.nt * self.my * self.mx, self._rdt(), "y")
        _check(lib().pat_slot_load(self._h, slot, _ptr(y), lam, L, _stream(stream)))

    def slot_move(self, dst: int, src: int, stream=None) -> None:
        _check(lib().pat_slot_move(self._h, dst, src, _stream(stream)))

    def slots_step(self, n: int, stream=None) -> int:
        """One FISTA iteration for slots [0, n); returns the kernel launches."""
        k = ctypes.c_int(0)
        _check(lib().pat_slots_step(self._h, n, ctypes.byref(k), _stream(stream)))
        return k.value

    def slot_read(self, slot: int, out=None, resid: bool = False, stream=None):
        """Copies the slot's current x_k into `out` (allocated on the device if
        None); returns (out, ||H y_k - d||^2 or None)."""
        if out is None:
            torch = _torch()
            out = torch.empty((self.nz, self.ny, self.nx), dtype=self._torch_dtype(), device="cuda")
        _need(out, self.nz * self.ny * self.nx, self._rdt(), "out")
        r2 = ctypes.c_double(0.0)
        _check(lib().pat_slot_read(self._h, slot, _ptr(out), ctypes.byref(r2) if resid else None,
                                   _stream(stream)))
        return out, (r2.value if resid else None)

    # ------------------------------------------------------------------ frequency shards
    def shard_info(self) -> dict:
        if self._sinf is None:
            inf = ShardInfo()
            _check(lib().pat_plan_shard_info(self._h, ctypes.byref(inf)))
            self._sinf = inf.as_dict()
        return dict(self._sinf)

    def shard_spectrum(self, side: int, x, send=None, stream=None):
        """Stage i of this rank's slices (side 0: depth slices of an object,
        1: time samples of data) into the all-to-all send buffer
        complex64 [world][slices][W]."""
        torch = _torch()
        inf = self.shard_info()
        n = inf["nt_local"] if side else inf["nz_local"]
        _need(x, n * self.ny * self.nx, np.float32, "x")
        if send is None:
            send = torch.empty((inf["world"], n, inf["slot_width"]), dtype=torch.complex64,
                               device=x.device)
        _need(send, inf["world"] * n * inf["slot_width"], np.complex64, "send")
        _check(lib().pat_shard_spectrum(self._h, side, _ptr(x), _ptr(send), _stream(stream)))
        return send

    def shard_contract(self, inp, out=None, adjoint: bool = False, stream=None):
        """Stage ii on this rank's rows: [nz][W] -> [nt][W] (or the adjoint)."""
        torch = _torch()
        inf = self.shard_info()
        W = inf["slot_width"]
        _need(inp, (self.nt if adjoint else self.nz) * W, np.complex64, "inp")
        rows = self.nz if adjoint else self.nt
        if out is None:
            out = torch.empty((rows, W), dtype=torch.complex64, device=inp.device)
        _need(out, rows * W, np.complex64, "out")
        _check(lib().pat_shard_contract(self._h, 1 if adjoint else 0, _ptr(inp), _ptr(out),
                                        _stream(stream)))
        return out

    def shard_image(self, side: int, recv, out=None, sub=None, resid: bool = False, stream=None):
        """Stage iii of this rank's slices from the received spectra
        [world][slices][W]; with `sub`, image - sub (and its FP64 sum of squares
        over this rank when resid). Returns (out, r2 or None)."""
        torch = _torch()
        inf = self.shard_info()
        n = inf["nt_local"] if side else inf["nz_local"]
        _need(recv, inf["world"] * n * inf["slot_width"], np.complex64, "recv")
        if out is None:
            out = torch.empty((n, self.ny, self.nx), dtype=torch.float32, device=recv.device)
        _need(out, n * self.ny * self.nx, np.float32, "out")
        if sub is not None:
            _need(sub, n * self.ny * self.nx, np.float32, "sub")
        r2 = ctypes.c_double(0.0)
        _check(lib().pat_shard_image(self._h, side, _ptr(recv), _ptr(out),
                                     _ptr(sub) if sub is not None else None,
                                     ctypes.byref(r2) if resid else None, _stream(stream)))
        return out, (r2.value if resid else None)

    def fista_step(self, y, xprev, grad, invL: float, lamL: float, beta: float, stream=None):
        """The FISTA update of Eq. 14-15 in place (pat_fista_step)."""
        fista_step(y, xprev, grad, invL, lamL, beta, stream)

    def axpby(self, y, x, a: float, b: float, stream=None) -> None:
        """y = a x + b y in place (pat_axpby)."""
        axpby(y, x, a, b, stream)

    # ------------------------------------------------------------------ stages
    def stage_spectrum(self, x, out=None, stream=None):
        """Zero-padded 2D real DFT of real [S][ny][nx] slices -> complex [S][px//2+1][py]."""
        torch = _torch()
        self._check_dtype(x)
        S = self._batch_of(x, self.ny * self.nx)
        cdt = torch.complex128 if self.fp64 else torch.complex64
        if out is None:
            out = torch.empty((S, self.px // 2 + 1, self.py), dtype=cdt, device=x.device)
        _need(out, S * (self.px // 2 + 1) * self.py, self._cdt(), "out")
        _check(lib().pat_stage_spectrum(self._h, _ptr(x), _ptr(out), S, _stream(stream)))
        return out

    def stage_contract(self, X, out, batch: int = 1, adjoint: bool = False, stream=None):
        """Stage ii alone on complex [batch][rows][bins_padded] device arrays."""
        if self._kp is None:
            self._kp = int(self.info()["bins_padded"])
        kp = self._kp
        rin, rout = (self.nt, self.nz) if adjoint else (self.nz, self.nt)
        _need(X, batch * rin * kp, self._cdt(), "X")
        _need(out, batch * rout * kp, self._cdt(), "out")
        _check(lib().pat_stage_contract(self._h, _ptr(X), _ptr(out), batch, 1 if adjoint else 0,
                                        _stream(stream)))
        return out

    def stage_contract_slots(self, X, out, batch: int, adjoint: bool = False, stream=None):
        """Stage ii of the folded split-BF16 path on spectra already in its
        representative-slot layout (rows of 4 * ceil(U/32) * 32 complex)."""
        _check(lib().pat_stage_contract_slots(self._h, _ptr(X), _ptr(out), batch,
                                              1 if adjoint else 0, _stream(stream)))
        return out

    def stage_image(self, X, out=None, stream=None):
        """Unnormalised inverse 2D DFT of [S][px//2+1][py] spectra, real part, cropped to [S][ny][nx]."""
        S = int(np.prod(X.shape)) // ((self.px // 2 + 1) * self.py)
        _need(X, S * (self.px // 2 + 1) * self.py, self._cdt(), "X")
        if out is None:
            out = self._empty_like_device((S, self.ny, self.nx), X)
        _need(out, S * self.ny * self.nx, self._rdt(), "out")
        _check(lib().pat_stage_image(self._h, _ptr(X), _ptr(out), S, _stream(stream)))
        return out


def plan_estimate(nx: int, ny: int, nz: int, nt: int, px: int | None = None, py: int | None = None,
                  max_batch: int = 1, fp64: bool = False, real_table: bool = True,
                  bf16_split: bool = False, fold: bool = False, radial: bool = False):
    """(table bytes including the split-BF16 tables, workspace bytes) a plan
    would take on the device; `fold` / `radial` estimate the D4-folded /
    radially shared representation a k-space library with dx = dy gets."""
    px = px if px is not None else _pow2_at_least(2 * nx)
    py = py if py is not None else _pow2_at_least(2 * ny)
    g = Geometry(nx, ny, nz, nt, px, py, max_batch,
                 (FLAG_FP64 if fp64 else 0) | (FLAG_BF16_SPLIT if bf16_split else 0))
    tb, ws = ctypes.c_int64(0), ctypes.c_int64(0)
    rep = 0 if not real_table else (3 if fold and radial else 2 if fold else 1)
    _check(lib().pat_plan_estimate(ctypes.byref(g), rep, ctypes.byref(tb), ctypes.byref(ws)))
    return tb.value, ws.value


def spectrum_noalloc(x, px: int, py: int, out=None, stream=None):
    """pat_spectrum_noalloc: stage-i spectrum of float32 [S][ny][nx] CUDA slices
    without a plan and without any device allocation inside the call (the
    library's static scratch holds the intermediate). `out`, if given, must be a
    complex64 CUDA tensor [S][px//2+1][py] on x's device; allocate it before
    calling when the caller itself cannot allocate. Runs on x's device (on
    `stream`, else that device's current stream)."""
    torch = _torch()
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32
            and x.is_contiguous() and x.dim() == 3):
        raise TypeError("x must be a contiguous float32 CUDA tensor [S][ny][nx]")
    S, ny, nx = int(x.shape[0]), int(x.shape[-2]), int(x.shape[-1])
    shape = (S, px // 2 + 1, py)
    if out is None:
        out = torch.empty(shape, dtype=torch.complex64, device=x.device)
    elif not (isinstance(out, torch.Tensor) and out.dtype == torch.complex64
              and tuple(out.shape) == shape and out.device == x.device and out.is_contiguous()):
        raise TypeError(f"out must be a contiguous complex64 tensor {shape} on {x.device}")
    with torch.cuda.device(x.device):
        s = _stream(stream) if stream is not None else int(
            torch.cuda.current_stream(x.device).cuda_stream)
        _check(lib().pat_spectrum_noalloc(_ptr(x), nx, ny, px, py, S, _ptr(out), s))
    return out


def fista_step(y, xprev, grad, invL: float, lamL: float, beta: float, stream=None) -> None:
    """pat_fista_step: the FISTA update of Eq. 14-15 in place on float32 CUDA arrays."""
    n = int(np.prod(y.shape))
    for a, what in ((y, "y"), (xprev, "xprev"), (grad, "grad")):
        _need(a, n, np.float32, what)
    _check(lib().pat_fista_step(_ptr(y), _ptr(xprev), _ptr(grad), n, invL, lamL, beta,
                                _stream(stream)))


def axpby(y, x, a: float, b: float, stream=None) -> None:
    """y = a x + b y in place on float32 CUDA arrays (pat_axpby)."""
    n = int(np.prod(y.shape))
    _need(y, n, np.float32, "y")
    _need(x, n, np.float32, "x")
    _check(lib().pat_axpby(_ptr(y), _ptr(x), n, a, b, _stream(stream)))


def shard_layout(nx: int, ny: int, nz: int, nt: int, px: int, py: int, fold: bool, rank: int,
                 world: int):
    """pat_shard_layout (host only): the partition of one rank and its slot maps
    (zmap, tmap: int32 [bins]; members_local: int32 [rows_per_rank][4] when folded)."""
    g = Geometry(nx, ny, nz, nt, px, py, 1, 0)
    inf = ShardInfo()
    _check(lib().pat_shard_layout(ctypes.byref(g), 1 if fold else 0, rank, world, ctypes.byref(inf),
                                  None, None, None))
    K = inf.bins
    zmap = np.empty(K, np.int32)
    tmap = np.empty(K, np.int32)
    mem = np.empty((inf.rows_per_rank, 4), np.int32)
    _check(lib().pat_shard_layout(ctypes.byref(g), 1 if fold else 0, rank, world, ctypes.byref(inf),
                                  zmap.ctypes.data, tmap.ctypes.data, mem.ctypes.data))
    return inf.as_dict(), zmap, tmap, (mem if fold else None)


def fold_blocks(P: int, radial: bool = True) -> dict:
    """pat_fold_blocks (host only): the block layout of the CUDA-core
    contraction of a folded P x P plan. Returns nrb, nch and int32 arrays
    rb_rep [nrb][32], rb_chunk [nrb], row_rep [nch][32], rep_row [U]."""
    nrb, nch = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().pat_fold_blocks(P, 1 if radial else 0, ctypes.byref(nrb), ctypes.byref(nch),
                                 None, None, None, None))
    U = (P // 2 + 1) * (P // 2 + 2) // 2
    out = {"rb_rep": np.empty((nrb.value, 32), np.int32), "rb_chunk": np.empty(nrb.value, np.int32),
           "row_rep": np.empty((nch.value, 32), np.int32), "rep_row": np.empty(U, np.int32)}
    _check(lib().pat_fold_blocks(P, 1 if radial else 0, ctypes.byref(nrb), ctypes.byref(nch),
                                 out["rb_rep"].ctypes.data, out["rb_chunk"].ctypes.data,
                                 out["row_rep"].ctypes.data, out["rep_row"].ctypes.data))
    out["nrb"], out["nch"] = nrb.value, nch.value
    return out


def workspace_size(nx: int, ny: int, nz: int, nt: int, px: int | None = None,
                   py: int | None = None, max_batch: int = 1, fp64: bool = False) -> int:
    """Bytes of caller-owned workspace a plan for this grid needs (pat_workspace_size)."""
    px = px if px is not None else _pow2_at_least(2 * nx)
    py = py if py is not None else _pow2_at_least(2 * ny)
    g = Geometry(nx, ny, nz, nt, px, py, max_batch, FLAG_FP64 if fp64 else 0)
    n = lib().pat_workspace_size(ctypes.byref(g))
    if n < 0:
        _check(int(n))
    return int(n)


def debug_live_allocations() -> int:
    """Device allocations the library currently holds (all plans)."""
    return int(lib().pat_debug_live_allocations())


def _pow2_at_least(n: int) -> int:
    p = 16
    while p < n:
        p *= 2
    return p


def _np_dtype(tdt):
    torch = _torch()
    return {torch.float32: np.float32, torch.float64: np.float64,
            torch.complex64: np.complex64, torch.complex128: np.complex128}.get(tdt, None)


def _table_format(table, plan: Plan):
    """(format code, contiguous array to pass) for a spatial or spectral table."""
    shape = tuple(table.shape)
    spatial = (plan.nz, plan.nt, plan.py, plan.px)
    spectral = (plan.nz, plan.nt, plan.py, plan.px // 2 + 1)
    dt = table.dtype if isinstance(table, np.ndarray) else _np_dtype(table.dtype)
    if isinstance(table, np.ndarray):
        table = np.ascontiguousarray(table)
    else:
        table = table.contiguous()
    if shape == spatial and dt in (np.float64, np.float32):
        return (TABLE_SPATIAL_F64 if dt == np.float64 else TABLE_SPATIAL_F32), table
    if shape == spectral and dt in (np.complex128, np.complex64):
        return (TABLE_SPECTRAL_C128 if dt == np.complex128 else TABLE_SPECTRAL_C64), table
    raise ValueError(f"table of shape {shape} / {dt}: expected spatial {spatial} real or "
                     f"spectral {spectral} complex")


def _autograd_fn():
    torch = _torch()

    class PatOp(torch.autograd.Function):
        """d = H x with backward H* (the hand-written adjoint kernels)."""

        @staticmethod
        def forward(ctx, x, plan: Plan):
            ctx.plan = plan
            return plan.forward(x.contiguous())

        @staticmethod
        def backward(ctx, g):
            return ctx.plan.adjoint(g.contiguous()), None

    return PatOp


def apply(plan: Plan, x):
    """Differentiable H x (torch.autograd): backward applies H*."""
    return _autograd_fn().apply(x, plan)
