"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/pat.h declares; argument errors come back as status codes without
touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2603_28150_gb300 import pat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pat.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pat_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = pat.lib()
    declared = _declared()
    assert len(declared) >= 13
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(pat.EXPORTS) == declared


def test_library_targets_sm103a():
    from paper_2603_28150_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB)


def test_argument_errors_without_gpu():
    L = pat.lib()
    out = ctypes.c_void_p(0)
    assert L.pat_plan_create(None, None, 0, None, ctypes.byref(out)) == pat.PAT_ERR_ARG
    g = pat.Geometry(32, 32, 4, 8, 80, 64, 1, 0)  # px = 80: neither 2^k nor 3 * 2^k
    buf = (ctypes.c_double * 4)()
    assert L.pat_plan_create(ctypes.byref(g), buf, 0, None, ctypes.byref(out)) == pat.PAT_ERR_UNSUPPORTED
    assert b"3*2^k" in L.pat_last_error()
    g = pat.Geometry(40, 32, 4, 8, 64, 64, 1, 0)  # 64 < 2*40-1: circular aliasing
    assert L.pat_plan_create(ctypes.byref(g), buf, 0, None, ctypes.byref(out)) == pat.PAT_ERR_ARG
    g = pat.Geometry(8, 8, 4, 8, 16, 16, 0, 0)  # max_batch 0
    assert L.pat_plan_create(ctypes.byref(g), buf, 0, None, ctypes.byref(out)) == pat.PAT_ERR_ARG
    g = pat.Geometry(8, 8, 4, 8, 16, 16, 1, 0)
    assert L.pat_plan_create(ctypes.byref(g), buf, 7, None, ctypes.byref(out)) == pat.PAT_ERR_ARG
    assert L.pat_forward(None, buf, buf, 1, None) == pat.PAT_ERR_ARG
    assert L.pat_plan_destroy(None) == pat.PAT_OK


@pytest.mark.parametrize("p", [16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024,
                               12, 20, 40, 80, 1536, 2048])
def test_transform_lengths_validated(p):
    """2^k and 3 * 2^k in [16, 1024] pass the geometry check (without a GPU the
    call then fails on the device allocation); other lengths are rejected as
    unsupported before anything else happens."""
    import numpy as np
    L = pat.lib()
    out = ctypes.c_void_p(0)
    n = max(1, p // 2)
    g = pat.Geometry(n, n, 1, 1, p, p, 1, 0)
    table = np.zeros(p * p)  # h[z][t][py][px], FP64, one depth and sample
    rc = L.pat_plan_create(ctypes.byref(g), table.ctypes.data_as(ctypes.c_void_p), 0, None,
                           ctypes.byref(out))
    n2 = p // 3 if p % 3 == 0 else p
    supported = 16 <= p <= 1024 and (n2 & (n2 - 1)) == 0
    if supported:
        assert rc != pat.PAT_ERR_UNSUPPORTED, L.pat_last_error()
        if rc == pat.PAT_OK:
            assert L.pat_plan_destroy(out) == pat.PAT_OK
    else:
        assert rc == pat.PAT_ERR_UNSUPPORTED
        assert b"3*2^k" in L.pat_last_error()


def test_medium_validation_without_gpu():
    L = pat.lib()
    out = ctypes.c_void_p(0)
    g = pat.Geometry(8, 8, 4, 8, 16, 16, 1, 0)
    m = pat.MediumC(1500.0, 1e-4, 1e-4, 1e-4, 2e-8, 4, 1)  # mz <= z0 + nz
    assert L.pat_plan_create_kspace(ctypes.byref(g), ctypes.byref(m), None, ctypes.byref(out)) == pat.PAT_ERR_ARG
    m = pat.MediumC(-1.0, 1e-4, 1e-4, 1e-4, 2e-8, 16, 1)
    assert L.pat_plan_create_kspace(ctypes.byref(g), ctypes.byref(m), None, ctypes.byref(out)) == pat.PAT_ERR_ARG


def test_product_has_no_cpu_fallback():
    """The binding never imports the oracle and has no numpy compute path."""
    import paper_2603_28150_gb300 as pkg
    for f in os.listdir(os.path.dirname(pkg.__file__)):
        if f.endswith(".py"):
            src = open(os.path.join(os.path.dirname(pkg.__file__), f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f
            assert "np.fft" not in src and "torch.fft" not in src, f


def test_workspace_size_without_gpu():
    """pat_workspace_size needs no device; it equals the workspace part of
    pat_plan_estimate, grows with max_batch and rejects invalid grids."""
    L = pat.lib()
    sizes = []
    for mb in (1, 2, 4):
        g = pat.Geometry(128, 128, 64, 256, 256, 256, mb, 0)
        n = L.pat_workspace_size(ctypes.byref(g))
        tb, ws = ctypes.c_int64(0), ctypes.c_int64(0)
        assert L.pat_plan_estimate(ctypes.byref(g), 1, ctypes.byref(tb), ctypes.byref(ws)) == pat.PAT_OK
        assert n == ws.value > 0
        sizes.append(n)
    assert sizes[0] < sizes[1] < sizes[2]
    # spectra X, Y (>= max(nz, nt) rows of K bins each) dominate
    assert sizes[0] > 2 * 256 * (129 * 256) * 8
    assert pat.workspace_size(128, 128, 64, 256) == sizes[0]
    bad = pat.Geometry(40, 32, 4, 8, 64, 64, 1, 0)
    assert L.pat_workspace_size(ctypes.byref(bad)) == pat.PAT_ERR_ARG
    assert L.pat_workspace_size(None) == pat.PAT_ERR_ARG


def test_allocation_fault_injection_without_gpu(monkeypatch):
    """PAT_DEBUG_FAIL_ALLOC = 1 fails the plan's first device allocation on the
    host (before any CUDA call): PAT_ERR_OOM, nothing left allocated."""
    L = pat.lib()
    g = pat.Geometry(16, 16, 4, 8, 32, 32, 1, 0)
    med = pat.MediumC(1500.0, 1e-4, 1e-4, 1e-4, 2e-8, 64, 1)
    out = ctypes.c_void_p(0)
    before = L.pat_debug_live_allocations()
    monkeypatch.setenv("PAT_DEBUG_FAIL_ALLOC", "1")
    assert L.pat_plan_create_kspace(ctypes.byref(g), ctypes.byref(med), None,
                                    ctypes.byref(out)) == pat.PAT_ERR_OOM
    assert out.value is None
    assert b"memory" in L.pat_last_error().lower()
    assert L.pat_debug_live_allocations() == before


def test_wait_limit_and_seed_arguments_without_gpu():
    L = pat.lib()
    assert L.pat_plan_set_wait_limit(None, 10) == pat.PAT_ERR_ARG
    d = ctypes.c_double(0.0)
    assert L.pat_power_norm_seed(None, 5, 1, ctypes.byref(d), None) == pat.PAT_ERR_ARG
    assert pat.WAIT_LIMIT_DEFAULT == 1 << 22


def test_shard_arguments_without_gpu():
    L = pat.lib()
    out = ctypes.c_void_p(0)
    g = pat.Geometry(16, 16, 6, 8, 32, 32, 1, 0)
    med = pat.MediumC(1500.0, 1e-4, 1e-4, 1e-4, 2e-8, 64, 1)
    # world must divide nz and nt
    assert L.pat_plan_create_kspace_shard(ctypes.byref(g), ctypes.byref(med), 0, 4, None,
                                          ctypes.byref(out)) == pat.PAT_ERR_UNSUPPORTED
    assert L.pat_plan_create_kspace_shard(ctypes.byref(g), ctypes.byref(med), 2, 2, None,
                                          ctypes.byref(out)) == pat.PAT_ERR_ARG
    g2 = pat.Geometry(16, 16, 6, 8, 32, 32, 2, 0)
    assert L.pat_plan_create_kspace_shard(ctypes.byref(g2), ctypes.byref(med), 0, 2, None,
                                          ctypes.byref(out)) == pat.PAT_ERR_UNSUPPORTED
    assert L.pat_shard_spectrum(None, 0, None, None, None) == pat.PAT_ERR_ARG
    assert L.pat_fista_step(None, None, None, 5, 1.0, 0.0, 0.0, None) == pat.PAT_ERR_ARG


def test_binding_rejects_mismatched_buffers_without_gpu():
    """The C ABI takes raw pointers and sizes: the Python binding checks the
    element count and type of every array it forwards, before any library
    call, so a short or wrongly typed buffer never reaches a kernel."""
    torch = pytest.importorskip("torch")
    f32, f64 = torch.zeros(8), torch.zeros(8, dtype=torch.float64)
    with pytest.raises(ValueError, match="xprev"):
        pat.fista_step(f32, f64, f32, 1.0, 0.0, 0.0)
    with pytest.raises(ValueError, match="grad"):
        pat.fista_step(f32, f32, torch.zeros(7), 1.0, 0.0, 0.0)
    with pytest.raises(ValueError, match="x"):
        pat.axpby(f32, torch.zeros(9), 1.0, 1.0)
    with pytest.raises(ValueError, match="expected 8 elements of float32"):
        pat._need(np.zeros(8), 8, np.float32, "a")
    pat._need(np.zeros((2, 4), np.float32), 8, np.float32, "a")  # shape is free, count is not
