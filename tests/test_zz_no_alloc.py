"""pat_spectrum_noalloc: the stage-i spectrum for callers that cannot allocate
device memory (their memory belongs to their own pool, or cudaMalloc is not
allowed where they call). It must give what pat_stage_spectrum gives, call
after call, although its intermediate lives in one static array shared by all
calls. Collected last on purpose (file name), so a failure here comes after
every other test has run; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2603_28150_gb300 import Plan, pat, synth

pytestmark = pytest.mark.gpu


def _call_c_abi(x, px, py, out):
    """Direct C-ABI call (device pointers, current stream)."""
    import torch
    S, ny, nx = x.shape
    rc = pat.lib().pat_spectrum_noalloc(ctypes.c_void_p(x.data_ptr()), nx, ny, px, py, S,
                                        ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def _reference(x, px, py):
    """The existing entry point (plan workspace) on the same slices."""
    S, ny, nx = x.shape
    plan = Plan(nx, ny, S, 1, px, py, table=np.zeros((S, 1, py, px)))
    return plan.stage_spectrum(x)


@pytest.mark.parametrize("shapes", [[(64, 128, 128, 256, 256), (16, 37, 50, 128, 128)],
                                    [(3, 5, 7, 16, 16), (256, 128, 128, 256, 256)]])
def test_noalloc_spectrum_matches_stage_spectrum_twice(shapes):
    import torch
    for i, (S, ny, nx, py, px) in enumerate(shapes):
        x = torch.tensor(synth.gaussian_field((S, ny, nx), seed=40 + i), dtype=torch.float32,
                         device="cuda")
        out = torch.empty((S, px // 2 + 1, py), dtype=torch.complex64, device="cuda")
        out.fill_(complex(float("nan"), float("nan")))  # stale values must all be overwritten
        assert _call_c_abi(x, px, py, out) == pat.PAT_OK, pat.lib().pat_last_error()
        ref = _reference(x, px, py)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - want).max() <= 2e-6 * np.abs(want).max()


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    # 512 slices of 256 rows at px = 512: 512 * 257 * 256 * 8 B > 64 MiB
    x = torch.zeros((512, 256, 256), dtype=torch.float32, device="cuda")
    out = torch.empty((512, 257, 512), dtype=torch.complex64, device="cuda")
    assert _call_c_abi(x, 512, 512, out) == pat.PAT_ERR_ARG
    assert b"static scratch" in pat.lib().pat_last_error()
    # the binding raises the same error
    with pytest.raises(pat.PatError):
        pat.spectrum_noalloc(x, 512, 512, out=out)
