"""GPU parity of the FFT stages (Sec. 3.2 stages i and iii) through the C ABI,
against numpy's FFT of the zero-padded slices (a library stand-in for the
oracle's own FFT, which is pinned to numpy in test_oracle_fft.py)."""
import numpy as np
import pytest

from paper_2603_28150_gb300 import Plan, synth
from tests.helpers import cuda, host

pytestmark = pytest.mark.gpu

# (nx, ny, px, py): every supported transform length (2^k and 3 * 2^k),
# odd/ragged sizes (odd row counts, a single row), non-square.
GRIDS = [(5, 7, 16, 16), (16, 16, 32, 32), (32, 32, 64, 64), (64, 50, 128, 128),
         (128, 128, 256, 256), (100, 60, 256, 128), (256, 256, 512, 512), (17, 3, 1024, 16),
         (512, 400, 1024, 1024), (29, 31, 64, 64), (45, 13, 128, 128), (101, 77, 256, 256),
         (3, 1, 256, 256), (200, 133, 512, 512),
         # 3 * 2^k lengths (a 24-point first pass), square, mixed with 2^k, ragged
         (12, 12, 24, 24), (20, 17, 48, 48), (48, 33, 96, 96), (96, 90, 192, 192),
         (150, 101, 384, 384), (384, 300, 768, 768), (11, 40, 24, 96), (100, 60, 256, 192),
         (30, 9, 768, 32)]


def _plan(nx, ny, px, py, nslices, fp64=False):
    # a trivial table: the stage entry points do not read it
    h = np.zeros((nslices, 1, py, px))
    return Plan(nx, ny, nslices, 1, px, py, table=h, fp64=fp64)


@pytest.mark.parametrize("nx,ny,px,py", GRIDS)
@pytest.mark.parametrize("fp64", [False, True])
def test_spectrum_matches_padded_fft(nx, ny, px, py, fp64):
    S = 3
    x = synth.gaussian_field((S, ny, nx), seed=nx + ny)
    plan = _plan(nx, ny, px, py, S, fp64)
    got = plan.stage_spectrum(cuda(x, fp64)).cpu().numpy().astype(np.complex128)
    pad = np.zeros((S, py, px))
    pad[:, :ny, :nx] = x
    ref = np.fft.fft2(pad)[:, :, :px // 2 + 1].transpose(0, 2, 1)  # [S][kx][ky]
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < (1e-13 if fp64 else 2e-6), err


@pytest.mark.parametrize("nx,ny,px,py", GRIDS)
@pytest.mark.parametrize("fp64", [False, True])
def test_image_matches_inverse_fft_crop(nx, ny, px, py, fp64):
    import torch
    S = 2
    g = np.random.default_rng(px + py)
    X = g.normal(size=(S, px // 2 + 1, py)) + 1j * g.normal(size=(S, px // 2 + 1, py))
    plan = _plan(nx, ny, px, py, S, fp64)
    Xt = torch.tensor(X, dtype=torch.complex128 if fp64 else torch.complex64, device="cuda")
    got = host(plan.stage_image(Xt))
    ref = np.fft.irfft2(X.transpose(0, 2, 1), s=(py, px)) * (px * py)
    ref = ref[:, :ny, :nx]
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < (1e-13 if fp64 else 2e-6), err


def test_spectrum_then_image_round_trip():
    nx, ny, px, py = 40, 24, 128, 64
    x = synth.gaussian_field((4, ny, nx), seed=3)
    plan = _plan(nx, ny, px, py, 4)
    back = host(plan.stage_image(plan.stage_spectrum(cuda(x)))) / (px * py)
    assert np.abs(back - x).max() < 2e-6 * np.abs(x).max()


@pytest.mark.parametrize("px,py", [(48, 48), (96, 384)])
def test_round_trip_three_times_power_of_two(px, py):
    nx, ny = px // 2, py // 2
    x = synth.gaussian_field((3, ny, nx), seed=px)
    plan = _plan(nx, ny, px, py, 3)
    back = host(plan.stage_image(plan.stage_spectrum(cuda(x)))) / (px * py)
    assert np.abs(back - x).max() < 2e-6 * np.abs(x).max()


@pytest.mark.parametrize("p", [20, 40, 1536, 2048, 12])
def test_unsupported_lengths_rejected(p):
    from paper_2603_28150_gb300 import PatError
    with pytest.raises(PatError):
        _plan(5, 5, p, 16, 1)
