"""Pins for the oracle's H (Eq. 7) and H* (Eq. 11): two independent forms,
a library convolution, closed-form special cases, the adjoint identity (Eq. 9)
and the dense matrix transpose."""
import numpy as np
import pytest
import scipy.signal

import oracle
from paper_2603_28150_gb300 import synth

TINY = oracle.Grid.square(8, 4, 16)
SMALL = oracle.Grid(nx=12, ny=10, nz=3, nt=5, px=32, py=32)  # rectangular, P > 2n


def _setup(g, seed=0, even=False):
    h = synth.random_kernels(g.nz, g.nt, g.px, g.py, seed=seed, even=even)
    rho = synth.gaussian_object(g.nx, g.ny, g.nz, seed=seed + 1)
    d = synth.gaussian_field((g.nt, g.ny, g.nx), seed=seed + 2)
    return h, rho, d


@pytest.mark.parametrize("g", [TINY, SMALL, oracle.Grid(nx=5, ny=7, nz=2, nt=3, px=16, py=16),
                               oracle.Grid(nx=20, ny=11, nz=2, nt=3, px=48, py=24)])
def test_spatial_and_fft_forms_agree(g):
    h, rho, d = _setup(g, 3)
    Hf = oracle.table_spectrum(h)
    assert oracle.rel_l2(oracle.forward_fft(Hf, rho, g), oracle.forward_spatial(h, rho, g)) < 1e-12
    assert oracle.rel_l2(oracle.adjoint_fft(Hf, d, g), oracle.adjoint_spatial(h, d, g)) < 1e-12


@pytest.mark.slow
def test_spatial_and_fft_forms_agree_32x32x16x64():
    g = oracle.Grid.square(32, 16, 64)
    h, rho, d = _setup(g, 11)
    Hf = oracle.table_spectrum(h)
    assert oracle.rel_l2(oracle.forward_fft(Hf, rho, g), oracle.forward_spatial(h, rho, g)) < 1e-12
    assert oracle.rel_l2(oracle.adjoint_fft(Hf, d, g), oracle.adjoint_spatial(h, d, g)) < 1e-12


@pytest.mark.parametrize("n,p", [(6, 16), (8, 16), (9, 32), (10, 24), (12, 48)])
def test_single_depth_single_time_is_scipy_convolution(n, p):
    """Nz = Nt = 1: H is one 2D linear convolution with the kernel restricted to
    displacements |u| <= n - 1 (the wrapped table unwrapped)."""
    g = oracle.Grid.square(n, 1, 1, pad=p)
    h, rho, _ = _setup(g, 21)  # asymmetric random kernel: catches a flipped sign
    u = np.arange(-(n - 1), n)
    k2 = h[0, 0][np.ix_(u % p, u % p)]  # k2[uy + n - 1, ux + n - 1] = h(u)
    full = scipy.signal.convolve2d(rho[0], k2, mode="full")
    expect = full[n - 1:2 * n - 1, n - 1:2 * n - 1]
    d = oracle.forward_fft(oracle.table_spectrum(h), rho, g)[0]
    ds = oracle.forward_spatial(h, rho, g)[0]
    assert np.abs(d - expect).max() < 1e-12 * np.abs(expect).max()
    assert np.abs(ds - expect).max() < 1e-12 * np.abs(expect).max()
    # the adjoint is the matching correlation
    y = synth.gaussian_field((n, n), 5)
    corr = scipy.signal.correlate2d(y, k2, mode="full")[n - 1:2 * n - 1, n - 1:2 * n - 1]
    adj = oracle.adjoint_fft(oracle.table_spectrum(h), y[None], g)[0]
    assert np.abs(adj - corr).max() < 1e-12 * np.abs(corr).max()


def test_delta_table_embeds_slices():
    """h_j(., t) = delta at displacement 0 iff t = tau(j): d_t = sum_{tau(j)=t} rho_j."""
    g = oracle.Grid.square(6, 3, 5, pad=16)
    tau = [1, 3, 1]
    h = np.zeros((g.nz, g.nt, g.py, g.px))
    for j, t in enumerate(tau):
        h[j, t, 0, 0] = 1.0
    rho = synth.gaussian_object(g.nx, g.ny, g.nz, seed=9)
    expect = np.zeros((g.nt, g.ny, g.nx))
    for j, t in enumerate(tau):
        expect[t] += rho[j]
    for d in (oracle.forward_fft(oracle.table_spectrum(h), rho, g), oracle.forward_spatial(h, rho, g)):
        assert np.abs(d - expect).max() < 1e-13


def test_shifted_delta_translates():
    """h(u) = delta(u - u0) gives d(s) = rho(s - u0) (zero where s - u0 leaves the grid)."""
    g = oracle.Grid.square(8, 1, 1)
    uy, ux = 2, -3
    h = np.zeros((1, 1, g.py, g.px))
    h[0, 0, uy % g.py, ux % g.px] = 1.0
    rho = synth.gaussian_object(g.nx, g.ny, 1, seed=4)
    expect = np.zeros((g.ny, g.nx))
    for sy in range(g.ny):
        for sx in range(g.nx):
            ry, rx = sy - uy, sx - ux
            if 0 <= ry < g.ny and 0 <= rx < g.nx:
                expect[sy, sx] = rho[0, ry, rx]
    d = oracle.forward_fft(oracle.table_spectrum(h), rho, g)[0]
    assert np.abs(d - expect).max() < 1e-14


@pytest.mark.parametrize("g", [TINY, SMALL])
@pytest.mark.parametrize("form", ["fft", "spatial"])
def test_adjoint_identity(g, form):
    """Eq. 9 with the Euclidean products of Eq. 10."""
    h, rho, d = _setup(g, 31)
    op = oracle.Operator(g, h=h, form=form)
    Ax, ATy = op.A(rho), op.AT(d)
    lhs = np.dot(Ax.ravel(), d.ravel())
    rhs = np.dot(rho.ravel(), ATy.ravel())
    assert abs(lhs - rhs) / (np.linalg.norm(Ax) * np.linalg.norm(d)) < 1e-12


def _dense(fn, in_shape):
    n = int(np.prod(in_shape))
    cols = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        cols.append(fn(e.reshape(in_shape)).ravel())
    return np.stack(cols, axis=1)


def test_dense_matrix_transpose_is_exact():
    g = oracle.Grid(nx=4, ny=4, nz=3, nt=5, px=8, py=8)
    h, _, _ = _setup(g, 41)
    MA = _dense(lambda x: oracle.forward_spatial(h, x, g), (g.nz, g.ny, g.nx))
    MAT = _dense(lambda y: oracle.adjoint_spatial(h, y, g), (g.nt, g.ny, g.nx))
    assert np.array_equal(MA.T, MAT)  # single nonzero product per entry: exact
    Hf = oracle.table_spectrum(h)
    MAf = _dense(lambda x: oracle.forward_fft(Hf, x, g), (g.nz, g.ny, g.nx))
    MATf = _dense(lambda y: oracle.adjoint_fft(Hf, y, g), (g.nt, g.ny, g.nx))
    assert np.abs(MAf - MA).max() < 1e-13 and np.abs(MATf - MA.T).max() < 1e-13


def test_linearity():
    g = TINY
    h, x, _ = _setup(g, 51)
    y = synth.gaussian_object(g.nx, g.ny, g.nz, seed=52)
    Hf = oracle.table_spectrum(h)
    a, b = 0.7, -2.3
    lhs = oracle.forward_fft(Hf, a * x + b * y, g)
    rhs = a * oracle.forward_fft(Hf, x, g) + b * oracle.forward_fft(Hf, y, g)
    assert oracle.rel_l2(lhs, rhs) < 1e-13


def test_transverse_shift_equivariance():
    """Translating an object whose support stays in the grid translates the data
    on the overlap (the cropped operator's form of the shift invariance, Sec. 2.1)."""
    g = oracle.Grid.square(12, 3, 6, pad=32)
    h, _, _ = _setup(g, 61)
    rho = np.zeros((g.nz, g.ny, g.nx))
    rho[:, 2:6, 3:7] = synth.gaussian_object(4, 4, g.nz, seed=62)
    ay, ax = 4, 3
    shifted = np.zeros_like(rho)
    shifted[:, 2 + ay:6 + ay, 3 + ax:7 + ax] = rho[:, 2:6, 3:7]
    Hf = oracle.table_spectrum(h)
    d0 = oracle.forward_fft(Hf, rho, g)
    d1 = oracle.forward_fft(Hf, shifted, g)
    assert np.abs(d1[:, ay:, ax:] - d0[:, :g.ny - ay, :g.nx - ax]).max() < 1e-13 * np.abs(d0).max()


def test_rejects_aliasing_padding():
    g = oracle.Grid(nx=9, ny=9, nz=1, nt=1, px=16, py=16)  # 16 < 2*9 - 1
    with pytest.raises(ValueError):
        oracle.forward_fft(np.zeros((1, 1, 16, 16), complex), np.zeros((1, 9, 9)), g)
