"""Pins for the oracle's wave solve (Eq. 1-2) and the impulse-response library
(Sec. 3.2), and the Table 1 analogue: H rho equals a wave-equation solve."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2603_28150_gb300 import synth

MED = oracle.Medium(c=1500.0, dx=100e-6, dy=100e-6, dz=100e-6, dt=20e-9)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_stepping_equals_closed_form():
    g = np.random.default_rng(0)
    p0 = g.normal(size=(16, 8, 16))
    a = oracle.kspace_solve(p0, MED, 24, [0, 3, 15])
    b = oracle.kspace_solve(p0, MED, 24, [0, 3, 15], closed_form=True)
    assert oracle.rel_l2(a, b) < 1e-12


def test_plane_wave_standing_wave():
    """p0 = cos(k . r) for a grid wave vector k: the exact solution of Eq. 1-2
    with zero initial velocity is cos(c |k| t) cos(k . r)."""
    mz, py, px = 16, 8, 32
    z, y, x = np.meshgrid(np.arange(mz), np.arange(py), np.arange(px), indexing="ij")
    mx, my, mzz = 3, 1, 2
    phase = 2 * np.pi * (mx * x / px + my * y / py + mzz * z / mz)
    p0 = np.cos(phase)
    kk = np.sqrt((2 * np.pi * mx / (px * MED.dx)) ** 2 + (2 * np.pi * my / (py * MED.dy)) ** 2
                 + (2 * np.pi * mzz / (mz * MED.dz)) ** 2)
    rec = oracle.kspace_solve(p0, MED, 40, [0, 5])
    for i, plane in enumerate([0, 5]):
        for n in range(40):
            expect = np.cos(MED.c * kk * n * MED.dt) * p0[plane]
            assert np.abs(rec[i, n] - expect).max() < 1e-12


def test_initial_condition_and_time_reversal_symmetry():
    """t = 0 returns p0 (Eq. 2); with dp/dt = 0 the solution is even in time,
    so stepping forward n steps equals the closed form at -n dt."""
    g = np.random.default_rng(1)
    p0 = g.normal(size=(8, 8, 8))
    rec = oracle.kspace_solve(p0, MED, 5, list(range(8)))
    assert np.abs(rec[:, 0] - p0).max() < 1e-13
    back = oracle.kspace_solve(p0, oracle.Medium(MED.c, MED.dx, MED.dy, MED.dz, -MED.dt), 5,
                               list(range(8)), closed_form=True)
    assert oracle.rel_l2(rec, back) < 1e-13


def _table_setup(n=8, nz=4, nt=16):
    g = oracle.Grid.square(n, nz, nt)
    return g, oracle.mz_for(nz, nt, MED)


def test_library_solve_equals_closed_form_and_is_real_and_d4_symmetric():
    g, mz = _table_setup(8, 5, 20)
    h = oracle.table_kspace_solve(g, MED, mz)
    Hs = oracle.table_spectrum(h)
    Hc = oracle.table_kspace_closed(g, MED, mz)
    scale = np.abs(Hc).max()
    assert np.abs(Hs - Hc).max() < 1e-12 * scale
    assert np.abs(Hs.imag).max() < 1e-14 * scale          # radially symmetric kernels: real spectrum
    ky, kx = (-np.arange(g.py)) % g.py, (-np.arange(g.px)) % g.px
    assert np.abs(Hc - Hc[:, :, ky][:, :, :, kx]).max() == 0  # even in (kx, ky)
    assert np.abs(Hc - np.swapaxes(Hc, 2, 3)).max() < 1e-15 * scale  # kx <-> ky
    assert np.abs(Hc[:, 0]).max() < 1e-14 * scale          # t = 0: nothing reached the sensor plane


def test_reciprocity_one_solve_equals_per_depth_solves():
    """Sec. 3.2: recording every plane of ONE point-source solve gives the same
    library as one solve per depth with the source at that depth and the
    sensor on plane 0; so does the paper's variant (source at the bottom)."""
    g, mz = _table_setup(8, 4, 12)
    h = oracle.table_kspace_solve(g, MED, mz)
    for j in range(g.nz):
        p0 = np.zeros((mz, g.py, g.px))
        p0[1 + j, 0, 0] = 1.0  # object depth z0 + j with z0 = 1
        rec = oracle.kspace_solve(p0, MED, g.nt, [0])[0]
        assert np.abs(rec - h[j]).max() < 1e-14 * np.abs(h).max()
    hb = oracle.table_kspace_solve(g, MED, mz, src_plane=mz - 1, sign=-1)
    assert np.abs(hb - h).max() < 1e-14 * np.abs(h).max()


def _forward_vs_solve(g, mz, seeds, z0=1):
    Hc = oracle.table_kspace_closed(g, MED, mz, z0=z0)
    l2, linf = [], []
    for s in seeds:
        rho = synth.gaussian_object(g.nx, g.ny, g.nz, seed=s)
        d = oracle.forward_fft(Hc, rho, g)
        p0 = np.zeros((mz, g.py, g.px))
        p0[z0:z0 + g.nz, :g.ny, :g.nx] = rho
        ref = oracle.kspace_solve(p0, MED, g.nt, [0])[0][:, :g.ny, :g.nx]
        l2.append(oracle.rel_l2(d, ref))
        linf.append(oracle.rel_linf(d, ref))
    return np.array(l2), np.array(linf)


def test_forward_equals_wave_solve_table1_analogue():
    """Table 1: over 100 Gaussian random objects H rho matches the wave solve at
    the level of rounding (paper: median 2.2e-15 rel l2, max 3.4e-15 rel linf)."""
    paper = json.load(open(os.path.join(GOLDEN, "table1_forward_equivalence.json")))
    g, mz = _table_setup(6, 3, 10)
    l2, linf = _forward_vs_solve(g, mz, range(100))
    # same order as the paper's numbers: within 10x of its worst case
    assert l2.max() < 10 * paper["rel_l2"]["max"]
    assert linf.max() < 10 * paper["rel_linf"]["max"]


@pytest.mark.slow
def test_forward_equals_wave_solve_32x32x16x64():
    g = oracle.Grid.square(32, 16, 64)
    mz = oracle.mz_for(g.nz, g.nt, MED)
    l2, linf = _forward_vs_solve(g, mz, [0, 1])
    assert l2.max() < 1e-12 and linf.max() < 1e-12


def test_forward_equals_wave_solve_with_physical_spectrum_from_spatial_table():
    """Same check with the spatial library (one solve) run through the FFT form
    and through the spatial form of Eq. 7."""
    g, mz = _table_setup(6, 3, 10)
    h = oracle.table_kspace_solve(g, MED, mz)
    rho = synth.blobs(g.nx, g.ny, g.nz, count=3, seed=2)
    p0 = np.zeros((mz, g.py, g.px))
    p0[1:1 + g.nz, :g.ny, :g.nx] = rho
    ref = oracle.kspace_solve(p0, MED, g.nt, [0], closed_form=True)[0][:, :g.ny, :g.nx]
    assert oracle.rel_l2(oracle.forward_spatial(h, rho, g), ref) < 1e-12
    assert oracle.rel_l2(oracle.forward_fft(oracle.table_spectrum(h), rho, g), ref) < 1e-12
