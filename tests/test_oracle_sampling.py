"""Pins of the oracle's measurement operator S (Sec. 2.3, Sec. 3.3): S keeps
the scan positions x = ox + sx i, y = oy + sy j of the sensor grid, S^T
zero-fills, and the composed pair S H / H* S^T is an exact adjoint pair.

Each pin checks the oracle against something other than itself: the scan-grid
sizes printed in Sec. 3.3, numpy's strided slicing, a brute-force matrix of S
built from the coordinate rule, and the plain operator when S is the identity."""
import numpy as np
import pytest

import oracle
from paper_2603_28150_gb300 import synth

PATTERNS = [(1, 1, 0, 0), (2, 2, 0, 0), (2, 2, 1, 1), (3, 2, 1, 0), (2, 3, 0, 2), (4, 1, 3, 0)]


def test_scan_grid_of_the_phantom_experiments():
    # Sec. 3.3: 101 x 101 scan positions at 20 um pitch (2.02 mm field of
    # view), reconstruction on a 10 um grid over the same field: 202 voxels a
    # side, every second one a scan position.
    n_rec = round(2.02e-3 / 10e-6)
    assert n_rec == 202
    assert len(oracle.scan_positions(n_rec, 2, 0)) == 101
    assert len(oracle.scan_positions(n_rec, 2, 1)) == 101
    d = np.zeros((3, n_rec, n_rec))
    assert oracle.sample_scan(d, 2, 2, 0, 0).shape == (3, 101, 101)


@pytest.mark.parametrize("sx,sy,ox,oy", PATTERNS)
def test_sample_equals_strided_slice(sx, sy, ox, oy):
    d = synth.gaussian_field((4, 11, 13), seed=sx + 7 * sy + 3 * ox + oy)
    ds = oracle.sample_scan(d, sx, sy, ox, oy)
    assert np.array_equal(ds, d[:, oy::sy, ox::sx])


@pytest.mark.parametrize("sx,sy,ox,oy", PATTERNS)
def test_zero_fill_is_the_transpose_of_sampling(sx, sy, ox, oy):
    ny, nx = 7, 9
    n = ny * nx
    # S as a matrix, column by column from unit images
    M = np.stack([oracle.sample_scan(np.eye(n)[c].reshape(ny, nx), sx, sy, ox, oy).ravel()
                  for c in range(n)], axis=1)
    # brute force from the coordinate rule: row r of S selects the r-th scan
    # position in row-major order over (y, x)
    pos = [(y, x) for y in range(ny) for x in range(nx)
           if y >= oy and (y - oy) % sy == 0 and x >= ox and (x - ox) % sx == 0]
    B = np.zeros((len(pos), n))
    for r, (y, x) in enumerate(pos):
        B[r, y * nx + x] = 1.0
    assert np.array_equal(M, B)
    my = len(range(oy, ny, sy))
    mx = len(range(ox, nx, sx))
    assert M.shape[0] == my * mx
    T = np.stack([oracle.zero_fill(np.eye(my * mx)[r].reshape(my, mx), ny, nx, sx, sy, ox, oy).ravel()
                  for r in range(my * mx)], axis=0)
    assert np.array_equal(T, M)                   # S^T is the transpose of S
    assert np.array_equal(M @ M.T, np.eye(my * mx))  # S S^T = I


def _op(g, sampling, seed=0):
    h = synth.random_kernels(g.nz, g.nt, g.px, g.py, seed=seed)
    return oracle.Operator(g, h=h, sampling=sampling), oracle.Operator(g, h=h)


G = oracle.Grid(nx=13, ny=10, nz=3, nt=5, px=32, py=32)


@pytest.mark.parametrize("sx,sy,ox,oy", PATTERNS)
def test_composed_pair_is_adjoint(sx, sy, ox, oy):
    op, _ = _op(G, (sx, sy, ox, oy))
    x = synth.gaussian_field(op.obj_shape, seed=1)
    y = synth.gaussian_field(op.data_shape, seed=2)
    lhs = float(np.sum(op.A(x) * y))
    rhs = float(np.sum(x * op.AT(y)))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("sx,sy,ox,oy", PATTERNS[1:])
def test_composed_pair_against_plain_operator(sx, sy, ox, oy):
    op, plain = _op(G, (sx, sy, ox, oy), seed=5)
    x = synth.gaussian_field(op.obj_shape, seed=3)
    assert np.array_equal(op.A(x), plain.A(x)[:, oy::sy, ox::sx])
    y = synth.gaussian_field(op.data_shape, seed=4)
    full = np.zeros(plain.data_shape)
    full[:, oy::sy, ox::sx] = y
    assert np.array_equal(op.AT(y), plain.AT(full))


def test_identity_sampling_is_the_plain_operator():
    op, plain = _op(G, (1, 1, 0, 0), seed=6)
    x = synth.gaussian_field(op.obj_shape, seed=8)
    y = synth.gaussian_field(op.data_shape, seed=9)
    assert op.data_shape == plain.data_shape
    assert np.array_equal(op.A(x), plain.A(x))
    assert np.array_equal(op.AT(y), plain.AT(y))
