"""Pins of the oracle's sensor-response folding (Sec. 2: the sensors' identical,
spatially invariant temporal response incorporated into the kernels by
temporal convolution).

The pins: a unit response is the identity; the operator built on folded
kernels equals the plain operator's data convolved along time with numpy's
convolve (causal, truncated to the recorded samples), pixel by pixel; two
responses fold as their convolution."""
import numpy as np
import pytest

import oracle
from paper_2603_28150_gb300 import synth

G = oracle.Grid(nx=6, ny=5, nz=3, nt=12, px=16, py=16)


def _h(seed=0):
    return synth.random_kernels(G.nz, G.nt, G.px, G.py, seed=seed)


def test_unit_response_is_identity():
    h = _h()
    assert np.array_equal(oracle.apply_sensor_response(h, [1.0]), h)
    assert np.array_equal(oracle.apply_sensor_response(h, [1.0, 0.0, 0.0]), h)


def test_delay_shifts_in_time():
    h = _h(1)
    hd = oracle.apply_sensor_response(h, [0.0, 0.0, 1.0])
    assert np.array_equal(hd[:, 2:], h[:, :-2])
    assert np.all(hd[:, :2] == 0)


@pytest.mark.parametrize("nr", [1, 3, 7, 20])
def test_folded_operator_equals_time_convolved_data(nr):
    h = _h(2)
    r = synth.gaussian_field((nr,), seed=nr)
    x = synth.gaussian_field((G.nz, G.ny, G.nx), seed=5)
    plain = oracle.Operator(G, h=h).A(x)
    folded = oracle.Operator(G, h=oracle.apply_sensor_response(h, r)).A(x)
    ref = np.empty_like(plain)
    for j in range(G.ny):
        for i in range(G.nx):
            ref[:, j, i] = np.convolve(plain[:, j, i], r)[:G.nt]
    assert np.abs(folded - ref).max() <= 1e-12 * np.abs(ref).max()


def test_two_responses_fold_as_their_convolution():
    h = _h(3)
    r1 = synth.gaussian_field((4,), seed=1)
    r2 = synth.gaussian_field((3,), seed=2)
    a = oracle.apply_sensor_response(oracle.apply_sensor_response(h, r1), r2)
    b = oracle.apply_sensor_response(h, np.convolve(r1, r2))
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
