"""Pins for the oracle's FISTA (Eq. 12-15) and power iteration: scipy's NNLS,
the KKT conditions of the l1 + non-negativity problem, the Beck-Teboulle rate
bound, the identity operator, and the SVD of the dense matrix."""
import numpy as np
import pytest
import scipy.optimize

import oracle
from paper_2603_28150_gb300 import synth

G = oracle.Grid(nx=3, ny=3, nz=2, nt=6, px=8, py=8)  # 18 unknowns, 54 data


def _problem(seed=0):
    h = synth.random_kernels(G.nz, G.nt, G.px, G.py, seed=seed)
    op = oracle.Operator(G, h=h)
    M = np.stack([op.A(e.reshape(op.obj_shape)).ravel()
                  for e in np.eye(int(np.prod(op.obj_shape)))], axis=1)
    x_true = np.abs(synth.gaussian_object(G.nx, G.ny, G.nz, seed=seed + 1))
    x_true[x_true < 0.6] = 0.0
    d = op.A(x_true) + 0.05 * synth.gaussian_field(op.data_shape, seed=seed + 2)
    return op, M, d


def test_power_iteration_matches_svd():
    op, M, _ = _problem(0)
    smax = np.linalg.svd(M, compute_uv=False)[0]
    L = oracle.power_norm(op, synth.gaussian_field(op.obj_shape, 5), iters=500)
    assert abs(L - smax ** 2) / smax ** 2 < 1e-8


def test_fista_lambda0_reaches_nnls():
    op, M, d = _problem(1)
    x_nnls, _ = scipy.optimize.nnls(M, d.ravel())
    L = np.linalg.svd(M, compute_uv=False)[0] ** 2
    res = oracle.fista(op, d, L, iters=5000)
    assert np.linalg.norm(res.x.ravel() - x_nnls) / np.linalg.norm(x_nnls) < 1e-6


def test_fista_lambda_positive_satisfies_kkt():
    op, M, d = _problem(2)
    L = np.linalg.svd(M, compute_uv=False)[0] ** 2
    lam = 1e-2 * np.abs(M.T @ d.ravel()).max()
    x = oracle.fista(op, d, L, iters=5000, lam=lam).x.ravel()
    grad = M.T @ (M @ x - d.ravel())
    pos = x > 1e-10
    assert pos.any() and (~pos).any()
    # stationarity on the support, dual feasibility off it
    assert np.abs(grad[pos] + lam).max() < 1e-8 * lam * 1e3
    assert (grad[~pos] + lam).min() > -1e-8 * lam * 1e3
    assert x.min() >= 0.0


def test_fista_rate_bound():
    """Beck & Teboulle (2009), Thm 4.4: F(x_k) - F* <= 2 L ||x_0 - x*||^2 / (k + 1)^2,
    with x* and F* from scipy's L-BFGS-B on the bound-constrained problem."""
    op, M, d = _problem(3)
    L = np.linalg.svd(M, compute_uv=False)[0] ** 2
    lam = 1e-3 * np.abs(M.T @ d.ravel()).max()
    b = d.ravel()

    def F(x):
        r = M @ x - b
        return 0.5 * r @ r + lam * x.sum(), M.T @ r + lam

    sol = scipy.optimize.minimize(F, np.zeros(M.shape[1]), jac=True, method="L-BFGS-B",
                                  bounds=[(0, None)] * M.shape[1],
                                  options={"ftol": 1e-15, "gtol": 1e-13, "maxiter": 10000})
    Fstar, R2 = sol.fun, float(sol.x @ sol.x)
    res = oracle.fista(op, d, L, iters=200, lam=lam, track=True)
    assert min(res.objective) >= Fstar - 1e-9 * abs(Fstar)
    for k, Fk in enumerate(res.objective, start=1):
        assert Fk - Fstar <= 2 * L * R2 / (k + 1) ** 2 + 1e-9 * abs(Fstar)


def test_fista_identity_operator_closed_form():
    """H = I (delta table with nz = nt, tau(j) = j) and L = 1: the first step
    lands on the minimiser max(d - lambda, 0) and the momentum keeps it there."""
    g = oracle.Grid.square(4, 3, 3)
    h = np.zeros((g.nz, g.nt, g.py, g.px))
    for j in range(g.nz):
        h[j, j, 0, 0] = 1.0
    op = oracle.Operator(g, h=h)
    d = synth.gaussian_field((g.nt, g.ny, g.nx), 4)
    lam = 0.3
    for iters in (1, 2, 7):
        x = oracle.fista(op, d, 1.0, iters=iters, lam=lam).x
        assert np.abs(x - np.maximum(d - lam, 0)).max() < 1e-14


def test_prox_is_the_minimiser():
    """prox of g = lam ||.||_1 + indicator(R+) against a brute-force 1D search."""
    v = np.linspace(-2, 2, 41)
    lam, step = 0.35, 0.8
    grid = np.linspace(0, 3, 300001)
    for vi in v:
        obj = 0.5 * (grid - vi) ** 2 + step * lam * grid
        assert abs(oracle.solvers.prox_g(np.array([vi]), step, lam)[0] - grid[np.argmin(obj)]) < 2e-5


@pytest.mark.parametrize("n", [1, 3])
def test_fista_zero_iterations_and_zero_data(n):
    op, M, d = _problem(4)
    L = np.linalg.svd(M, compute_uv=False)[0] ** 2
    assert np.all(oracle.fista(op, d, L, iters=0).x == 0)
    assert np.all(oracle.fista(op, np.zeros_like(d), L, iters=n).x == 0)
