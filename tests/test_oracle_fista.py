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


# --------------------------------------------------------------------------------------
# Pins of the momentum step (t-recurrence and beta_k): the fixed-point and KKT pins
# above hold for any convergent scheme, so these target the acceleration itself.

class _Dense:
    """A dense matrix in the operator interface the oracle's FISTA takes."""

    def __init__(self, M):
        self.M = M
        self.obj_shape = (M.shape[1],)

    def A(self, x):
        return self.M @ x

    def AT(self, y):
        return self.M.T @ y


def _difference_problem(n):
    """f(x) = 1/2 ||M x - e_1||^2 with M the (n+1) x n first-difference matrix, so
    M^T M is the 1-D Laplacian tridiag(-1, 2, -1) (Nesterov's worst case for
    first-order methods; condition number ~ 4 n^2 / pi^2). Its minimiser has the
    closed form x*_i = (n - i) / (n + 1) > 0, so the non-negativity of Eq. 14 is
    inactive there and F* = f(x*)."""
    M = np.zeros((n + 1, n))
    for i in range(n):
        M[i, i], M[i + 1, i] = 1.0, -1.0
    b = np.zeros(n + 1)
    b[0] = 1.0
    xs = (n - np.arange(n)) / (n + 1.0)
    return M, b, xs


def _rate_gap(n=200, iters=200):
    """max_k (F(x_k) - F*) / (2 L ||x_0 - x*||^2 / (k + 1)^2) of the oracle's FISTA."""
    M, b, xs = _difference_problem(n)
    assert np.abs(M.T @ (M @ xs - b)).max() < 1e-12  # the closed form is the minimiser
    L = np.linalg.svd(M, compute_uv=False)[0] ** 2
    Fs = 0.5 * float(np.sum((M @ xs - b) ** 2))
    res = oracle.fista(_Dense(M), b, L, iters=iters, track=True)
    k = np.arange(1, iters + 1)
    bound = 2.0 * L * float(xs @ xs) / (k + 1.0) ** 2
    return float(np.max((np.array(res.objective) - Fs) / bound))


def test_fista_rate_bound_ill_conditioned():
    """Beck & Teboulle (2009), Thm 4.4 on a problem with condition number ~1.6e4
    where the bound is tight to a factor ~5 and plain proximal gradient (ISTA,
    F - F* ~ 1/k) exceeds it within 200 iterations."""
    M, _, _ = _difference_problem(200)
    s = np.linalg.svd(M, compute_uv=False)
    assert (s[0] / s[-1]) ** 2 > 1e4
    assert _rate_gap() <= 1.0


@pytest.mark.parametrize("slip", ["ista", "t_update_without_square"])
def test_rate_bound_catches_planted_momentum_slips(monkeypatch, slip):
    """The same bound fails when a mistake is planted in the oracle's momentum:
    no extrapolation (ISTA), or t_{k+1} = (1 + sqrt(1 + 4 t_k)) / 2."""
    if slip == "ista":
        monkeypatch.setattr(oracle.solvers, "momentum", lambda t, tn: 0.0)
    else:
        monkeypatch.setattr(oracle.solvers, "next_t", lambda t: (1.0 + np.sqrt(1.0 + 4.0 * t)) / 2.0)
    assert _rate_gap() > 1.0


def _three_sequence_iterates(M, b, L, lam, x0, iters):
    """FISTA in Tseng's three-sequence form (Tseng 2008; Beck & Teboulle's scheme
    rewritten with z_k = x_{k-1} + t_k (x_k - x_{k-1}) and theta_k = 1 / t_k):
        y_k = (1 - theta_k) x_{k-1} + theta_k z_{k-1}
        x_k = y_k - G(y_k) / L,   z_k = z_{k-1} - t_k G(y_k) / L,
    G = grad f + lambda. It never forms an extrapolation weight beta_k. While the
    iterates stay positive the prox of Eq. 14 is the shift by lambda / L, so this
    equals the oracle's x_k exactly (to rounding)."""
    x, z, t, out = x0.copy(), x0.copy(), 1.0, []
    for _ in range(iters):
        y = (1.0 - 1.0 / t) * x + (1.0 / t) * z
        G = M.T @ (M @ y - b) + lam
        x = y - G / L
        z = z - t * G / L
        out.append(x.copy())
        t = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
    return out


def _three_sequence_gap(iters=60):
    n = 40
    M, _, _ = _difference_problem(n)
    i = np.arange(n)
    b = M @ (42.0 + np.sin(i))
    L = np.linalg.svd(M, compute_uv=False)[0] ** 2
    lam = 0.05
    x0 = 40.0 + np.sin(i) + 0.5 * np.cos(0.7 * i)
    ref = _three_sequence_iterates(M, b, L, lam, x0, iters)
    assert min(r.min() for r in ref) > 1.0  # positive throughout: the prox is a shift
    gap = 0.0
    for k in (1, 2, 3, 4, 7, 20, iters):
        xo = oracle.fista(_Dense(M), b, L, iters=k, lam=lam, x0=x0).x
        gap = max(gap, float(np.abs(xo - ref[k - 1]).max() / np.abs(ref[k - 1]).max()))
    return gap


def test_fista_equals_three_sequence_form():
    assert _three_sequence_gap() < 1e-12


@pytest.mark.parametrize("beta", [
    lambda t, tn: (tn - 1.0) / tn,                           # beta from t_{k+1} alone
    lambda t, tn: (t - 1.0) / t,                             # beta from t_k alone
    lambda t, tn: (tn - 1.0) / oracle.solvers.next_t(tn),    # beta one step ahead
    lambda t, tn: t / tn,                                    # (t_k - 1) written as t_k
], ids=["t_next_only", "t_only", "one_ahead", "dropped_minus_one"])
def test_three_sequence_form_catches_planted_beta_slips(monkeypatch, beta):
    """A mis-indexed extrapolation weight still converges at the accelerated rate
    (the bound above does not see it) but leaves the exact trajectory."""
    monkeypatch.setattr(oracle.solvers, "momentum", beta)
    assert _three_sequence_gap() > 1e-6


def test_momentum_sequence_identities():
    """t_{k+1}^2 - t_{k+1} = t_k^2 (the defining equation of the update), t_1 = 1,
    and t_k >= (k + 1) / 2 (Beck & Teboulle, Lemma 4.3)."""
    M, b, _ = _difference_problem(8)
    t = np.array(oracle.fista(_Dense(M), b, 4.0, iters=300, track=True).t)
    assert len(t) == 301 and t[0] == 1.0
    assert np.abs(t[1:] ** 2 - t[1:] - t[:-1] ** 2).max() <= 1e-12 * t[-1] ** 2
    k = np.arange(1, len(t) + 1)
    assert np.all(t >= (k + 1) / 2.0)
