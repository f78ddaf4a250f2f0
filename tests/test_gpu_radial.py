"""Radial sharing of the folded table on the GPU. Plans whose D4
representatives of equal kx^2 + ky^2 share one stored row give the same H
(Eq. 7-8), H* (Eq. 11) and FISTA (Eq. 12-14) as plans with one row per
representative and one row per bin, and match the FP64 oracle; a user table
with the D4 symmetry but unequal spectra on one radius keeps one row per
representative."""
import numpy as np
import pytest

import oracle
from paper_2603_28150_gb300 import Medium, Plan, pat, synth
from tests.helpers import MED_CFG1, cuda, host

pytestmark = pytest.mark.gpu

GEOMS = [oracle.Grid.square(32, 16, 64),                        # P = 64: 16 chunks for 18
         oracle.Grid(nx=20, ny=20, nz=8, nt=24, px=48, py=48),    # 3 * 2^k transforms
         oracle.Grid.square(64, 32, 128),                         # P = 128: 52 chunks for 68
         oracle.Grid.square(40, 12, 20, pad=96)]


def _medium(g):
    mz = oracle.mz_for(g.nz, g.nt, MED_CFG1)
    m = MED_CFG1
    return Medium(m.c, m.dx, m.dy, m.dz, m.dt, mz, 1), mz


def _plans(g, B=1):
    med, _ = _medium(g)
    kw = dict(medium=med, max_batch=B)
    return (Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, **kw),
            Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, radial=False, **kw),
            Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, fold=False, **kw))


@pytest.mark.parametrize("g", GEOMS, ids=["p64", "p48", "p128", "p96"])
@pytest.mark.parametrize("B", [1, 3])
def test_radial_plan_equals_d4_bins_and_oracle(g, B):
    pr, pd, pu = _plans(g, B)
    ir, idd, iu = pr.info(), pd.info(), pu.info()
    fr, fd = pat.fold_blocks(g.px, True), pat.fold_blocks(g.px, False)
    assert fr["nch"] < fd["nch"]
    assert (ir["folded"], ir["radial"]) == (1, 1)
    assert (idd["folded"], idd["radial"]) == (1, 0) and (iu["folded"], iu["radial"]) == (0, 0)
    assert ir["table_rows"] == idd["table_rows"]           # representatives
    assert ir["stored_rows"] == 32 * fr["nch"] and idd["stored_rows"] == 32 * fd["nch"]
    assert ir["table_bytes"] * fd["nch"] == idd["table_bytes"] * fr["nch"]
    _, mz = _medium(g)
    op = oracle.Operator(g, Hf=oracle.table_kspace_closed(g, MED_CFG1, mz))
    xs = np.stack([synth.blobs(g.nx, g.ny, g.nz, count=4, seed=60 + s) for s in range(B)])
    ys = np.stack([synth.gaussian_field((g.nt, g.ny, g.nx), 70 + s) for s in range(B)])
    for name, run, ref in (("H", lambda p: p.forward(cuda(xs)), [op.A(x) for x in xs]),
                           ("H*", lambda p: p.adjoint(cuda(ys)), [op.AT(y) for y in ys])):
        r, d, u = (host(run(p)) for p in (pr, pd, pu))
        assert np.abs(r - d).max() <= 1e-6 * np.abs(d).max(), name
        assert np.abs(r - u).max() <= 1e-6 * np.abs(u).max(), name
        for b in range(B):
            assert oracle.rel_l2(r[b], ref[b]) < 1e-5, (name, b)


def test_radial_fista_equals_d4():
    """The FISTA graph (fused residual and step passes) on a radial plan."""
    g = oracle.Grid.square(64, 32, 128)
    pr, pd, _ = _plans(g)
    y = cuda(host(pd.forward(cuda(synth.blobs(g.nx, g.ny, g.nz, count=6, seed=5)))))
    L = 1.01 * pd.power_norm(cuda(np.ones((g.nz, g.ny, g.nx), np.float32)), 30)
    xr, rr = pr.fista(y, iters=30, L=L)
    xd, rd = pd.fista(y, iters=30, L=L)
    assert oracle.rel_l2(host(xr), host(xd)) < 1e-5


def _d4_images(a, b, P):
    pts = set()
    for kx, ky in ((a, b), (b, a)):
        for sx in (1, -1):
            for sy in (1, -1):
                pts.add(((sx * kx) % P, (sy * ky) % P))
    return pts


def test_user_tables_share_rows_only_when_the_radii_agree():
    g = oracle.Grid.square(32, 16, 64)
    _, mz = _medium(g)
    Hf = oracle.table_kspace_closed(g, MED_CFG1, mz)        # [nz][nt][py][px], real values
    half = lambda H: np.ascontiguousarray(H[..., : g.px // 2 + 1])  # noqa: E731
    pr = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=half(Hf))
    assert (pr.info()["folded"], pr.info()["radial"]) == (1, 1)
    # 7^2 + 1^2 = 5^2 + 5^2 = 50: scale the eight images of (7, 1) only. The
    # table keeps the D4 symmetry but representatives (7, 1) and (5, 5) differ.
    bad = Hf.copy()
    for kx, ky in _d4_images(7, 1, g.px):
        bad[:, :, ky, kx] *= 1.05
    pb = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=half(bad))
    pu = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=half(bad), fold=False)
    assert (pb.info()["folded"], pb.info()["radial"]) == (1, 0)
    op = oracle.Operator(g, Hf=bad)
    x = synth.blobs(g.nx, g.ny, g.nz, count=5, seed=9)
    y = synth.gaussian_field((g.nt, g.ny, g.nx), 10)
    for got, alt, ref in ((pb.forward(cuda(x)), pu.forward(cuda(x)), op.A(x)),
                          (pb.adjoint(cuda(y)), pu.adjoint(cuda(y)), op.AT(y))):
        got, alt = host(got), host(alt)
        assert np.abs(got - alt).max() <= 1e-6 * np.abs(alt).max()
        assert oracle.rel_l2(got, ref) < 1e-5


def test_estimate_matches_plans():
    """pat_plan_estimate with the folded, radially shared representation gives
    the table bytes a k-space plan allocates (tensor tiles included), and at
    least its workspace (the estimate counts the host staging too)."""
    g = oracle.Grid.square(64, 32, 128)
    med, _ = _medium(g)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, medium=med)
    tb, ws = pat.plan_estimate(g.nx, g.ny, g.nz, g.nt, g.px, g.py, fold=True, radial=True)
    inf = plan.info()
    assert inf["radial"] == 1 and inf["table_bytes"] == tb and inf["workspace_bytes"] <= ws
    g2 = oracle.Grid.square(32, 128, 256)
    med2, _ = _medium(g2)
    p2 = Plan(g2.nx, g2.ny, g2.nz, g2.nt, g2.px, g2.py, max_batch=4, medium=med2,
              bf16_split=True)
    tb2, ws2 = pat.plan_estimate(g2.nx, g2.ny, g2.nz, g2.nt, g2.px, g2.py, max_batch=4,
                                 bf16_split=True, fold=True, radial=True)
    inf2 = p2.info()
    assert inf2["table_bytes"] + inf2["tensor_table_bytes"] == tb2
    assert inf2["workspace_bytes"] <= ws2
