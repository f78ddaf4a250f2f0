"""GPU parity of H (Eq. 7-8), H* (Eq. 11), the gradient (Eq. 15), the power
iteration and FISTA (Eq. 12-14) through the C ABI, element by element against
the FP64 oracle on identical seeded inputs.

Tolerances: FP32 plans <= 1e-5 relative l2 (the target for the single-precision
path); FP64 plans <= 1e-12."""
import numpy as np
import pytest

import oracle
from paper_2603_28150_gb300 import Medium, PatError, Plan, synth
from tests.helpers import MED_CFG1, MED_50UM, cuda, host, kspace_table

pytestmark = pytest.mark.gpu

CFG1 = oracle.Grid.square(32, 16, 64)            # 32^2 -> 64^2, 16 depths, 64 samples
RAGGED = oracle.Grid(nx=23, ny=17, nz=5, nt=9, px=64, py=64)   # odd sizes, several k-blocks
RECT = oracle.Grid(nx=20, ny=9, nz=3, nt=7, px=64, py=32)      # px != py
SMALLP = oracle.Grid(nx=5, ny=6, nz=3, nt=4, px=16, py=16)     # K = 9*16: ragged last k-block
P48 = oracle.Grid(nx=20, ny=17, nz=4, nt=9, px=48, py=48)      # 3 * 2^k transforms
RECT3 = oracle.Grid(nx=11, ny=40, nz=3, nt=5, px=24, py=96)    # 3 * 2^k, px != py


def _tables(g, kind, seed=0):
    if kind == "random":      # asymmetric kernels: complex spectra
        return synth.random_kernels(g.nz, g.nt, g.px, g.py, seed=seed)
    if kind == "even":        # even kernels: real spectra
        return synth.random_kernels(g.nz, g.nt, g.px, g.py, seed=seed, even=True)
    if kind == "d4":          # the square's symmetries: real spectra of {|kx|, |ky|}
        return synth.random_kernels(g.nz, g.nt, g.px, g.py, seed=seed, d4=True)
    return kspace_table(g, MED_CFG1)[0]


def _expect_fold(g, kind):
    return kind in ("d4", "kspace") and g.px == g.py


def _ref_ops(h, g):
    Hf = oracle.table_spectrum(h)
    return (lambda x: oracle.forward_fft(Hf, x, g)), (lambda y: oracle.adjoint_fft(Hf, y, g))


@pytest.mark.parametrize("g", [CFG1, RAGGED, RECT, SMALLP, P48, RECT3],
                         ids=["cfg1", "ragged", "rect", "p16", "p48", "rect24x96"])
@pytest.mark.parametrize("kind", ["random", "even", "d4", "kspace"])
@pytest.mark.parametrize("fp64", [False, True])
def test_forward_and_adjoint_match_oracle(g, kind, fp64):
    if kind == "d4" and g.px != g.py:
        pytest.skip("the square's symmetries need a square padded grid")
    h = _tables(g, kind, seed=g.nx)
    A, AT = _ref_ops(h, g)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, fp64=fp64)
    info = plan.info()
    assert info["real_table"] == (0 if kind == "random" else 1)
    assert info["folded"] == (1 if _expect_fold(g, kind) and not fp64 else 0)
    rho = synth.blobs(g.nx, g.ny, g.nz, count=8, seed=1) + 0.1 * synth.gaussian_object(g.nx, g.ny, g.nz, 2)
    y = synth.gaussian_field((g.nt, g.ny, g.nx), seed=3)
    tol = 1e-12 if fp64 else 1e-5
    d = host(plan.forward(cuda(rho, fp64)))
    assert oracle.rel_l2(d, A(rho)) < tol
    assert oracle.rel_linf(d, A(rho)) < 10 * tol
    a = host(plan.adjoint(cuda(y, fp64)))
    assert oracle.rel_l2(a, AT(y)) < tol
    assert oracle.rel_linf(a, AT(y)) < 10 * tol


@pytest.mark.parametrize("fp64", [False, True])
def test_forced_complex_equals_real_path(fp64):
    g = CFG1
    h = _tables(g, "kspace")
    pr = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, fp64=fp64, fold=False)
    pc = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, fp64=fp64, force_complex=True)
    assert pr.info()["real_table"] == 1 and pc.info()["real_table"] == 0
    assert pc.info()["table_bytes"] == 2 * pr.info()["table_bytes"]
    rho = synth.blobs(g.nx, g.ny, g.nz, count=8, seed=4)
    dr, dc = host(pr.forward(cuda(rho, fp64))), host(pc.forward(cuda(rho, fp64)))
    assert oracle.rel_l2(dr, dc) < (1e-13 if fp64 else 1e-6)


@pytest.mark.parametrize("g", [CFG1, oracle.Grid.square(48, 12, 40), SMALLP,
                               oracle.Grid.square(40, 12, 20, pad=96)],
                         ids=["cfg1", "n48", "p16", "p96"])
@pytest.mark.parametrize("B", [1, 3])
def test_folded_equals_unfolded(g, B):
    """One table row per representative {|kx|, |ky|} gives what one row per bin gives."""
    h = _tables(g, "d4", seed=31)
    pf = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, max_batch=B)
    pu = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, max_batch=B, fold=False)
    fi, ui = pf.info(), pu.info()
    assert fi["folded"] == 1 and ui["folded"] == 0
    assert fi["radial"] == 0     # random D4 kernels: representatives of one radius differ
    P = g.px
    assert fi["table_rows"] == (P // 2 + 1) * (P // 2 + 2) // 2 and ui["table_rows"] == ui["bins"]
    # rows are stored in blocks of 32
    assert fi["table_bytes"] * ((ui["bins"] + 31) // 32) == ui["table_bytes"] * ((fi["table_rows"] + 31) // 32)
    xs = np.stack([synth.blobs(g.nx, g.ny, g.nz, count=4, seed=40 + s) for s in range(B)])
    ys = np.stack([synth.gaussian_field((g.nt, g.ny, g.nx), 50 + s) for s in range(B)])
    for a, b in ((pf.forward(cuda(xs)), pu.forward(cuda(xs))),
                 (pf.adjoint(cuda(ys)), pu.adjoint(cuda(ys)))):
        a, b = host(a), host(b)
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max()


def test_fold_rejected_when_not_symmetric():
    g = CFG1
    h = _tables(g, "d4", seed=32)
    P = g.px
    h[3, 10, 1, 2] += 0.5           # breaks ux <-> uy for one plane ...
    h[3, 10, P - 1, P - 2] += 0.5   # ... but keeps h(-u) = h(u): still a real spectrum
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h)
    assert plan.info()["folded"] == 0 and plan.info()["real_table"] == 1


@pytest.mark.parametrize("fp64", [False, True])
def test_adjoint_identity_on_gpu(fp64):
    """Eq. 9 evaluated with the FP64 inner-product kernel."""
    import torch
    g = CFG1
    h = _tables(g, "random", seed=5)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, fp64=fp64)
    x = cuda(synth.gaussian_object(g.nx, g.ny, g.nz, 6), fp64)
    y = cuda(synth.gaussian_field((g.nt, g.ny, g.nx), 7), fp64)
    Ax, ATy = plan.forward(x), plan.adjoint(y)
    lhs, rhs = plan.dot(Ax, y), plan.dot(x, ATy)
    nAx, ny_ = np.sqrt(plan.dot(Ax, Ax)), np.sqrt(plan.dot(y, y))
    gap = abs(lhs - rhs) / (nAx * ny_)
    assert gap < (1e-12 if fp64 else 1e-6), gap
    # the FP64 dot itself against numpy
    ref = float(np.dot(host(Ax).ravel(), host(y).ravel()))
    assert abs(lhs - ref) <= 1e-12 * nAx * ny_
    # deterministic: same bits twice
    assert plan.dot(Ax, y) == lhs
    torch.cuda.synchronize()


@pytest.mark.parametrize("kind", ["random", "even"])
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("B", [2, 3, 6])  # 2- and 4-volume groups and their tails
def test_batch_equals_single_volumes(kind, fp64, B):
    g = RAGGED
    h = _tables(g, kind, seed=8)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, max_batch=B, fp64=fp64)
    xs = np.stack([synth.blobs(g.nx, g.ny, g.nz, count=3, seed=s) for s in range(B)])
    ys = np.stack([synth.gaussian_field((g.nt, g.ny, g.nx), 20 + s) for s in range(B)])
    A, AT = _ref_ops(h, g)
    d = host(plan.forward(cuda(xs, fp64)))
    a = host(plan.adjoint(cuda(ys, fp64)))
    tol = 1e-12 if fp64 else 1e-5
    for b in range(B):
        assert oracle.rel_l2(d[b], A(xs[b])) < tol
        assert oracle.rel_l2(a[b], AT(ys[b])) < tol
    one = host(plan.forward(cuda(xs[1:2], fp64)))
    assert np.abs(one[0] - d[1]).max() <= 10 * tol * np.abs(d[1]).max()


def test_host_pointers_equal_device_pointers():
    import torch
    g = RAGGED
    h = _tables(g, "even", seed=9)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, max_batch=2)
    x = np.ascontiguousarray(synth.gaussian_object(g.nx, g.ny, g.nz, 10)[None].repeat(2, 0), np.float32)
    d_host = plan.forward(torch.from_numpy(x))          # CPU tensor in, CPU tensor out
    d_dev = plan.forward(torch.from_numpy(x).cuda())
    assert d_host.device.type == "cpu"
    assert torch.equal(d_host, d_dev.cpu())
    a_host = plan.adjoint(d_host)
    a_dev = plan.adjoint(d_dev)
    assert torch.equal(a_host, a_dev.cpu())


def test_gradient_and_residual():
    g = CFG1
    h = _tables(g, "kspace")
    A, AT = _ref_ops(h, g)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h)
    x = synth.blobs(g.nx, g.ny, g.nz, count=5, seed=11)
    y = A(synth.blobs(g.nx, g.ny, g.nz, count=5, seed=12))
    grad, r2 = plan.gradient(cuda(x), cuda(y))
    r = A(x) - y
    assert oracle.rel_l2(host(grad), AT(r)) < 1e-5
    assert abs(r2 - float(np.dot(r.ravel(), r.ravel()))) < 1e-5 * float(np.dot(r.ravel(), r.ravel()))


def test_power_norm_matches_oracle():
    g = oracle.Grid.square(16, 8, 32)
    h = _tables(g, "kspace")
    v0 = synth.gaussian_field((g.nz, g.ny, g.nx), 13)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h)
    L_gpu = plan.power_norm(cuda(v0), 30)
    L_ref = oracle.power_norm(oracle.Operator(g, h=h), v0, 30)
    assert abs(L_gpu - L_ref) / L_ref < 1e-5


@pytest.mark.parametrize("lam_rel", [0.0, 1e-3])
def test_fista_100_iterations_match_oracle(lam_rel):
    """100 FISTA iterations, same L and x0 = 0, FP32 path within 1e-5 of FP64."""
    g = CFG1
    h = _tables(g, "kspace")
    op = oracle.Operator(g, h=h)
    p0 = synth.vessel_phantom(g.nx, g.nz, seed=14)
    clean = op.A(p0)
    y = clean + 0.05 * np.sqrt(np.mean(clean ** 2)) * synth.gaussian_field(clean.shape, 15)
    L = 1.01 * oracle.power_norm(op, synth.gaussian_field(op.obj_shape, 16), 50)
    lam = lam_rel * float(np.abs(op.AT(y)).max())
    ref = oracle.fista(op, y, L, iters=100, lam=lam, track=True)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h)
    x, rep = plan.fista(cuda(y), iters=100, lam=lam, L=L)
    assert rep["iters"] == 100 and rep["L"] == L
    err = oracle.rel_l2(host(x), ref.x)
    assert err < 1e-5, err
    assert abs(rep["resid2_first"] - ref.resid2[0]) < 1e-5 * ref.resid2[0]
    assert abs(rep["resid2_last"] - ref.resid2[-1]) < 1e-4 * ref.resid2[-1]
    # graph replay: a second solve gives the same bits
    x2, _ = plan.fista(cuda(y), iters=100, lam=lam, L=L)
    assert np.array_equal(host(x2), host(x))


def test_fista_batched_and_warm_start():
    g = RAGGED
    h = _tables(g, "even", seed=17)
    op = oracle.Operator(g, h=h)
    ys = np.stack([op.A(synth.blobs(g.nx, g.ny, g.nz, count=3, seed=s)) for s in range(3)])
    L = 1.01 * oracle.power_norm(op, synth.gaussian_field(op.obj_shape, 18), 60)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, max_batch=3)
    x, _ = plan.fista(cuda(ys), iters=20, L=L)
    for b in range(3):
        assert oracle.rel_l2(host(x)[b], oracle.fista(op, ys[b], L, iters=20).x) < 1e-5
    # warm start: 10 + 10 iterations from x_10 is not the same as 20 (momentum restarts),
    # but it must equal the oracle started from the same x_10
    x10, _ = plan.fista(cuda(ys[:1]), iters=10, L=L)
    xw, _ = plan.fista(cuda(ys[:1]), x=x10.clone(), iters=10, L=L, warm_start=True)
    ref10 = oracle.fista(op, ys[0], L, iters=10)
    refw = oracle.fista(op, ys[0], L, iters=10, x0=ref10.x)
    assert oracle.rel_l2(host(xw)[0], refw.x) < 1e-5


def test_fista_estimates_L_when_not_given():
    g = oracle.Grid.square(16, 8, 32)
    h = _tables(g, "kspace")
    op = oracle.Operator(g, h=h)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h)
    y = op.A(synth.blobs(g.nx, g.ny, g.nz, count=3, seed=19))
    _, rep = plan.fista(cuda(y), iters=5, L=0.0, power_iters=80)
    L_ref = oracle.power_norm(op, synth.gaussian_field(op.obj_shape, 20), 2000)
    est = rep["L"] / 1.01
    # power iteration approaches ||H*H|| from below (Rayleigh bound), within 1% after 80 steps
    assert 0.99 * L_ref < est <= L_ref * (1 + 1e-5), (est, L_ref)


def test_kspace_generated_table_matches_oracle_library():
    """Library generated on the device from the medium (Eq. 1-2 closed form)
    vs the oracle's one-solve library, through the operator."""
    g = CFG1
    med = MED_CFG1
    mz = oracle.mz_for(g.nz, g.nt, med)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py,
                medium=Medium(med.c, med.dx, med.dy, med.dz, med.dt, mz, 1))
    assert plan.info()["real_table"] == 1
    h = oracle.table_kspace_solve(g, med, mz)
    A, AT = _ref_ops(h, g)
    rho = synth.blobs(g.nx, g.ny, g.nz, count=8, seed=21)
    y = synth.gaussian_field((g.nt, g.ny, g.nx), 22)
    assert oracle.rel_l2(host(plan.forward(cuda(rho))), A(rho)) < 1e-5
    assert oracle.rel_l2(host(plan.adjoint(cuda(y))), AT(y)) < 1e-5


def test_edge_cases():
    import torch
    g = SMALLP
    h = _tables(g, "random", seed=23)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, max_batch=2)
    empty = torch.empty((0, g.nz, g.ny, g.nx), device="cuda")
    out = plan.forward(empty)
    assert out.shape[0] == 0
    with pytest.raises(PatError):
        plan.forward(torch.zeros((3, g.nz, g.ny, g.nx), device="cuda"))  # > max_batch
    # zero object -> zero data exactly
    z = plan.forward(torch.zeros((1, g.nz, g.ny, g.nx), device="cuda"))
    assert torch.count_nonzero(z) == 0
    # single voxel, single depth, single sample grid
    g1 = oracle.Grid(nx=1, ny=1, nz=1, nt=1, px=16, py=16)
    h1 = _tables(g1, "random", seed=24)
    p1 = Plan(1, 1, 1, 1, 16, 16, table=h1)
    d1 = host(p1.forward(cuda(np.array([[[2.0]]]))))
    assert abs(d1[0, 0, 0] - 2.0 * h1[0, 0, 0, 0]) < 1e-6 * abs(h1[0, 0, 0, 0]) + 1e-7


def test_cfg2_sampled_outputs_full_size():
    """128^2 -> 256^2, 64 depths, 256 samples, table generated on the device
    (the benchmarked configuration): sampled time samples of H rho and sampled
    depths of H* d against the oracle's closed-form library for those samples."""
    g = oracle.Grid.square(128, 64, 256)
    med = MED_50UM
    mz = oracle.mz_for(g.nz, g.nt, med)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py,
                medium=Medium(med.c, med.dx, med.dy, med.dz, med.dt, mz, 1))
    rho = synth.vessel_phantom(g.nx, g.nz, seed=0)
    d = host(plan.forward(cuda(rho)))
    for t in (0, 97, 255):
        Hf = oracle.table_kspace_closed(g, med, mz, t_idx=[t])
        gt = oracle.Grid(g.nx, g.ny, g.nz, 1, g.px, g.py)
        ref = oracle.forward_fft(Hf, rho, gt)[0]
        scale = np.abs(d).max()
        assert np.abs(d[t] - ref).max() < 1e-5 * scale, t
    y = synth.gaussian_field((g.nt, g.ny, g.nx), 1)
    a = host(plan.adjoint(cuda(y)))
    for j in (0, 63):
        Hf = oracle.table_kspace_closed(g, med, mz, z_idx=[j])
        gz = oracle.Grid(g.nx, g.ny, 1, g.nt, g.px, g.py)
        ref = oracle.adjoint_fft(Hf, y, gz)[0]
        assert oracle.rel_l2(a[j], ref) < 1e-5, j


def test_three_times_power_of_two_sampled_outputs():
    """96^2 -> 192^2 (a 3 * 2^k padded grid), 32 depths, 128 samples, table
    generated on the device: sampled time samples of H rho and depths of H* d
    against the oracle's closed-form library for those samples (the oracle's
    192-point transforms are DFTs of the definition, so the grid stays modest;
    the stage tests cover 384 and 768 against numpy's FFT)."""
    g = oracle.Grid.square(96, 32, 128, pad=192)
    med = MED_50UM
    mz = oracle.mz_for(g.nz, g.nt, med)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py,
                medium=Medium(med.c, med.dx, med.dy, med.dz, med.dt, mz, 1))
    assert plan.info()["folded"] == 1
    rho = synth.vessel_phantom(g.nx, g.nz, seed=2)
    d = host(plan.forward(cuda(rho)))
    for t in (0, 77, 127):
        Hf = oracle.table_kspace_closed(g, med, mz, t_idx=[t])
        gt = oracle.Grid(g.nx, g.ny, g.nz, 1, g.px, g.py)
        ref = oracle.forward_fft(Hf, rho, gt)[0]
        assert np.abs(d[t] - ref).max() < 1e-5 * np.abs(d).max(), t
    y = synth.gaussian_field((g.nt, g.ny, g.nx), 4)
    a = host(plan.adjoint(cuda(y)))
    for j in (0, 31):
        Hf = oracle.table_kspace_closed(g, med, mz, z_idx=[j])
        gz = oracle.Grid(g.nx, g.ny, 1, g.nt, g.px, g.py)
        ref = oracle.adjoint_fft(Hf, y, gz)[0]
        assert oracle.rel_l2(a[j], ref) < 1e-5, j


def test_largest_padded_grid_1024():
    """The largest supported padded length, 512^2 -> 1024^2 (8 depths, 16
    samples): a library generated on the device (real, D4-folded, radially
    shared: 131,841 representatives) against the oracle's closed-form
    library at sampled time samples and depths, and an asymmetric random
    library (complex spectra, one row per bin) against the oracle's operator."""
    g = oracle.Grid.square(512, 8, 16)
    med = MED_50UM
    mz = oracle.mz_for(g.nz, g.nt, med)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py,
                medium=Medium(med.c, med.dx, med.dy, med.dz, med.dt, mz, 1))
    info = plan.info()
    assert info["folded"] == 1 and info["radial"] == 1, info
    rho = synth.vessel_phantom(g.nx, g.nz, seed=3)
    d = host(plan.forward(cuda(rho)))
    for t in (0, 15):
        Hf = oracle.table_kspace_closed(g, med, mz, t_idx=[t])
        gt = oracle.Grid(g.nx, g.ny, g.nz, 1, g.px, g.py)
        ref = oracle.forward_fft(Hf, rho, gt)[0]
        assert np.abs(d[t] - ref).max() < 1e-5 * np.abs(d).max(), t
    y = synth.gaussian_field((g.nt, g.ny, g.nx), 6)
    a = host(plan.adjoint(cuda(y)))
    for j in (0, 7):
        Hf = oracle.table_kspace_closed(g, med, mz, z_idx=[j])
        gz = oracle.Grid(g.nx, g.ny, 1, g.nt, g.px, g.py)
        ref = oracle.adjoint_fft(Hf, y, gz)[0]
        assert oracle.rel_l2(a[j], ref) < 1e-5, j
    plan.close()
    g2 = oracle.Grid(nx=512, ny=512, nz=2, nt=2, px=1024, py=1024)
    h = synth.random_kernels(g2.nz, g2.nt, g2.px, g2.py, seed=7)
    A, AT = _ref_ops(h, g2)
    p2 = Plan(g2.nx, g2.ny, g2.nz, g2.nt, g2.px, g2.py, table=h)
    assert p2.info()["real_table"] == 0
    r2 = synth.blobs(g2.nx, g2.ny, g2.nz, count=6, seed=8)
    y2 = synth.gaussian_field((g2.nt, g2.ny, g2.nx), seed=9)
    assert oracle.rel_l2(host(p2.forward(cuda(r2))), A(r2)) < 1e-5
    assert oracle.rel_l2(host(p2.adjoint(cuda(y2))), AT(y2)) < 1e-5


def test_in_vivo_geometry_768():
    """The in vivo scan grid (384 x 326 transverse, padded to 768 x 768, a
    3 * 2^k length) with an asymmetric random library: H and H* against the
    FP64 oracle (few depths and samples keep the oracle's 768-point DFTs
    within seconds)."""
    g = oracle.Grid(nx=384, ny=326, nz=2, nt=3, px=768, py=768)
    h = synth.random_kernels(g.nz, g.nt, g.px, g.py, seed=5)
    A, AT = _ref_ops(h, g)
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h)
    rho = synth.blobs(g.nx, g.ny, g.nz, count=6, seed=1)
    y = synth.gaussian_field((g.nt, g.ny, g.nx), seed=2)
    assert oracle.rel_l2(host(plan.forward(cuda(rho))), A(rho)) < 1e-5
    assert oracle.rel_l2(host(plan.adjoint(cuda(y))), AT(y)) < 1e-5


def test_fista_100_cfg2_matches_oracle():
    """The benchmarked reconstruction: 128^2 -> 256^2, 64 depths, 256 samples,
    dx = 50 um, dt = 10 ns, vessel phantom + 5 % noise, 100 FISTA iterations
    (lambda = 0, x0 = 0) on the plan the bench uses (library generated on the
    device, real spectra, D4-folded: the radix-16 x 16 transforms, the folded
    contraction grid and the fused residual / step passes at full size).
    The oracle runs the same iterations on its closed-form library (complex128
    full planes, ~17 GB of host memory) with the same L."""
    g = oracle.Grid.square(128, 64, 256)
    med = MED_50UM
    mz = oracle.mz_for(g.nz, g.nt, med)
    Hf = oracle.table_kspace_closed(g, med, mz)
    op = oracle.Operator(g, Hf=Hf)
    p0 = synth.vessel_phantom(g.nx, g.nz, seed=0)
    clean = op.A(p0)
    y = clean + 0.05 * np.sqrt(np.mean(clean ** 2)) * synth.gaussian_field(clean.shape, seed=1000)
    L = 1.01 * oracle.power_norm(op, synth.gaussian_field(op.obj_shape, 3), 20)
    ref = oracle.fista(op, y, L, iters=100, track=True)
    del op, Hf
    plan = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py,
                medium=Medium(med.c, med.dx, med.dy, med.dz, med.dt, mz, 1))
    assert plan.info()["folded"] == 1 and plan.info()["real_table"] == 1
    x, rep = plan.fista(cuda(y), iters=100, L=L)
    err = oracle.rel_l2(host(x), ref.x)
    assert err < 1e-5, err
    assert abs(rep["resid2_first"] - ref.resid2[0]) < 1e-5 * ref.resid2[0]
    assert abs(rep["resid2_last"] - ref.resid2[-1]) < 1e-4 * ref.resid2[-1]


@pytest.mark.parametrize("nz,nt", [(72, 40), (64, 256), (16, 33), (128, 64)],
                         ids=["z72_t40", "z64_t256", "z16_t33", "z128_t64"])
@pytest.mark.parametrize("B", [1, 3])
def test_folded_table_stream_shapes(nz, nt, B):
    """The folded contractions at depth / time counts beyond the small test
    grids: a ragged last z-group (72 depths = 18 groups of 4, more than the 16
    groups one adjoint z-chunk holds), ragged last time blocks (40 and 33
    samples), the benchmark's counts, and a 128-depth table: folded ==
    unfolded, and both equal the FP64 oracle."""
    g = oracle.Grid.square(24, nz, nt, pad=64)
    h = _tables(g, "d4", seed=nz + nt)
    pf = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, max_batch=B)
    pu = Plan(g.nx, g.ny, g.nz, g.nt, g.px, g.py, table=h, max_batch=B, fold=False)
    assert pf.info()["folded"] == 1
    xs = np.stack([synth.blobs(g.nx, g.ny, g.nz, count=4, seed=60 + s) for s in range(B)])
    ys = np.stack([synth.gaussian_field((g.nt, g.ny, g.nx), 70 + s) for s in range(B)])
    A, AT = _ref_ops(h, g)
    df, du = host(pf.forward(cuda(xs))), host(pu.forward(cuda(xs)))
    af, au = host(pf.adjoint(cuda(ys))), host(pu.adjoint(cuda(ys)))
    pf.check()
    assert np.abs(df - du).max() <= 1e-6 * np.abs(du).max()
    assert np.abs(af - au).max() <= 1e-6 * np.abs(au).max()
    for b in range(B):
        assert oracle.rel_l2(df[b], A(xs[b])) < 1e-5
        assert oracle.rel_l2(af[b], AT(ys[b])) < 1e-5
