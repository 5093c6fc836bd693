"""GPU parity of the pixel-exact near field (dbie_set_quadrature(-1): the lambda = 0 kernel
integrated exactly over every pixel at points with z <= near_z) with the oracle's exact rule:
B, grad B and dB/dlambda in both precisions, the objective and its lambda-gradient, the Hessian,
the fixed-lambda and implicit adjoints, the simplex search, the closed form on uniform data, the
height switch, a batched solve mixing rules, and the argument errors.

Gates are those of the midpoint rule (gates.py) on tolerance scales that add the correction's
own absolute-value sums; the GPU integrates the 7 x 7 pixels around a point exactly in FP64 and
the other pixels by a 3 x 3 Gauss rule in FP32 (mixed form), whose deviation from the exact
integrals is below 1e-7 of the scale."""
import numpy as np
import pytest

import oracle
from gates import TOL_FP64, abs_scales, check_B, check_grad, oracle_boundary
from synth.active_region import Magnetogram
from test_gpu_eval import random_mag, random_points
from test_oracle_pins import square_integral

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbie():
    import paper_1306_1122_gb300 as d
    return d


def pxe_scales(mag, xyz, lam, near_z):
    """Tolerance scales: the midpoint absolute-value sums at lambda and at 0 (the subtracted
    midpoint part), plus, at corrected points, the largest |B0| of the 7 x 7 pixels around the
    point (an exact pixel integral is at most one solid angle) and 3 / z times it for the
    derivatives."""
    sB, sG = abs_scales(mag, xyz, lam)
    s0B, s0G = abs_scales(mag, xyz, np.zeros_like(np.asarray(lam, np.float64)))
    xyz = np.asarray(xyz, np.float64)
    comps = [np.abs(np.asarray(c, np.float64)) for c in (mag.Bx, mag.By, mag.Bz)]
    wB = np.zeros((len(xyz), 3))
    for n, (x, y, z) in enumerate(xyz):
        if z > near_z:
            continue
        i0 = int(np.rint((x - mag.x0) / mag.hx))
        j0 = int(np.rint((y - mag.y0) / mag.hy))
        sl = (slice(max(j0 - 3, 0), max(j0 + 4, 0)), slice(max(i0 - 3, 0), max(i0 + 4, 0)))
        for p in range(3):
            blk = comps[p][sl]
            wB[n, p] = blk.max() if blk.size else 0.0
    return sB + s0B + wB, sG + s0G + 3.0 * wB / xyz[:, 2:3]


def _mag_h(nx, ny, seed, h):
    m = random_mag(nx, ny, seed, x0=-3.0 * h, y0=2.0 * h, h=h)
    return m


@pytest.mark.parametrize("nx,ny,h,n", [(40, 36, 1.0, 160), (33, 29, 0.5, 120)])
@pytest.mark.parametrize("precision", [1, 0])
def test_pxe_eval_matches_oracle(dbie, nx, ny, h, n, precision):
    mag = _mag_h(nx, ny, 400 + nx, h)
    xyz, lam = random_points(mag, n, 401 + nx, zlo=0.3 * h, zhi=3.0 * h, lam=0.3 / h)
    near_z = 2.0 * h
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    r = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), grad=True, dlam=True,
               options=dbie.Options(precision=precision))
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in r.items()}
    bd = oracle_boundary(mag)
    x64, l64 = xyz.astype(np.float64), lam.astype(np.float64)
    B, G, dl = oracle.field(bd, x64, l64, quad_order=-1, pxe_near_z=near_z)
    Bm, _, _ = oracle.field(bd, x64, l64)
    sB, sG = pxe_scales(mag, xyz, l64, near_z)
    near = xyz[:, 2] <= near_z
    assert near.sum() >= n // 3 and (~near).sum() >= 5
    # the correction is far above every gate at the corrected points, absent at the others
    assert np.median(np.abs(B - Bm)[near].max(1) / sB[near].max(1)) > 1e-4
    assert np.all(B[~near] == Bm[~near])
    if precision == 1:
        assert np.all(np.abs(got["B"] - B) <= TOL_FP64 * sB)
        assert np.all(np.abs(got["gradB"] - G) <= TOL_FP64 * sG[:, :, None])
        assert np.all(np.abs(got["dBdlam"] - dl) <= TOL_FP64 * (np.abs(dl) + sB * 100))
    else:
        rb = check_B(got["B"], B, sB)
        assert rb["bad"].size == 0, rb
        rg = check_grad(got["gradB"], G, sG[:, :, None])
        assert rg["ok"], rg
        assert check_grad(got["dBdlam"], dl, np.abs(dl).max())["ok"]
    f.close()


def test_pxe_uniform_field_is_the_solid_angle_on_gpu(dbie):
    """Uniform B0 on (2a+1)^2 unit pixels, lambda = 0, point above the centre: the solid angle of
    the pixels' square over 2 pi (closed form), no lattice term (the midpoint rule is 0.24 off at
    z = 0.5, 8e-3 at z = 1)."""
    a = 60
    n = 2 * a + 1
    one = np.ones((n, n), np.float32)
    mag = Magnetogram(n, n, one, one, one, x0=-a, y0=-a)
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    z = np.array([0.5, 1.0, 2.0], np.float32)
    xyz = np.stack([np.zeros(3), np.zeros(3), z], 1).astype(np.float32)
    for prec, tol in ((1, 1e-11), (0, 2e-6)):
        r = f.eval(torch.from_numpy(xyz), torch.zeros((3, 3)), options=dbie.Options(precision=prec))
        torch.cuda.synchronize()
        B = r["B"].cpu().numpy()
        for k, zz in enumerate(z.astype(np.float64)):
            exact = square_integral(zz, a + 0.5, 0.0)
            assert np.all(np.abs(B[k] - exact) < tol), (prec, zz, B[k] - exact)
    f.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_pxe_objective_and_hessian_match_oracle(dbie, precision):
    mag = random_mag(36, 32, 410)
    xyz, lam32 = random_points(mag, 200, 411, zlo=0.5, zhi=2.5, lam=0.15)
    lam = np.abs(lam32.astype(np.float64))
    gs = mag.hx / 6.0
    bd = oracle_boundary(mag)
    x64 = xyz.astype(np.float64)
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    opt = dbie.Options(precision=precision)
    r = f.objective(torch.from_numpy(xyz), torch.from_numpy(lam.astype(np.float32)), opt)
    h = f.hessian(torch.from_numpy(xyz), torch.from_numpy(lam), opt)
    torch.cuda.synchronize()
    lam_f = lam.astype(np.float32).astype(np.float64)
    fo, go, po, do = oracle.objective_grad(bd, x64, lam_f, gs, pxe_near_z=2.0)
    phi, grad, H, _ = oracle.hessian(bd, x64, lam, gs, pxe_near_z=2.0)
    p0, _, _, _ = oracle.hessian(bd, x64, lam, gs)
    assert np.median(np.abs(phi - p0)) > 1e-3          # the correction moves Phi
    got = {k: v.cpu().numpy() for k, v in r.items()}
    gh = {k: v.cpu().numpy() for k, v in h.items()}
    if precision == 1:
        assert np.allclose(got["phi"], po, rtol=1e-9, atol=1e-12)
        assert np.allclose(got["dphi"], do, rtol=1e-7, atol=1e-9 * np.abs(do).max())
        assert np.allclose(gh["phi"], phi, rtol=1e-9, atol=1e-12)
        assert np.abs(gh["grad"] - grad).max() <= 1e-9 * np.abs(grad).max()
        assert np.abs(gh["hess"] - H).max() <= 1e-9 * np.abs(H).max()
    else:
        assert np.abs(got["phi"] - po).max() < 1e-4
        assert np.linalg.norm(got["dphi"] - do) < 1e-3 * np.linalg.norm(do)
        assert np.abs(gh["phi"] - phi).max() < 1e-4
        assert np.linalg.norm(gh["grad"] - grad) <= 1e-3 * np.linalg.norm(grad)
        assert np.linalg.norm(gh["hess"] - H) <= 1e-3 * np.linalg.norm(H)
    f.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_pxe_vjp_matches_oracle(dbie, precision):
    mag = random_mag(34, 30, 420)
    xyz, lam = random_points(mag, 260, 421, zlo=0.3, zhi=4.0)
    l64 = lam.astype(np.float64)
    gB = np.random.default_rng(422).normal(size=(260, 3))
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    gB0, _ = f.vjp(torch.from_numpy(xyz), torch.from_numpy(l64), torch.from_numpy(gB), glam=False,
                   options=dbie.Options(precision=precision))
    torch.cuda.synchronize()
    bd = oracle_boundary(mag)
    ref = oracle.vjp(bd, xyz.astype(np.float64), l64, gB, quad_order=-1)
    mid = oracle.vjp(bd, xyz.astype(np.float64), l64, gB)
    assert np.linalg.norm(ref - mid) > 1e-2 * np.linalg.norm(ref)
    err = np.linalg.norm(gB0.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= (1e-10 if precision == 1 else 1e-5), err
    # accumulate adds to what is there
    acc = torch.ones_like(gB0)
    f.vjp(torch.from_numpy(xyz), torch.from_numpy(l64), torch.from_numpy(gB), glam=False,
          options=dbie.Options(precision=precision), gB0=acc)
    torch.cuda.synchronize()
    assert torch.allclose(acc - 1.0, gB0, rtol=1e-12, atol=1e-12 * float(gB0.abs().max()))
    f.close()


def _newton(bd, pts, lam, gs, nz, mode=0):
    lam = lam.copy()
    for _ in range(30):
        _, gr, H, _ = oracle.hessian(bd, pts, lam, gs, pxe_near_z=nz, lambda_mode=mode)
        if mode == 1:
            ok = H[:, 0, 0] > 0
            st = np.where(ok, gr[:, 0] / np.where(ok, H[:, 0, 0], 1.0), 0.0)
            lam -= st[:, None]
        else:
            ok = np.linalg.eigvalsh(H)[:, 0] > 0
            Hs = np.where(ok[:, None, None], H, np.eye(3))
            st = np.where(ok[:, None], np.linalg.solve(Hs, gr[:, :, None])[:, :, 0], 0.0)
            lam -= st
        if np.abs(st).max() < 1e-15:
            break
    return lam


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("mode", [0, 1])
def test_pxe_implicit_vjp_matches_oracle(dbie, precision, mode):
    """At well-conditioned minima of the corrected objective (oracle quasi-Newton, then Newton),
    per-component and tied lambda."""
    from synth.workloads import small_ll
    w = small_ll()
    bd = oracle_boundary(w.mag)
    gs = w.mag.hx / 6.0
    nz = 2.0 * w.mag.hx
    rng = np.random.default_rng(430 + mode)
    near = w.points[w.points[:, 2] <= nz]
    pts = near[np.sort(rng.choice(len(near), min(192, len(near)), replace=False))].astype(np.float64)
    r = oracle.solve(bd, pts, oracle.Options(method=1, max_iter=80, tol=1e-13, quad_order=-1,
                                               lambda_mode=mode))
    lam = _newton(bd, pts, r["lam"], gs, nz, mode)
    _, gr, H, _ = oracle.hessian(bd, pts, lam, gs, pxe_near_z=nz, lambda_mode=mode)
    ev = np.linalg.eigvalsh(H[:, :1, :1] if mode == 1 else H)
    good = (np.abs(gr).max(1) < 1e-10) & (ev[:, 0] > 0) & (ev[:, -1] < 1e3 * ev[:, 0])
    assert good.sum() >= 32, good.sum()
    pts, lam = pts[good].astype(np.float32), lam[good]
    gB = rng.normal(size=(len(pts), 3))
    ref, v_ref, fl_ref = oracle.implicit_vjp(bd, pts.astype(np.float64), lam, gB, gs,
                                             lambda_mode=mode, pxe_near_z=nz)
    assert not fl_ref.any()
    f = dbie.DBIEField.from_magnetogram(w.mag)
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    opt = dbie.Options(precision=precision, lambda_mode=mode)
    gB0, v, fl = f.vjp_implicit(torch.from_numpy(pts), torch.from_numpy(lam), torch.from_numpy(gB),
                                options=opt)
    h = f.hessian(torch.from_numpy(pts), torch.from_numpy(lam), opt)
    torch.cuda.synchronize()
    gB0, v = gB0.cpu().numpy(), v.cpu().numpy()
    assert not fl.cpu().numpy().any()
    err = np.linalg.norm(gB0 - ref) / np.linalg.norm(ref)
    _, _, Ho, _ = oracle.hessian(bd, pts.astype(np.float64), lam, gs, pxe_near_z=nz,
                                 lambda_mode=mode)
    herr = np.linalg.norm(h["hess"].cpu().numpy() - Ho) / np.linalg.norm(Ho)
    if precision == 1:
        assert err <= 1e-9, err
        assert np.abs(v - v_ref).max() <= 1e-8 * np.abs(v_ref).max()
        assert herr <= 1e-9, herr
    else:
        assert err <= 1e-4, err
        assert herr <= 1e-3, herr
    f.close()


def test_pxe_solve_follows_oracle(dbie):
    """FP64 form: the simplex on the corrected objective takes the oracle's steps; mixed: B at the
    returned lambda meets the B gate of the rule."""
    mag = random_mag(30, 30, 440)
    rng = np.random.default_rng(441)
    pts = np.stack([rng.uniform(4, 25, 96), rng.uniform(4, 25, 96), rng.uniform(0.4, 3.0, 96)],
                   1).astype(np.float32)
    bd = oracle_boundary(mag)
    ref = oracle.solve(bd, pts.astype(np.float64), oracle.Options(quad_order=-1, max_iter=30),
                       codes_cap=64)
    mid = oracle.solve(bd, pts.astype(np.float64), oracle.Options(max_iter=30), codes_cap=64)
    assert np.mean([a != b for a, b in zip(ref["codes"], mid["codes"])]) > 0.2
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    r = f.solve(torch.from_numpy(pts), dbie.Options(precision=1, max_iter=30), codes=64)
    torch.cuda.synchronize()
    codes = [bytes(row).rstrip(b"\0").decode() for row in r["codes"].cpu().numpy()]
    same = np.array([a == b for a, b in zip(codes, ref["codes"])])
    assert same.mean() >= 0.95, same.mean()
    lam = r["lam"].cpu().numpy()
    assert np.all(np.abs(lam[same] - ref["lam"][same])
                  <= 1e-6 * np.maximum(np.abs(ref["lam"][same]), 1 / 30))
    rm = f.solve(torch.from_numpy(pts), dbie.Options(max_iter=30))
    torch.cuda.synchronize()
    lm = rm["lam"].cpu().numpy()
    B, _, _ = oracle.field(bd, pts.astype(np.float64), lm, quad_order=-1)
    sB, _ = pxe_scales(mag, pts, lm, 2.0)
    assert check_B(rm["B"].cpu().numpy(), B, sB)["bad"].size == 0
    f.close()


def test_pxe_quasi_newton_fp64_first_steps_follow_oracle(dbie):
    """FP64 quasi-Newton search with the correction: after a few accepted steps the lambda of the
    GPU and of the oracle's BFGS agree."""
    mag = random_mag(28, 28, 450)
    rng = np.random.default_rng(451)
    pts = np.stack([rng.uniform(4, 23, 64), rng.uniform(4, 23, 64), rng.uniform(0.4, 2.0, 64)],
                   1).astype(np.float32)
    bd = oracle_boundary(mag)
    ref = oracle.solve(bd, pts.astype(np.float64), oracle.Options(method=1, max_iter=3,
                                                                    quad_order=-1))
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    r = f.solve(torch.from_numpy(pts), dbie.Options(precision=1, method=1, max_iter=3))
    torch.cuda.synchronize()
    lam = r["lam"].cpu().numpy()
    close = np.all(np.abs(lam - ref["lam"]) <= 1e-7 * np.maximum(np.abs(ref["lam"]), 1e-3), axis=1)
    assert close.mean() >= 0.9, close.mean()
    f.close()


def test_pxe_height_switch_batched_and_errors(dbie):
    import paper_1306_1122_gb300._native as N
    mag = random_mag(26, 24, 460)
    xyz, lam = random_points(mag, 80, 461, zlo=0.4, zhi=3.0)
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    g = dbie.DBIEField.from_magnetogram(mag)
    # near_z = 0: no correction, the midpoint rule's bits
    for prec in (1, 0):
        o = dbie.Options(precision=prec, near_z=0.0)
        a = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), grad=True, options=o)
        b = g.eval(torch.from_numpy(xyz), torch.from_numpy(lam), grad=True, options=o)
        torch.cuda.synchronize()
        assert torch.equal(a["B"], b["B"]) and torch.equal(a["gradB"], b["gradB"])
    # a batched solve mixing the two rules equals the solves one by one
    pts = torch.from_numpy(xyz)
    opt = dbie.Options(precision=1, max_iter=20)
    rb = dbie.solve_batched([f, g], [pts, pts], opt)
    ra, rg = f.solve(pts, opt), g.solve(pts, opt)
    torch.cuda.synchronize()
    for got, one in zip(rb, (ra, rg)):
        assert torch.allclose(got["B"], one["B"], rtol=1e-9, atol=1e-9 * float(one["B"].abs().max()))
    assert not torch.allclose(ra["B"], rg["B"], rtol=1e-6)
    # back to pixel centres: the same bits as a context that never changed its rule
    f.set_quadrature(0)
    a = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam))
    b = g.eval(torch.from_numpy(xyz), torch.from_numpy(lam))
    torch.cuda.synchronize()
    assert torch.equal(a["B"], b["B"])
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    with pytest.raises(N.DBIEError) as e:
        f.noise_var(torch.from_numpy(xyz), torch.from_numpy(lam.astype(np.float64)))
    assert e.value.status == N.DBIE_EINVAL
    with pytest.raises(N.DBIEError):
        f.set_quadrature(-2)
    f.close()
    g.close()


def test_pxe_full_size_ll128_sampled(dbie):
    """The bench's workload at full size with the exact near field: all 131,072 points of the
    128^2 Low & Lou case through the full simplex search on the GPU (mixed), then on a seeded
    sample of 384 points (half of them at z <= 2 px) B at the GPU's lambda against the oracle's
    exact rule, and the fixed-lambda adjoint of the sample against the oracle's."""
    from synth import workloads
    w = workloads.ll128()
    f = dbie.DBIEField.from_magnetogram(w.mag)
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    pts = torch.from_numpy(w.points).cuda()
    r = f.solve(pts)
    torch.cuda.synchronize()
    B, lam = r["B"].cpu().numpy(), r["lam"].cpu().numpy()
    assert np.isfinite(B).all() and (r["status"].cpu().numpy() >= 0).all()
    rng = np.random.default_rng(470)
    near = np.nonzero(w.points[:, 2] <= 2.0)[0]
    far = np.nonzero(w.points[:, 2] > 2.0)[0]
    idx = np.sort(np.concatenate([rng.choice(near, 192, replace=False),
                                  rng.choice(far, 192, replace=False)]))
    bd = oracle_boundary(w.mag)
    x64 = w.points[idx].astype(np.float64)
    Bo, _, _ = oracle.field(bd, x64, lam[idx], quad_order=-1)
    sB, _ = pxe_scales(w.mag, w.points[idx], lam[idx], 2.0)
    rb = check_B(B[idx], Bo, sB)
    assert rb["bad"].size == 0, rb
    gB = rng.normal(size=(len(idx), 3))
    gB0, _ = f.vjp(torch.from_numpy(w.points[idx]), torch.from_numpy(lam[idx]),
                   torch.from_numpy(gB), glam=False)
    torch.cuda.synchronize()
    ref = oracle.vjp(bd, x64, lam[idx], gB, quad_order=-1)
    assert np.linalg.norm(gB0.cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)
    f.close()


def test_pxe_host_memory_path_equals_device_path(dbie):
    """The C ABI with host buffers (mem_kind = host) in the exact-near-field mode gives the same
    bits as the device path: field evaluation (B, grad B) and the fixed-lambda adjoint."""
    import ctypes

    import paper_1306_1122_gb300._native as N
    mag = random_mag(30, 26, 480)
    xyz, lam = random_points(mag, 300, 481, zlo=0.3, zhi=3.5)
    gB = np.random.default_rng(482).normal(size=(300, 3))
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    r = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), grad=True)
    gd, _ = f.vjp(torch.from_numpy(xyz), torch.from_numpy(lam.astype(np.float64)),
                  torch.from_numpy(gB), glam=False)
    torch.cuda.synchronize()
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)   # noqa: E731
    h = N.dbie_create(mag.nx, mag.ny, mag.x0, mag.y0, mag.hx, mag.hy, mag.dA,
                      *(P(c) for c in (mag.Bx, mag.By, mag.Bz)), N.DBIE_MEM_HOST, None)
    N.dbie_set_quadrature(h, -1, None)
    B = np.zeros((300, 3))
    G = np.zeros((300, 9))
    N.dbie_eval(h, 300, P(xyz), P(lam), None, N.DBIE_MEM_HOST, P(B), P(G), None, None, None)
    lam64 = np.ascontiguousarray(lam.astype(np.float64))
    g0 = np.zeros((mag.ny * mag.nx, 3))
    N.dbie_vjp(h, 300, P(xyz), P(lam64), P(gB), None, N.DBIE_MEM_HOST, P(g0), None, 0, None)
    N.dbie_destroy(h)
    f.close()
    assert np.array_equal(B, r["B"].cpu().numpy())
    assert np.array_equal(G.reshape(-1, 3, 3), r["gradB"].cpu().numpy())
    assert np.array_equal(g0.reshape(mag.ny, mag.nx, 3), gd.cpu().numpy())


@pytest.mark.parametrize("nx,ny", [(1, 7), (5, 3), (3, 300), (257, 2)])
@pytest.mark.parametrize("precision", [1, 0])
def test_pxe_ragged_grids_and_far_points(dbie, nx, ny, precision):
    """Degenerate and ragged magnetograms (a single column, fewer pixels than the 7 x 7 window,
    one tile plus a pixel) and points far outside the lattice (windows clipped to nothing, or to
    a strip): B, grad B and the adjoint against the oracle's exact rule."""
    mag = random_mag(nx, ny, 490 + nx + ny, x0=-1.0, y0=2.0, smooth=False)
    rng = np.random.default_rng(491 + nx)
    n = 120
    x = rng.uniform(mag.x0 - 6, mag.x0 + (nx - 1) + 6, n)
    y = rng.uniform(mag.y0 - 6, mag.y0 + (ny - 1) + 6, n)
    z = rng.uniform(0.3, 2.5, n)
    xyz = np.stack([x, y, z], 1).astype(np.float32)
    lam = rng.uniform(-0.3, 0.3, (n, 3)).astype(np.float32)
    gB = rng.normal(size=(n, 3))
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    opt = dbie.Options(precision=precision)
    r = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), grad=True, options=opt)
    gB0, _ = f.vjp(torch.from_numpy(xyz), torch.from_numpy(lam.astype(np.float64)),
                   torch.from_numpy(gB), glam=False, options=opt)
    torch.cuda.synchronize()
    bd = oracle_boundary(mag)
    x64, l64 = xyz.astype(np.float64), lam.astype(np.float64)
    B, G, _ = oracle.field(bd, x64, l64, quad_order=-1)
    ref = oracle.vjp(bd, x64, l64, gB, quad_order=-1)
    sB, sG = pxe_scales(mag, xyz, l64, 2.0)
    got_B, got_G = r["B"].cpu().numpy(), r["gradB"].cpu().numpy()
    if precision == 1:
        assert np.all(np.abs(got_B - B) <= TOL_FP64 * sB)
        assert np.all(np.abs(got_G - G) <= TOL_FP64 * sG[:, :, None])
        assert np.linalg.norm(gB0.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
    else:
        assert check_B(got_B, B, sB)["bad"].size == 0
        assert check_grad(got_G, G, sG[:, :, None])["ok"]
        assert np.linalg.norm(gB0.cpu().numpy() - ref) <= 1e-5 * np.linalg.norm(ref)
    f.close()


def test_pxe_gradcheck_and_set_boundary(dbie):
    """With the exact near field: torch.autograd.gradcheck through dbie_apply (FP64 form, B0 on
    multiples of 1/16 and a step of 1/64, exact in float32; the forward includes the correction
    and the backward its transpose), and dbie_set_boundary restages the rule: the same bits as a
    new context on the new magnetogram."""
    rng = np.random.default_rng(495)
    ny, nx, n = 5, 6, 5
    B0 = torch.from_numpy(np.round(rng.normal(0, 20, (ny, nx, 3)) * 16) / 16).cuda()
    f = dbie.DBIEField(B0[..., 0].float(), B0[..., 1].float(), B0[..., 2].float())
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    xyz = torch.from_numpy(np.stack([rng.uniform(0, 5, n), rng.uniform(0, 4, n),
                                     rng.uniform(0.4, 2.5, n)], 1).astype(np.float32)).cuda()
    lam = torch.from_numpy(np.round(rng.uniform(-0.4, 0.4, (n, 3)) * 4096) / 4096).cuda()
    opt = dbie.Options(precision=1)
    B0.requires_grad_(True)
    lam.requires_grad_(True)
    fn = lambda b0, l: dbie.dbie_apply(f, b0, l, xyz, opt)   # noqa: E731
    assert torch.autograd.gradcheck(fn, (B0, lam), eps=2.0 ** -10, atol=1e-5, rtol=1e-4)
    # set_boundary in the exact-near-field mode
    mag2 = random_mag(nx, ny, 496)
    f.set_boundary(torch.from_numpy(mag2.Bx).cuda(), torch.from_numpy(mag2.By).cuda(),
                   torch.from_numpy(mag2.Bz).cuda())
    a = f.eval(xyz, lam.detach().float(), grad=True)
    g = dbie.DBIEField.from_magnetogram(mag2)
    g.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    b = g.eval(xyz, lam.detach().float(), grad=True)
    torch.cuda.synchronize()
    assert torch.equal(a["B"], b["B"]) and torch.equal(a["gradB"], b["gradB"])
    f.close()
    g.close()
