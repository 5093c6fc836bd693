"""GPU parity of the nine-node element quadrature (Eq. 15, dbie_set_quadrature) with the oracle's
element rule: B, its gradient and dB/dlambda (both precisions, near field included), the
adjoint gathered back to the nodes, the lambda search, the closed form on uniform data, and the
argument errors."""
import numpy as np
import pytest

import oracle
from gates import TOL_FP64, check_B, check_grad, oracle_boundary
from synth.active_region import Magnetogram
from test_gpu_eval import random_mag, random_points
from test_oracle_pins import square_integral

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbie():
    import paper_1306_1122_gb300 as d
    return d


def q9_abs_scales(mag, xyz, lam, g):
    """Tolerance scales of the element rule: per point and component the sum over Gauss points of
    |K| |interpolated B0 x weights| (and of the gradient kernels), as the pair sums see them."""
    gx, gw = np.polynomial.legendre.leggauss(g)
    L = [lambda t: 0.5 * t * (t - 1), lambda t: 1 - t * t, lambda t: 0.5 * t * (t + 1)]
    nex, ney = (mag.nx - 1) // 2, (mag.ny - 1) // 2
    X, Y, V = [], [], [[], [], []]
    comps = [np.asarray(c, np.float64) for c in (mag.Bx, mag.By, mag.Bz)]
    for ey in range(ney):
        for ex in range(nex):
            for b in range(g):
                for a in range(g):
                    X.append(mag.x0 + (2 * ex + 1 + gx[a]) * mag.hx)
                    Y.append(mag.y0 + (2 * ey + 1 + gx[b]) * mag.hy)
                    w = gw[a] * gw[b] * mag.hx * mag.hy / (2 * np.pi)
                    for p in range(3):
                        v = sum(L[ia](gx[a]) * L[jb](gx[b]) * comps[p][2 * ey + jb, 2 * ex + ia]
                                for ia in range(3) for jb in range(3))
                        V[p].append(abs(v * w))
    X, Y, V = np.array(X), np.array(Y), [np.array(v) for v in V]
    sB = np.zeros((len(xyz), 3))
    sG = np.zeros((len(xyz), 3))
    for n, (x, y, z) in enumerate(np.asarray(xyz, np.float64)):
        dx, dy = x - X, y - Y
        r = np.sqrt(dx * dx + dy * dy + z * z)
        for p in range(3):
            lr = lam[n, p] * r
            u = lr * np.sin(lr) + np.cos(lr)
            psi = (lam[n, p] ** 2 * np.cos(lr) - 3 * u / r ** 2) / r ** 3
            sB[n, p] = np.sum(np.abs(z * u / r ** 3) * V[p])
            sG[n, p] = np.sum((np.abs(z * dx * psi) + np.abs(z * dy * psi)
                               + np.abs(u / r ** 3 + z * z * psi)) * V[p])
    return sB, sG


@pytest.mark.parametrize("nx,ny,g,n", [(33, 25, 2, 97), (41, 27, 4, 150), (29, 31, 6, 64)])
@pytest.mark.parametrize("precision", [1, 0])
def test_q9_eval_matches_oracle(dbie, nx, ny, g, n, precision):
    mag = random_mag(nx, ny, 200 + g, x0=-4.0, y0=2.0)
    xyz, lam = random_points(mag, n, 300 + g, zlo=0.4, zhi=14.0, lam=0.3)
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(g)
    r = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), grad=True, dlam=True,
               options=dbie.Options(precision=precision))
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in r.items()}
    B, G, dl = oracle.field(oracle_boundary(mag), xyz.astype(np.float64), lam.astype(np.float64),
                            quad_order=g)
    sB, sG = q9_abs_scales(mag, xyz, lam.astype(np.float64), g)
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
    # back to pixel centres: the same bits as a context that never changed its rule
    f.set_quadrature(0)
    r0 = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), options=dbie.Options(precision=precision))
    f2 = dbie.DBIEField.from_magnetogram(mag)
    r1 = f2.eval(torch.from_numpy(xyz), torch.from_numpy(lam), options=dbie.Options(precision=precision))
    torch.cuda.synchronize()
    assert torch.equal(r0["B"], r1["B"])
    f.close()
    f2.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_q9_vjp_matches_oracle(dbie, precision):
    mag = random_mag(35, 23, 210)
    xyz, lam = random_points(mag, 300, 211, zlo=0.5, zhi=12.0)
    gB = np.random.default_rng(212).normal(size=(300, 3))
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(3)
    gB0, _ = f.vjp(torch.from_numpy(xyz), torch.from_numpy(lam.astype(np.float64)),
                   torch.from_numpy(gB), glam=False, options=dbie.Options(precision=precision))
    torch.cuda.synchronize()
    ref = oracle.vjp(oracle_boundary(mag), xyz.astype(np.float64), lam.astype(np.float64), gB,
                     quad_order=3)
    err = np.linalg.norm(gB0.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= (1e-10 if precision == 1 else 1e-5), err
    f.close()


def test_q9_solve_follows_oracle(dbie):
    """FP64 form: the simplex on the element rule takes the oracle's steps; mixed: B at the
    returned lambda meets the B gate of the element rule."""
    mag = random_mag(25, 25, 220)
    rng = np.random.default_rng(221)
    pts = np.stack([rng.uniform(4, 20, 96), rng.uniform(4, 20, 96), rng.uniform(1, 8, 96)],
                   1).astype(np.float32)
    bd = oracle_boundary(mag)
    ref = oracle.solve(bd, pts.astype(np.float64), oracle.Options(quad_order=4, max_iter=30),
                       codes_cap=64)
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(4)
    r = f.solve(torch.from_numpy(pts), dbie.Options(precision=1, max_iter=30), codes=64)
    torch.cuda.synchronize()
    codes = [bytes(row).rstrip(b"\0").decode() for row in r["codes"].cpu().numpy()]
    same = np.array([a == b for a, b in zip(codes, ref["codes"])])
    assert same.mean() >= 0.95, same.mean()
    lam = r["lam"].cpu().numpy()
    assert np.all(np.abs(lam[same] - ref["lam"][same]) <= 1e-6 * np.maximum(np.abs(ref["lam"][same]), 1 / 25))
    rm = f.solve(torch.from_numpy(pts), dbie.Options(max_iter=30))
    torch.cuda.synchronize()
    lm = rm["lam"].cpu().numpy()
    B, _, _ = oracle.field(bd, pts.astype(np.float64), lm, quad_order=4)
    sB, _ = q9_abs_scales(mag, pts, lm, 4)
    assert check_B(rm["B"].cpu().numpy(), B, sB)["bad"].size == 0
    f.close()


def test_q9_uniform_field_closed_form_on_gpu(dbie):
    """Uniform B0 on (2a+1)^2 nodes: the element rule's result is the kernel integral over the
    node square to the Gauss error -- no lattice term (8e-3 for the midpoint rule at z = 1)."""
    a = 60
    n = 2 * a + 1
    one = np.ones((n, n), np.float32)
    mag = Magnetogram(n, n, one, one, one, x0=-a, y0=-a)
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(8)
    z = np.array([1.0, 2.0, 3.0], np.float32)
    xyz = np.stack([np.zeros(3), np.zeros(3), z], 1).astype(np.float32)
    for prec, tol in ((1, 2e-6), (0, 3e-6)):
        for lam in (0.0, 0.2):
            r = f.eval(torch.from_numpy(xyz), torch.from_numpy(np.full((3, 3), lam, np.float32)),
                       options=dbie.Options(precision=prec))
            torch.cuda.synchronize()
            B = r["B"].cpu().numpy()
            for k, zz in enumerate(z.astype(np.float64)):
                exact = square_integral(zz, float(a), float(np.float32(lam)))
                assert np.all(np.abs(B[k] - exact) < tol), (prec, lam, zz, B[k] - exact)
    f.close()


def test_q9_argument_errors(dbie):
    import paper_1306_1122_gb300._native as N
    even = random_mag(20, 21, 230)
    f = dbie.DBIEField.from_magnetogram(even)
    with pytest.raises(N.DBIEError) as e:
        f.set_quadrature(2)
    assert e.value.status == N.DBIE_EINVAL
    f.close()
    mag = random_mag(21, 21, 231)
    f = dbie.DBIEField.from_magnetogram(mag)
    for bad in (-2, 9):
        with pytest.raises(N.DBIEError):
            f.set_quadrature(bad)
    f.set_quadrature(3)
    xyz, lam = random_points(mag, 10, 232)
    with pytest.raises(N.DBIEError):
        f.noise_var(torch.from_numpy(xyz), torch.from_numpy(lam.astype(np.float64)))
    g = dbie.DBIEField.from_magnetogram(mag)
    with pytest.raises(N.DBIEError):
        dbie.solve_batched([f, g], [torch.from_numpy(xyz), torch.from_numpy(xyz)])
    f.close()
    g.close()


def _q9_field(dbie, seed, n=24, g=3):
    mag = random_mag(21, 19, seed)
    rng = np.random.default_rng(seed + 1)
    pts = np.stack([rng.uniform(5, 15, n), rng.uniform(5, 13, n), rng.uniform(1.0, 4.0, n)],
                   1).astype(np.float32)
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(g)
    return mag, pts, f


def test_q9_objective_gradient_and_hessian_are_consistent(dbie):
    """Element rule, FP64 form: dPhi/dlambda of dbie_objective is the central difference of its
    Phi, dbie_hessian's gradient equals it, and the Hessian is the central difference of the
    gradient (the lambda-derivative sums over Gauss points)."""
    mag, pts, f = _q9_field(dbie, 500)
    rng = np.random.default_rng(502)
    lam = rng.uniform(0.02, 0.2, (len(pts), 3))
    opt = dbie.Options(precision=1)
    P = torch.from_numpy(pts)

    def obj(l):
        r = f.objective(P, torch.from_numpy(l.astype(np.float32)), opt)
        return r["phi"].cpu().numpy(), r["dphi"].cpu().numpy()

    lam32 = lam.astype(np.float32).astype(np.float64)     # objective takes float32 lambda
    phi, dphi = obj(lam32)
    h = f.hessian(P, torch.from_numpy(lam32), opt)
    torch.cuda.synchronize()
    gh, H = h["grad"].cpu().numpy(), h["hess"].cpu().numpy()
    assert np.allclose(h["phi"].cpu().numpy(), phi, rtol=1e-10, atol=1e-13)
    assert np.abs(gh - dphi).max() <= 1e-9 * np.abs(dphi).max()
    d = 2.0 ** -10                                          # exact in float32 around lambda
    fd = np.zeros_like(dphi)
    for q in range(3):
        e = np.zeros(3)
        e[q] = d
        fd[:, q] = (obj(lam32 + e)[0] - obj(lam32 - e)[0]) / (2 * d)
    # O(d^2) truncation of the differences: ~1e-6 of the gradient's scale
    assert np.abs(fd - dphi).max() <= 1e-4 * np.abs(dphi).max(), np.abs(fd - dphi).max()
    for q in range(3):
        e = np.zeros(3)
        e[q] = 1e-5
        gp = f.hessian(P, torch.from_numpy(lam32 + e), opt)["grad"].cpu().numpy()
        gm = f.hessian(P, torch.from_numpy(lam32 - e), opt)["grad"].cpu().numpy()
        assert np.abs((gp - gm) / 2e-5 - H[:, :, q]).max() <= 1e-4 * np.abs(H).max()
    f.close()


def test_q9_quasi_newton_and_implicit_adjoint(dbie):
    """Element rule, FP64 form: the quasi-Newton search lowers Phi from its start and returns B
    equal to the oracle's element rule at its lambda.  At Newton-polished minima (the GPU's own
    gradient and Hessian) the implicit adjoint equals the fixed-lambda adjoint minus
    v . d(grad_lambda Phi)/dB0, with v the call's H^-1 dL/dlambda and the derivative of the
    gradient (lambda held in FP64) by central differences in B0 (steps of 2^-4, exact in float32)."""
    mag, pts, f = _q9_field(dbie, 510, n=48)
    opt = dbie.Options(precision=1, method=1, max_iter=60, tol=1e-14)
    P = torch.from_numpy(pts)
    r = f.solve(P, opt)
    torch.cuda.synchronize()
    lam = r["lam"].cpu().numpy()
    start = np.full_like(lam, 1.0 / (max(mag.nx, mag.ny) * mag.hx))
    phi_end = f.objective(P, torch.from_numpy(lam.astype(np.float32)), dbie.Options(precision=1))
    phi_start = f.objective(P, torch.from_numpy(start.astype(np.float32)), dbie.Options(precision=1))
    torch.cuda.synchronize()
    assert np.all(phi_end["phi"].cpu().numpy() <= phi_start["phi"].cpu().numpy() + 1e-12)
    B, _, _ = oracle.field(oracle_boundary(mag), pts.astype(np.float64), lam, quad_order=3)
    sB, _ = q9_abs_scales(mag, pts, lam, 3)
    assert np.all(np.abs(r["B"].cpu().numpy() - B) <= TOL_FP64 * sB)

    o1 = dbie.Options(precision=1)
    ln = lam.copy()
    for _ in range(30):
        h = f.hessian(P, torch.from_numpy(ln), o1)
        gr, H = h["grad"].cpu().numpy(), h["hess"].cpu().numpy()
        ok = np.linalg.eigvalsh(H)[:, 0] > 0
        Hs = np.where(ok[:, None, None], H, np.eye(3))
        st = np.where(ok[:, None], np.linalg.solve(Hs, gr[:, :, None])[:, :, 0], 0.0)
        ln -= st
        if np.abs(st).max() < 1e-15:
            break
    h = f.hessian(P, torch.from_numpy(ln), o1)
    gr, H = h["grad"].cpu().numpy(), h["hess"].cpu().numpy()
    ev = np.linalg.eigvalsh(H)
    good = (np.abs(gr).max(1) < 1e-10) & (ev[:, 0] > 0) & (ev[:, -1] < 1e3 * ev[:, 0])
    assert good.sum() >= 4, good.sum()
    Pg, lg = P[torch.from_numpy(np.nonzero(good)[0])], ln[good]
    rng = np.random.default_rng(512)
    gB = rng.normal(size=(len(lg), 3))
    gB0, v, fl = f.vjp_implicit(Pg, torch.from_numpy(lg), torch.from_numpy(gB), options=o1)
    gfix, _ = f.vjp(Pg, torch.from_numpy(lg), torch.from_numpy(gB), glam=False, options=o1)
    torch.cuda.synchronize()
    assert not fl.cpu().numpy().any()
    gB0, v, gfix = gB0.cpu().numpy(), v.cpu().numpy(), gfix.cpu().numpy()
    assert np.abs(gB0 - gfix).max() > 1e-2 * np.abs(gfix).max()   # the implicit term matters
    comps = [np.array(c, np.float32) for c in (mag.Bx, mag.By, mag.Bz)]
    g2 = dbie.DBIEField.from_magnetogram(mag)
    g2.set_quadrature(3)

    def grad_at(cs):
        g2.set_boundary(*(torch.from_numpy(c).cuda() for c in cs))
        return g2.hessian(Pg, torch.from_numpy(lg), o1)["grad"].cpu().numpy()

    dd = 2.0 ** -4
    top = np.argsort(np.abs(gB0 - gfix).ravel())[-3:]          # where the implicit term is largest
    picks = [np.unravel_index(t, gB0.shape) for t in top]
    picks += [(rng.integers(0, mag.ny), rng.integers(0, mag.nx), rng.integers(0, 3)) for _ in range(3)]
    for j, i, p in picks:
        cp = [c.copy() for c in comps]
        cm = [c.copy() for c in comps]
        cp[p][j, i] += dd
        cm[p][j, i] -= dd
        assert cp[p][j, i] - comps[p][j, i] == dd and comps[p][j, i] - cm[p][j, i] == dd
        dgrad = (grad_at(cp) - grad_at(cm)) / (2 * dd)
        ref = gfix[j, i, p] - np.sum(v * dgrad)
        scale = np.abs(gfix[j, i, p]) + np.sum(np.abs(v * dgrad))
        assert abs(gB0[j, i, p] - ref) <= 1e-6 * scale + 1e-13, (gB0[j, i, p], ref)
    g2.close()
    f.close()
