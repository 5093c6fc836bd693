"""Pins of the FP64 oracle against facts fixed by the mathematics of Eq. 6 / Eq. 16.

Each test checks the oracle against something other than its own formula: closed forms of the
kernel integral, potential fields that the lambda = 0 quadrature must reproduce, finite
differences of the oracle's own values (derivatives of Eq. 13 / dB/dlambda), invariances, an
adjoint identity, and scipy's Nelder-Mead for the simplex logic."""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle


def uniform_square(a, h, value=1.0):
    n = 2 * a + 1
    g = oracle.Grid(n, n, x0=-a * h, y0=-a * h, hx=h, hy=h)
    one = np.full((n, n), value, np.float32)
    return oracle.Boundary(g, one, one, one)


def lattice_term(z, h, lam, M=12):
    """Poisson-summation excess of the pixel sum over the integral for uniform data:
    sum over non-zero lattice frequencies of the plane-wave response exp(-z sqrt(k^2 - lam^2))."""
    s = 0.0
    for m1 in range(-M, M + 1):
        for m2 in range(-M, M + 1):
            if m1 or m2:
                k = 2 * np.pi * np.hypot(m1, m2) / h
                s += np.exp(-z * np.sqrt(k * k - lam * lam))
    return s


def square_integral(z, A, lam):
    """Integral of the DBIE kernel over the square [-A, A]^2 for a point above its centre.
    In polar form the radial integral has the antiderivative -cos(lam r)/r, so the integral is
    the angular mean of cos(lam z) - z cos(lam R')/R' with R' the distance to the square's edge."""
    if lam == 0.0:
        return 2 / np.pi * np.arctan(A * A / (z * np.sqrt(2 * A * A + z * z)))  # solid angle / 2 pi

    def F(th):
        R = A / max(abs(np.cos(th)), abs(np.sin(th)))
        Rp = np.hypot(R, z)
        return np.cos(lam * z) - z * np.cos(lam * Rp) / Rp

    v, _ = quad(F, 0, 2 * np.pi, points=[np.pi / 4 * (2 * k + 1) for k in range(4)], limit=400,
                epsabs=1e-13, epsrel=1e-13)
    return v / (2 * np.pi)


@pytest.mark.parametrize("h", [1.0, 0.5])
@pytest.mark.parametrize("z", [0.75, 1.0, 2.0, 3.0])
def test_uniform_field_lambda0_solid_angle_plus_lattice(oracle_lib, z, h):
    """P1: uniform B0 at lambda = 0 -> solid angle / 2 pi of the square plus the lattice term."""
    a = 300 if h == 1.0 else 200
    bd = uniform_square(a, h)
    B, _, _ = oracle.field(bd, [[0, 0, z * h]], [[0, 0, 0]])
    expect = square_integral(z * h, (a + 0.5) * h, 0.0) + lattice_term(z * h, h, 0.0)
    assert np.all(np.abs(B[0] - expect) < 5e-8), (B[0], expect)
    # the lattice term itself is resolved (it is 8.04e-3 at z = 1 pixel)
    if z <= 1.0:
        cont = square_integral(z * h, (a + 0.5) * h, 0.0)
        assert abs((B[0, 0] - cont) / lattice_term(z * h, h, 0.0) - 1) < 1e-5


@pytest.mark.parametrize("z", [1.0, 2.0, 3.0])
def test_uniform_field_lambda_closed_form(oracle_lib, z):
    """P2: uniform B0 at lambda != 0.  Per component (its own lambda) the pixel sum minus the
    lattice term, extrapolated h -> 0 over the same square (h and h/3), equals the closed form."""
    lams = [0.05, 0.3, 0.0]
    A = 40.5
    S = []
    for a, h in [(40, 1.0), (121, 1.0 / 3.0)]:
        B, _, _ = oracle.field(uniform_square(a, h), [[0, 0, z]], [lams])
        S.append(B[0] - np.array([lattice_term(z, h, l) for l in lams]))
    C = (9 * S[1] - S[0]) / 8
    for p, lam in enumerate(lams):
        exact = square_integral(z, A, lam)
        assert abs(C[p] - exact) < 1e-7, (p, lam, C[p], exact)
        assert abs(S[0][p] - exact) > 10 * abs(C[p] - exact) or lam == 0.0 or lam == 0.05


def _bipole():
    d = 6.0
    return [(np.array([-5.0, 2.0, -d]), 1.0), (np.array([6.0, -3.0, -d]), -1.0)]


def _potential(P, src):
    P = np.atleast_2d(np.asarray(P, np.float64))
    B = np.zeros_like(P)
    G = np.zeros((len(P), 3, 3))
    for s, q in src:
        D = P - s
        r = np.linalg.norm(D, axis=1)
        B += q * D / r[:, None] ** 3
        G += q * (np.eye(3)[None] / r[:, None, None] ** 3
                  - 3 * D[:, :, None] * D[:, None, :] / r[:, None, None] ** 5)
    return B, G


@pytest.fixture(scope="module")
def bipole_boundary():
    a = 300
    n = 2 * a + 1
    j, i = np.mgrid[0:n, 0:n].astype(np.float64)
    P0 = np.stack([(i - a).ravel(), (j - a).ravel(), np.zeros(n * n)], 1)
    B0, _ = _potential(P0, _bipole())
    g = oracle.Grid(n, n, x0=-a, y0=-a)
    return oracle.Boundary(g, *(B0[:, c].reshape(n, n) for c in range(3)))


def test_submerged_bipole_reproduced_at_lambda0(oracle_lib, bipole_boundary):
    """P5: every component of a submerged potential field is harmonic and decays, so the
    lambda = 0 quadrature returns it, with its gradient, up to truncation and FP32 input rounding."""
    pts = np.array([[0, 0, 3.0], [4, -2, 4.0], [-7, 5, 6.0], [-3.5, 1.25, 3.0], [2.25, -6.5, 8.0]])
    B, G, _ = oracle.field(bipole_boundary, pts, np.zeros_like(pts))
    Bt, Gt = _potential(pts, _bipole())
    rel_B = np.linalg.norm(B - Bt, axis=1) / np.linalg.norm(Bt, axis=1)
    rel_G = np.linalg.norm((G - Gt).reshape(len(pts), -1), axis=1) / np.linalg.norm(
        Gt.reshape(len(pts), -1), axis=1)
    assert rel_B.max() < 1e-6, rel_B
    assert rel_G.max() < 3e-6, rel_G
    # J = curl B = 0 and div B = 0 for a potential field: f is degenerate, g tiny
    f, g, phi, J, D = oracle.objective(B, G, g_scale=1 / 6)
    assert np.all(np.linalg.norm(J, axis=1) < 3e-6 * np.linalg.norm(Gt.reshape(len(pts), -1), axis=1))
    assert np.all(g < 1e-5)


def _random_boundary(seed, nx=17, ny=13, x0=-8.0, y0=-6.0, h=1.0):
    rng = np.random.default_rng(seed)
    g = oracle.Grid(nx, ny, x0=x0, y0=y0, hx=h, hy=h)
    return oracle.Boundary(g, *(rng.normal(0, 100, (ny, nx)).astype(np.float32) for _ in range(3)))


def test_spatial_and_lambda_derivatives_match_central_differences(oracle_lib):
    """Eq. 13 at fixed lambda: analytic dB/dx_j and dB/dlambda equal central differences of B."""
    bd = _random_boundary(1)
    pts = np.array([[0.3, -0.7, 1.5], [2.0, 1.0, 4.0], [-3.1, 2.2, 0.9]])
    lam = np.array([[0.11, -0.23, 0.37], [0.0, 0.5, 0.05], [0.8, 0.01, -0.2]])
    B, G, dl = oracle.field(bd, pts, lam)
    d = 1e-4
    for j in range(3):
        e = np.zeros(3); e[j] = d
        Bp, _, _ = oracle.field(bd, pts + e, lam)
        Bm, _, _ = oracle.field(bd, pts - e, lam)
        fd = (Bp - Bm) / (2 * d)
        scale = np.abs(G).max(axis=(1, 2))[:, None]
        assert np.all(np.abs(fd - G[:, :, j]) < 1e-6 * scale), (j, fd, G[:, :, j])
    Bp, _, _ = oracle.field(bd, pts, lam + d)
    Bm, _, _ = oracle.field(bd, pts, lam - d)
    fd = (Bp - Bm) / (2 * d)
    assert np.allclose(fd, dl, rtol=1e-6, atol=1e-6 * np.abs(dl).max())


def test_forward_difference_mode_is_first_order(oracle_lib):
    """The literal first-order difference of Sect. 2.1 (step delta) agrees with the analytic
    derivative to O(delta)."""
    bd = _random_boundary(2)
    pts = np.array([[0.5, 0.5, 2.0], [1.0, -2.0, 3.0]])
    lam = np.array([[0.1, 0.2, 0.3], [0.05, 0.0, 0.4]])
    _, G, _ = oracle.field(bd, pts, lam)
    errs = []
    for delta in (1e-2, 1e-3):
        _, Gf, _ = oracle.field(bd, pts, lam, deriv=1, fd_delta=delta)
        errs.append(np.abs(Gf - G).max())
    assert errs[1] < errs[0] / 5 and errs[1] < 1e-2 * np.abs(G).max()


def test_adjoint_identity_and_linearity(oracle_lib):
    """Transpose of Eq. 16: <gB, A B0> = <A^T gB, B0>, from two independent loops, and a column of
    A from a one-pixel difference (B is linear in B0)."""
    bd = _random_boundary(3)
    rng = np.random.default_rng(7)
    n = 9
    pts = np.stack([rng.uniform(-8, 8, n), rng.uniform(-6, 6, n), rng.uniform(0.5, 6, n)], 1)
    lam = rng.uniform(-0.5, 0.5, (n, 3))
    gB = rng.normal(0, 1, (n, 3))
    B, _, _ = oracle.field(bd, pts, lam)
    gB0 = oracle.vjp(bd, pts, lam, gB)
    B0 = np.stack([c.astype(np.float64) for c in bd.B], axis=-1)
    lhs = np.sum(gB * B)
    rhs = np.sum(gB0 * B0)
    assert abs(lhs - rhs) < 1e-12 * (np.abs(gB).sum() * np.abs(B).max() + 1)
    # column check: unit pixel perturbation of component p at pixel (jj, ii)
    jj, ii, p = 5, 7, 1
    comps = [c.copy() for c in bd.B]
    comps[p][jj, ii] += 1.0
    bd2 = oracle.Boundary(bd.grid, *comps)
    B2, _, _ = oracle.field(bd2, pts, lam)
    col = B2[:, p] - B[:, p]
    assert np.allclose(np.sum(gB[:, p] * col), gB0[jj, ii, p], rtol=1e-8, atol=1e-10)


def test_invariances(oracle_lib):
    """Evenness in lambda, linearity in B0, joint translation, and the x -> -x mirror."""
    bd = _random_boundary(4)
    pts = np.array([[0.25, 1.5, 2.0], [-4.0, 3.0, 1.0], [6.0, -5.0, 7.5]])
    lam = np.array([[0.2, -0.4, 0.1], [0.0, 0.3, -0.3], [0.15, 0.15, 0.6]])
    B, G, _ = oracle.field(bd, pts, lam)
    Bn, _, _ = oracle.field(bd, pts, -lam)
    assert np.array_equal(B, Bn)
    bd2 = oracle.Boundary(bd.grid, *(2 * c for c in bd.B))
    B2, _, _ = oracle.field(bd2, pts, lam)
    assert np.array_equal(B2, 2 * B)
    g = bd.grid
    gt = oracle.Grid(g.nx, g.ny, x0=g.x0 + 16.0, y0=g.y0 - 8.0)
    Bt, _, _ = oracle.field(oracle.Boundary(gt, *bd.B), pts + [16.0, -8.0, 0.0], lam)
    assert np.allclose(Bt, B, rtol=1e-13, atol=1e-11)
    # mirror about x = 0: the grid -8..8 maps onto itself with i -> nx-1-i, Bx -> -Bx
    bm = oracle.Boundary(g, -bd.B[0][:, ::-1], bd.B[1][:, ::-1], bd.B[2][:, ::-1])
    pm = pts * [-1, 1, 1]
    Bm, Gm, _ = oracle.field(bm, pm, lam)
    assert np.allclose(Bm, B * [-1, 1, 1], rtol=1e-12, atol=1e-10)
    # d/dx flips sign on By, Bz and stays on Bx; d/dy, d/dz flip on Bx only
    sgn = np.array([[1, -1, -1], [-1, 1, 1], [-1, 1, 1]])
    assert np.allclose(Gm, G * sgn, rtol=1e-11, atol=1e-9)


def test_objective_special_cases(oracle_lib):
    """Eq. 8, 9, 14 on hand-built gradients: J parallel / perpendicular / at 30 deg to B,
    a symmetric gradient (J = 0) and a divergence of known size."""
    B = np.array([[2.0, 0.0, 0.0]] * 4)
    G = np.zeros((4, 3, 3))
    G[0, 2, 1] = 1.0   # dBz/dy = 1 -> J = (1, 0, 0), parallel to B
    G[1, 1, 0] = 1.0   # dBy/dx = 1 -> J = (0, 0, 1), perpendicular
    G[2, 2, 1] = np.cos(np.pi / 6); G[2, 1, 0] = np.sin(np.pi / 6)   # J at 30 degrees
    G[3] = np.diag([1.0, 2.0, 3.0])  # symmetric: no current, div = 6
    f, g, phi, J, D = oracle.objective(B, G, g_scale=1.0 / 6.0, w_g=2.0)
    assert np.allclose(J[0], [1, 0, 0]) and np.allclose(J[1], [0, 0, 1])
    assert np.allclose(f, [0.0, 1.0, 0.5, 0.0], atol=1e-15)
    assert np.allclose(D, [0, 0, 0, 6.0]) and np.allclose(g, [0, 0, 0, 0.5])
    assert np.allclose(phi, f + 2.0 * g)


@pytest.mark.parametrize("n,Phi", [(1, np.pi / 4), (3, 4 * np.pi / 5)])
def test_lowlou_field_satisfies_force_free_conditions(oracle_lib, n, Phi):
    """The generator's Low & Lou field gives f ~ 0, g ~ 0 through the oracle's Eq. 8/9 when its
    gradient is taken by central differences (checks the test field and the objective together);
    n = 1 is the workloads' case, n = 3, Phi = 4 pi / 5 the case of the paper's Table 1."""
    from synth import LowLou
    ll = LowLou(n, 1, 0.3, Phi)
    P = np.array([[0.1, -0.2, 0.3], [-0.4, 0.5, 0.2], [0.3, 0.3, 0.6]])
    h = 1e-5
    G = np.zeros((len(P), 3, 3))
    for j in range(3):
        e = np.zeros(3); e[j] = h
        G[:, :, j] = (ll.field(*(P + e).T) - ll.field(*(P - e).T)) / (2 * h)
    B = ll.field(*P.T)
    f, g, _, J, _ = oracle.objective(B, G, g_scale=1e-2)
    assert np.all(f < 1e-7) and np.all(g < 1e-7)
    alpha = ll.alpha(*P.T)
    assert np.allclose(J, alpha[:, None] * B, rtol=1e-6, atol=1e-6 * np.abs(B).max())


TESTFUNS = {
    "quadratic": (lambda x: float(np.sum((x - [0.3, -0.2, 0.7]) ** 2 * [1.0, 3.0, 0.5]) + 0.1), 3),
    "rosen3": (lambda x: float(sum(100 * (x[1:] - x[:-1] ** 2) ** 2 + (1 - x[:-1]) ** 2)), 3),
    "bumpy1d": (lambda x: float(np.cos(3 * x[0]) + 0.1 * x[0] ** 2), 1),
}


@pytest.mark.parametrize("name", sorted(TESTFUNS))
@pytest.mark.parametrize("tol,max_iter", [(1e-6, 50), (1e-10, 400)])
def test_nelder_mead_matches_scipy(oracle_lib, name, tol, max_iter):
    """The oracle's simplex steps are the standard ones: run from the same initial simplex with
    only the value-spread test active, scipy's Nelder-Mead takes identical steps."""
    from scipy.optimize import minimize
    fun, n = TESTFUNS[name]
    x0 = np.array([0.0, 0.0, 0.0])[:n]
    step = 0.25
    sim0 = np.array([x0 + (step if v else 0.0) * (np.arange(n) == v - 1) for v in range(n + 1)])
    ours = oracle.nelder_mead(lambda x: (fun(x), 0), sim0, tol, max_iter)
    ref = minimize(fun, x0, method="Nelder-Mead",
                   options=dict(initial_simplex=sim0, xatol=np.inf, fatol=tol,
                                maxiter=max_iter + 1, maxfev=10 ** 9))
    assert ours["nfev"] == ref.nfev
    assert ours["iters"] == ref.nit - 1
    assert np.array_equal(ours["x"], ref.x)
    assert ours["fx"] == ref.fun
    assert ours["status"] == (0 if ref.status == 0 else 1)


def test_nelder_mead_stops_on_eq12_flag(oracle_lib):
    """The Eq. 12 test (f <= eps_f and g <= eps_g at the best vertex) ends the search early."""
    fun = TESTFUNS["quadratic"][0]
    sim0 = np.array([[0, 0, 0], [0.25, 0, 0], [0, 0.25, 0], [0, 0, 0.25]], float)
    full = oracle.nelder_mead(lambda x: (fun(x), 0), sim0, 1e-12, 300)
    early = oracle.nelder_mead(lambda x: (fun(x), fun(x) < 0.2), sim0, 1e-12, 300)
    assert early["iters"] < full["iters"] and early["fx"] < 0.2 and early["status"] == 0


def test_solve_improves_objective_and_reports_abs_lambda(oracle_lib):
    """Per-point solve on the small Low & Lou case: Phi at lambda* never exceeds Phi(0), lambda*
    is reported as |lambda|, and every step code is a valid simplex move."""
    from synth import workloads
    w = workloads.small_ll()
    m = w.mag
    bd = oracle.Boundary(oracle.Grid(m.nx, m.ny), m.Bx, m.By, m.Bz)
    idx = np.array([0, 137, 600, 1500, 2047])
    pts = w.points[idx].astype(np.float64)
    opt = oracle.Options()
    res = oracle.solve(bd, pts, opt)
    B0, G0, _ = oracle.field(bd, pts, np.zeros_like(pts))
    _, _, phi0, _, _ = oracle.objective(B0, G0, g_scale=1 / 6)
    assert np.all(res["phi"] <= phi0 + 1e-15)
    assert np.all(res["lam"] >= 0)
    assert all(set(c) <= set("REOIS") for c in res["codes"])
    assert np.all((res["status"] == 0) | (res["iters"] == opt.max_iter))


def test_lambda_gradient_of_objective_matches_central_differences(oracle_lib):
    """dPhi/dlambda (chain rule through B, its gradient, J and div B) equals central differences
    of the oracle's own Phi, and the second derivatives d^2B/(dx dlambda) equal differences of G."""
    bd = _random_boundary(11)
    pts = np.array([[0.3, -0.7, 1.5], [2.0, 1.0, 4.0], [-3.1, 2.2, 2.9], [4.4, -1.0, 6.0]])
    lam = np.array([[0.11, -0.23, 0.37], [0.02, 0.5, 0.05], [0.8, 0.1, -0.2], [0.3, 0.3, 0.3]])
    gs = 1.0 / 6.0
    f, g, phi, dphi = oracle.objective_grad(bd, pts, lam, gs)
    B, G, dl, dG = oracle.field_dl(bd, pts, lam)
    h = 1e-5
    for q in range(3):
        e = np.zeros(3); e[q] = h
        _, _, pp, _ = oracle.objective_grad(bd, pts, lam + e, gs)
        _, _, pm, _ = oracle.objective_grad(bd, pts, lam - e, gs)
        assert np.allclose((pp - pm) / (2 * h), dphi[:, q], rtol=1e-5, atol=1e-7), q
        _, Gp, _ = oracle.field(bd, pts, lam + e)
        _, Gm, _ = oracle.field(bd, pts, lam - e)
        fd = (Gp - Gm)[:, q, :] / (2 * h)
        assert np.allclose(fd, dG[:, q, :], rtol=1e-6, atol=1e-8 * np.abs(dG).max()), q


@pytest.mark.parametrize("name", ["quadratic", "rosen3"])
def test_bfgs_reaches_minimum_and_decreases(oracle_lib, name):
    """The oracle's quasi-Newton search: monotone decrease (Armijo) and the known minimum of a
    convex quadratic (exactly) and of Rosenbrock's function (to tolerance)."""
    A = np.array([1.0, 3.0, 0.5])
    c = np.array([0.3, -0.2, 0.7])
    vals = []

    def quad(x):
        vals.append(float(np.sum(A * (x - c) ** 2) + 0.1))
        return vals[-1], 2 * A * (x - c), 0

    def rosen(x):
        v = float(sum(100 * (x[1:] - x[:-1] ** 2) ** 2 + (1 - x[:-1]) ** 2))
        gr = np.zeros(3)
        gr[:-1] += -400 * x[:-1] * (x[1:] - x[:-1] ** 2) - 2 * (1 - x[:-1])
        gr[1:] += 200 * (x[1:] - x[:-1] ** 2)
        vals.append(v)
        return v, gr, 0

    fun = quad if name == "quadratic" else rosen
    r = oracle.bfgs(fun, np.zeros(3), step=0.25, tol=1e-14, max_iter=500)
    target = c if name == "quadratic" else np.ones(3)
    assert np.allclose(r["x"], target, atol=1e-5), r
    assert r["status"] == 0 and r["nfev"] == len(vals)


def test_bfgs_solve_improves_on_start(oracle_lib):
    """method = 1 on points of the small Low & Lou case: Phi never above Phi at the start."""
    from synth import workloads
    w = workloads.small_ll()
    m = w.mag
    bd = oracle.Boundary(oracle.Grid(m.nx, m.ny), m.Bx, m.By, m.Bz)
    pts = w.points[[3, 400, 1200]].astype(np.float64)
    r = oracle.solve(bd, pts, oracle.Options(method=1, max_iter=20))
    s = 1.0 / 32.0   # the search starts at lambda = s (1, 1, 1), off the stationary point 0
    _, _, phi0, grad0 = oracle.objective_grad(bd, pts, np.full((3, 3), s), 1.0 / 6.0)
    assert np.all(np.abs(grad0) > 0)
    assert np.all(r["phi"] <= phi0 + 1e-15) and np.all(r["nfev"] > 3)
