"""Pins of the oracle's pixel-exact near field (exact integration of the lambda = 0 kernel over
each pixel, the remainder on the midpoint rule of Eq. 16) against facts the mathematics fixes:
scipy's 2-D integrals of z / (2 pi r^3) over rectangles, the closed-form solid angle of a square
for a point above its centre and the polar form of the lambda != 0 integral, per-pixel scipy
integrals for piecewise-constant data, central differences for the derivatives, the adjoint
identity and differences through the lambda search."""
import numpy as np
import pytest
from scipy import integrate

import oracle
from test_oracle_pins import square_integral, uniform_square
from gates import oracle_boundary
from synth.workloads import lowlou_magnetogram

TWO_PI = 2 * np.pi


def k0(y, x, z):
    return z / (TWO_PI * (x * x + y * y + z * z) ** 1.5)


def rect_quad(xa, xb, ya, yb, z):
    v, _ = integrate.dblquad(k0, xa, xb, ya, yb, args=(z,), epsabs=1e-13, epsrel=1e-12)
    return v


@pytest.mark.parametrize("rect,z", [((-0.5, 0.5, -0.5, 0.5), 0.5), ((0.5, 1.5, -0.5, 0.5), 1.0),
                                    ((-3.5, -2.5, 1.5, 2.5), 0.75), ((-0.2, 0.7, -1.1, 0.3), 2.0),
                                    ((2.0, 5.0, 3.0, 4.0), 0.3)])
def test_rect_integral_is_scipys(rect, z):
    """orc_rect_exact's value is scipy's 2-D integral; its derivatives with respect to the point
    are central differences of scipy's integral (the rectangle is fixed, the point moves)."""
    xa, xb, ya, yb = rect
    out = oracle.rect_exact(xa, xb, ya, yb, z)
    assert abs(out[0] - rect_quad(xa, xb, ya, yb, z)) < 1e-11
    d = 1e-4
    fd = [(rect_quad(xa - d, xb - d, ya, yb, z) - rect_quad(xa + d, xb + d, ya, yb, z)) / (2 * d),
          (rect_quad(xa, xb, ya - d, yb - d, z) - rect_quad(xa, xb, ya + d, yb + d, z)) / (2 * d),
          (rect_quad(xa, xb, ya, yb, z + d) - rect_quad(xa, xb, ya, yb, z - d)) / (2 * d)]
    assert np.abs(out[1:] - fd).max() < 1e-7 * max(1.0, np.abs(fd).max()), (out[1:], fd)


def test_rect_integral_limits():
    """The whole plane carries weight 1 (solid angle 2 pi) and a quadrant 1/4, whatever z."""
    for z in (0.1, 1.0, 7.0):
        assert abs(oracle.rect_exact(-1e9, 1e9, -1e9, 1e9, z)[0] - 1.0) < 1e-8
        assert abs(oracle.rect_exact(0.0, 1e9, 0.0, 1e9, z)[0] - 0.25) < 1e-8


@pytest.mark.parametrize("z", [0.5, 1.0, 2.0])
def test_uniform_field_is_the_solid_angle(z):
    """Uniform B0 on (2a+1)^2 unit pixels, point above the centre, lambda = 0: the pixel-exact
    rule is the solid angle of the pixels' square [-a-1/2, a+1/2]^2 over 2 pi (closed form), with
    no lattice term (the midpoint rule is 8e-3 off at z = 1, 0.24 at z = 0.5)."""
    a = 40
    bd = uniform_square(a, 1.0)
    exact = square_integral(z, a + 0.5, 0.0)
    B, _, _ = oracle.field(bd, [[0, 0, z]], [[0, 0, 0]], quad_order=-1)
    assert np.abs(B[0] - exact).max() < 1e-12, B[0] - exact
    mid, _, _ = oracle.field(bd, [[0, 0, z]], [[0, 0, 0]])
    assert abs(mid[0, 0] - exact) > 1e-5


@pytest.mark.parametrize("z,lam,band", [(0.5, 0.1, 0.1), (0.5, 0.3, 0.1), (1.0, 0.2, 0.3)])
def test_uniform_field_lambda_keeps_only_the_remainder_lattice_term(z, lam, band):
    """lambda != 0: the exact integral over the square is the angular mean of
    cos(lam z) - z cos(lam R') / R' (polar antiderivative).  The pixel-exact rule leaves only the
    midpoint error of the remainder kernel z [u - 1] / (2 pi r^3) ~ lam^2 z / (4 pi r).  By
    Poisson summation (the 2-D transform of z / r is 2 pi z exp(-k z) / k) its lattice part is
    about lam^2 z / 2 sum_{m != 0} exp(-2 pi |m| z) / (2 pi |m|); the rest is the truncated
    square's edge term of the slowly decaying remainder (a few 1e-6 here)."""
    a = 80
    bd = uniform_square(a, 1.0)
    exact = square_integral(z, a + 0.5, lam)
    B, _, _ = oracle.field(bd, [[0, 0, z]], [[lam] * 3], quad_order=-1)
    mid, _, _ = oracle.field(bd, [[0, 0, z]], [[lam] * 3])
    err, err_mid = B[0, 0] - exact, abs(mid[0, 0] - exact)
    m = np.array([(i, j) for i in range(-12, 13) for j in range(-12, 13) if i or j], float)
    km = TWO_PI * np.hypot(m[:, 0], m[:, 1])
    est = lam * lam * z / 2 * np.sum(np.exp(-km * z) / km)
    assert abs(err - est) < band * est and abs(err) < 0.01 * err_mid, (err, est, err_mid)


def test_uniform_field_off_centre_is_scipys():
    """A point off the pixel centres and off the square's centre: scipy's integral of K0 over the
    whole pixel rectangle."""
    a = 10
    bd = uniform_square(a, 1.0)
    for P in ([0.3, -0.2, 0.5], [2.5, 1.5, 1.0], [-4.1, 6.6, 1.7]):
        B, _, _ = oracle.field(bd, [P], [[0, 0, 0]], quad_order=-1)
        ex = rect_quad(-a - 0.5 - P[0], a + 0.5 - P[0], -a - 0.5 - P[1], a + 0.5 - P[1], P[2])
        assert np.abs(B[0] - ex).max() < 1e-10, (B[0] - ex)


def _piecewise_boundary(nx, ny, seed, hx=1.0, hy=1.0):
    rng = np.random.default_rng(seed)
    g = oracle.Grid(nx, ny, x0=-(nx - 1) / 2 * hx, y0=-(ny - 1) / 2 * hy, hx=hx, hy=hy)
    comps = [(rng.integers(-64, 65, (ny, nx)) / 16.0).astype(np.float32) for _ in range(3)]
    return oracle.Boundary(g, *comps), comps


@pytest.mark.parametrize("hx,hy", [(1.0, 1.0), (0.5, 0.75)])
def test_piecewise_constant_data_is_scipys_pixel_integrals(hx, hy):
    """Random data constant on each pixel, lambda = 0: sum over pixels of the value times scipy's
    integral of K0 over the pixel rectangle; also with non-square pixels."""
    nx, ny = 8, 7
    bd, comps = _piecewise_boundary(nx, ny, 3, hx, hy)
    g = bd.grid
    for P in ([0.0, 0.0, 0.5 * hx], [0.4 * hx, -0.9 * hy, 1.1 * hx]):
        W = np.zeros((ny, nx))
        for j in range(ny):
            for i in range(nx):
                xc, yc = g.x0 + i * hx, g.y0 + j * hy
                W[j, i] = rect_quad(xc - hx / 2 - P[0], xc + hx / 2 - P[0], yc - hy / 2 - P[1],
                                    yc + hy / 2 - P[1], P[2])
        ref = np.array([np.sum(W * c.astype(np.float64)) for c in comps])
        B, _, _ = oracle.field(bd, [P], [[0, 0, 0]], quad_order=-1, pxe_near_z=10.0)
        assert np.abs(B[0] - ref).max() < 1e-10 * max(1.0, np.abs(ref).max()), (B[0] - ref)


def test_gradient_is_the_derivative_of_the_field():
    """G of the pixel-exact rule (midpoint part and correction) against central differences of
    its B in the point position, at lambda = 0 and lambda != 0."""
    bd, _ = _piecewise_boundary(12, 11, 4)
    d = 1e-4
    for P, lam in (([0.2, -0.3, 0.8], 0.0), ([1.0, 2.0, 1.5], 0.15), ([-2.4, 0.5, 0.6], 0.3)):
        L = [[lam, 0.5 * lam, 2 * lam]]
        _, G, _ = oracle.field(bd, [P], L, quad_order=-1, pxe_near_z=5.0)
        fd = np.zeros((3, 3))
        for j in range(3):
            e = np.zeros(3)
            e[j] = d
            Bp, _, _ = oracle.field(bd, [np.add(P, e)], L, quad_order=-1, pxe_near_z=5.0)
            Bm, _, _ = oracle.field(bd, [np.subtract(P, e)], L, quad_order=-1, pxe_near_z=5.0)
            fd[:, j] = (Bp[0] - Bm[0]) / (2 * d)
        assert np.abs(G[0] - fd).max() < 2e-6 * np.abs(fd).max(), (G[0] - fd)


def test_correction_is_lambda_independent_and_switched_by_near_z():
    """The correction does not depend on lambda (pxe(lam) - pxe(0) = midpoint(lam) - midpoint(0)),
    and points above near_z take the midpoint rule unchanged."""
    bd, _ = _piecewise_boundary(10, 10, 5)
    P = np.array([[0.1, 0.2, 0.7], [1.0, -1.0, 1.9], [0.0, 0.0, 2.5]])
    lam = np.array([[0.2, 0.1, 0.3]] * 3)
    Bx, Gx, _ = oracle.field(bd, P, lam, quad_order=-1)
    B0x, G0x, _ = oracle.field(bd, P, 0 * lam, quad_order=-1)
    Bm, Gm, _ = oracle.field(bd, P, lam)
    B0m, G0m, _ = oracle.field(bd, P, 0 * lam)
    assert np.allclose(Bx - B0x, Bm - B0m, rtol=0, atol=1e-13)
    assert np.allclose(Gx - G0x, Gm - G0m, rtol=0, atol=1e-12)
    assert np.all(Bx[2] == Bm[2]) and np.all(Gx[2] == Gm[2])           # z = 2.5 > 2 hx
    assert np.abs(Bx[:2] - Bm[:2]).max() > 1e-3                          # z <= 2 hx corrected
    dB, dG = oracle.pxe_correction(bd, P[0])
    assert np.allclose(Bx[0], Bm[0] + dB, rtol=0, atol=1e-14)


def test_adjoint_identity():
    """<gB, B(B0)> = <A^T gB, B0> for the pixel-exact rule (B is linear in B0), with points on
    both sides of near_z."""
    bd, comps = _piecewise_boundary(9, 8, 6)
    rng = np.random.default_rng(6)
    P = np.stack([rng.uniform(-3, 3, 10), rng.uniform(-3, 3, 10), rng.uniform(0.4, 3.0, 10)], 1)
    lam = rng.uniform(0.0, 0.3, (10, 3))
    gB = rng.normal(size=(10, 3))
    B, _, _ = oracle.field(bd, P, lam, quad_order=-1)
    gB0 = oracle.vjp(bd, P, lam, gB, quad_order=-1)
    lhs = np.sum(gB * B)
    rhs = sum(np.sum(gB0[:, :, p] * comps[p].astype(np.float64)) for p in range(3))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))
    assert np.abs(gB0 - oracle.vjp(bd, P, lam, gB)).max() > 1e-3


def test_hessian_and_gradient_carry_the_correction():
    """Phi and dPhi/dlambda of the hyper-dual pass equal those of the first-order pass with the
    same correction; the Hessian is the central difference of that gradient; and the correction
    changes Phi at points with z <= near_z."""
    mag = lowlou_magnetogram(12)
    bd = oracle_boundary(mag)
    gs = mag.hx / 6.0
    rng = np.random.default_rng(9)
    pts = np.stack([rng.uniform(3, 8, 6), rng.uniform(3, 8, 6), rng.uniform(0.5, 2.0, 6)], 1)
    lam = rng.uniform(0.5, 3.0, (6, 3)) / 12.0
    nz = 2.0 * mag.hx
    phi, grad, H, _ = oracle.hessian(bd, pts, lam, gs, pxe_near_z=nz)
    _, _, p1, g1 = oracle.objective_grad(bd, pts, lam, gs, pxe_near_z=nz)
    assert np.allclose(phi, p1, rtol=1e-12, atol=0) and np.allclose(grad, g1, rtol=1e-9, atol=1e-12)
    p0, _, _, _ = oracle.hessian(bd, pts, lam, gs)
    assert np.abs(phi - p0).max() > 1e-4
    d = 1e-6
    for q in range(3):
        e = np.zeros(3)
        e[q] = d
        gp = oracle.objective_grad(bd, pts, lam + e, gs, pxe_near_z=nz)[3]
        gm = oracle.objective_grad(bd, pts, lam - e, gs, pxe_near_z=nz)[3]
        fd = (gp - gm) / (2 * d)
        assert np.abs(H[:, :, q] - fd).max() < 1e-5 * np.abs(H).max()


def test_implicit_vjp_through_the_search():
    """gB0 through the search with the correction against central differences of
    L(B0) = sum gB . B(lambda*(B0), B0), lambda* re-found by Newton on the corrected objective
    after each perturbation (B0 +- 2^-6 is exact in float32)."""
    mag = lowlou_magnetogram(12)
    bd = oracle_boundary(mag)
    gs = mag.hx / 6.0
    nz = 2.0 * mag.hx
    rng = np.random.default_rng(11)
    pts = np.stack([rng.uniform(3, 8, 40), rng.uniform(3, 8, 40), rng.uniform(0.6, 2.0, 40)], 1)
    r = oracle.solve(bd, pts, oracle.Options(method=1, max_iter=60, tol=1e-14, quad_order=-1))

    def newton(b, lam):
        lam = lam.copy()
        for _ in range(40):
            _, gr, Hh, _ = oracle.hessian(b, pts_g, lam, gs, pxe_near_z=nz)
            st = np.linalg.solve(Hh, gr[:, :, None])[:, :, 0]
            lam -= st
            if np.abs(st).max() < 1e-15:
                break
        return lam

    pts_g = pts
    lam = newton(bd, r["lam"])
    _, gr, H, _ = oracle.hessian(bd, pts, lam, gs, pxe_near_z=nz)
    ev = np.linalg.eigvalsh(H)
    good = (np.abs(gr).max(1) < 1e-12) & (ev[:, 0] > 0) & (ev[:, -1] < 1e4 * ev[:, 0])
    assert good.sum() >= 4, good.sum()
    pts_g = pts[good][:4]
    lamP = lam[good][:4]
    gB = rng.normal(size=(len(pts_g), 3))
    gB0, v, flags = oracle.implicit_vjp(bd, pts_g, lamP, gB, gs, pxe_near_z=nz)
    assert not flags.any()

    def L(Bc):
        b2 = oracle.Boundary(bd.grid, *Bc)
        lm = newton(b2, lamP)
        return np.sum(gB * oracle.field(b2, pts_g, lm, quad_order=-1, pxe_near_z=nz)[0])

    dd = 2.0 ** -6
    for _ in range(4):
        j, i, p = rng.integers(0, 12), rng.integers(0, 12), rng.integers(0, 3)
        Bp = [b.copy() for b in bd.B]
        Bm = [b.copy() for b in bd.B]
        Bp[p][j, i] += dd
        Bm[p][j, i] -= dd
        fd = (L(Bp) - L(Bm)) / (2 * dd)
        assert abs(gB0[j, i, p] - fd) <= 1e-6 * abs(fd) + 1e-12, (gB0[j, i, p], fd)


def test_solve_reports_the_corrected_field():
    """The simplex search with the pixel-exact rule reports B = the corrected field at its
    lambda, and its Phi there."""
    mag = lowlou_magnetogram(12)
    bd = oracle_boundary(mag)
    gs = mag.hx / 6.0
    rng = np.random.default_rng(12)
    pts = np.stack([rng.uniform(2, 9, 8), rng.uniform(2, 9, 8), rng.uniform(0.5, 2.0, 8)], 1)
    r = oracle.solve(bd, pts, oracle.Options(quad_order=-1))
    B, G, _ = oracle.field(bd, pts, r["lam"], quad_order=-1)
    assert np.allclose(r["B"], B, rtol=1e-13, atol=1e-15)
    f, g, phi, _, _ = oracle.objective(B, G, gs)
    assert np.allclose(r["phi"], phi, rtol=1e-12, atol=1e-15)
