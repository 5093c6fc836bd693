"""Pins of the oracle's nine-node element quadrature (Eq. 15) against facts the mathematics fixes:
numpy's Gauss-Legendre rule, closed-form kernel integrals over the elements' square (at lambda = 0
and lambda != 0; no lattice term, unlike the midpoint rule), scipy's 2-D integral of the kernel
times biquadratic data (which the nine-node interpolation reproduces exactly), finite differences
for the derivatives, and the adjoint identity."""
import numpy as np
import pytest
from scipy import integrate

import oracle
from test_oracle_pins import square_integral, uniform_square


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6, 8, 12])
def test_gauss_legendre_is_numpys(m):
    x, w = oracle.gauss_legendre(m)
    X, W = np.polynomial.legendre.leggauss(m)
    assert np.abs(x - X).max() < 1e-14 and np.abs(w - W).max() < 1e-14


@pytest.mark.parametrize("z,lam,order,tol", [(2.0, 0.0, 8, 1e-9), (1.0, 0.0, 8, 1e-6),
                                             (3.0, 0.0, 4, 1e-6), (2.0, 0.3, 8, 1e-9),
                                             (3.0, 0.05, 6, 1e-9)])
def test_uniform_field_is_the_exact_integral(z, lam, order, tol):
    """Uniform B0 on (2a+1)^2 nodes: the element rule integrates the kernel over the node square
    [-a, a]^2 (no lattice term): solid angle / 2 pi at lambda = 0, the angular mean of
    cos(lam z) - z cos(lam R')/R' otherwise; the error falls with the Gauss order."""
    a = 40
    bd = uniform_square(a, 1.0)
    B, _, _ = oracle.field(bd, [[0, 0, z]], [[lam, lam, lam]], quad_order=order)
    exact = square_integral(z, float(a), lam)
    assert np.all(np.abs(B[0] - exact) < tol), (B[0] - exact)
    lo, _, _ = oracle.field(bd, [[0, 0, z]], [[lam, lam, lam]], quad_order=2)
    assert abs(lo[0, 0] - exact) > abs(B[0, 0] - exact)
    if lam == 0.0 and z == 1.0:
        # the midpoint rule's lattice term at z = 1 pixel is 8e-3; the elements remove it
        mid, _, _ = oracle.field(bd, [[0, 0, z]], [[0, 0, 0]])
        assert abs(mid[0, 0] - square_integral(z, a + 0.5, 0.0)) > 5e-3


def test_biquadratic_data_is_integrated_exactly():
    """B0 = q(x, y) biquadratic within every element (q = 1 + x/4 - y/8 + x^2 y / 64) is
    reproduced exactly by the nine-node shape functions, so the element rule equals the 2-D
    integral of K q over the node rectangle (scipy) up to the Gauss rule's error."""
    nx, ny = 21, 17
    g = oracle.Grid(nx, ny, x0=-7.0, y0=-5.0)
    j, i = np.mgrid[0:ny, 0:nx].astype(np.float64)
    x, y = g.x0 + i, g.y0 + j

    def q(x, y):
        return 1 + x / 4 - y / 8 + x * x * y / 64

    vals = q(x, y).astype(np.float32)
    assert np.all(vals.astype(np.float64) == q(x, y))     # exact in float32 at the nodes
    bd = oracle.Boundary(g, vals, vals, vals)
    P = np.array([1.3, 0.4, 2.5])
    for lam in (0.0, 0.2):
        B, _, _ = oracle.field(bd, [P], [[lam] * 3], quad_order=8)

        def f(yy, xx):
            dx, dy = P[0] - xx, P[1] - yy
            r = np.sqrt(dx * dx + dy * dy + P[2] ** 2)
            return P[2] * (lam * r * np.sin(lam * r) + np.cos(lam * r)) / (2 * np.pi * r ** 3) * q(xx, yy)

        x0, x1, y0, y1 = g.x0, g.x0 + nx - 1, g.y0, g.y0 + ny - 1
        ref = sum(integrate.dblquad(f, xa, xb, ya, yb, epsabs=0, epsrel=1e-12)[0]
                  for xa, xb in ((x0, P[0]), (P[0], x1)) for ya, yb in ((y0, P[1]), (P[1], y1)))
        assert abs(B[0, 0] - ref) < 1e-8 * abs(ref), (B[0, 0], ref)


def test_shape_functions_are_a_partition_of_unity_and_interpolate():
    """Node weights sum over nodes to the rule's integral of the kernel alone; a single-node
    boundary gives exactly that node's weight (the weights are the coefficients of Eq. 16)."""
    g = oracle.Grid(9, 7, x0=0.0, y0=0.0, hx=0.7, hy=1.2)
    one = np.ones((7, 9), np.float32)
    P = (2.1, 3.3, 1.7)
    w = oracle.node_weights_q9(oracle.Boundary(g, one, one, one), P, 0.25, 5)
    B, G, dl = oracle.field(oracle.Boundary(g, one, one, one), [P], [[0.25] * 3], quad_order=5)
    assert abs(w[..., 0].sum() - B[0, 0]) < 1e-14
    assert abs(w[..., 3].sum() - G[0, 0, 2]) < 1e-13 and abs(w[..., 4].sum() - dl[0, 0]) < 1e-14
    for (jj, ii) in ((0, 0), (3, 4), (6, 8), (2, 1)):
        imp = np.zeros((7, 9), np.float32)
        imp[jj, ii] = 1.0
        Bi, _, _ = oracle.field(oracle.Boundary(g, imp, imp, imp), [P], [[0.25] * 3], quad_order=5)
        assert abs(Bi[0, 0] - w[jj, ii, 0]) < 1e-15


def test_q9_derivatives_match_central_differences():
    rng = np.random.default_rng(3)
    g = oracle.Grid(15, 11, x0=-2.0, y0=1.0)
    comps = [rng.normal(0, 50, (11, 15)).astype(np.float32) for _ in range(3)]
    bd = oracle.Boundary(g, *comps)
    P = np.array([[3.3, 5.1, 1.8], [8.0, 2.0, 3.5]])
    lam = np.array([[0.1, -0.3, 0.2], [0.05, 0.15, -0.1]])
    B, G, dl = oracle.field(bd, P, lam, quad_order=4)
    h = 1e-5
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        Bp, _, _ = oracle.field(bd, P + e, lam, quad_order=4)
        Bm, _, _ = oracle.field(bd, P - e, lam, quad_order=4)
        assert np.allclose((Bp - Bm) / (2 * h), G[:, :, j], rtol=1e-6, atol=1e-7 * np.abs(G).max())
    Bp, _, _ = oracle.field(bd, P, lam + h, quad_order=4)
    Bm, _, _ = oracle.field(bd, P, lam - h, quad_order=4)
    assert np.allclose((Bp - Bm) / (2 * h), dl, rtol=1e-6, atol=1e-7 * np.abs(dl).max())


def test_q9_adjoint_identity_and_solve():
    rng = np.random.default_rng(4)
    g = oracle.Grid(13, 9)
    comps = [rng.normal(0, 30, (9, 13)).astype(np.float32) for _ in range(3)]
    bd = oracle.Boundary(g, *comps)
    P = np.stack([rng.uniform(0, 12, 7), rng.uniform(0, 8, 7), rng.uniform(0.5, 4, 7)], 1)
    lam = rng.uniform(-0.3, 0.3, (7, 3))
    gB = rng.normal(size=(7, 3))
    B, _, _ = oracle.field(bd, P, lam, quad_order=3)
    gB0 = oracle.vjp(bd, P, lam, gB, quad_order=3)
    lhs = np.sum(gB * B)
    rhs = sum(np.sum(gB0[..., p] * comps[p].astype(np.float64)) for p in range(3))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + np.abs(gB).sum())
    # the simplex runs on the element rule too and lowers Phi from its start
    r = oracle.solve(bd, P, oracle.Options(quad_order=3, max_iter=20))
    _, G0, _ = oracle.field(bd, P, np.zeros((7, 3)), quad_order=3)
    B0v, _, _ = oracle.field(bd, P, np.zeros((7, 3)), quad_order=3)
    _, _, phi0, _, _ = oracle.objective(B0v, G0, 1.0 / 6.0)
    assert np.all(r["phi"] <= phi0 + 1e-15)
