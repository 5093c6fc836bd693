"""Pins of the oracle's second-order quantities (CPU): the lambda-Hessian of Phi, the gradient of a
loss through the lambda search (implicit differentiation of the stationarity condition) and the
noise variance of B.  None is in the paper; each is pinned to something other than its own code:
the hand-written first-order chain rule, differences of it, finite differences of the whole
solve-then-evaluate pipeline, impulse responses of Eq. 16 and a library 2-D integral."""
import numpy as np
import pytest
from scipy import integrate

import oracle
from gates import oracle_boundary
from synth.workloads import lowlou_magnetogram, small_ll


@pytest.fixture(scope="module")
def ll():
    w = small_ll()
    return w, oracle_boundary(w.mag)


def test_hessian_gradient_is_the_chain_rule_gradient(ll):
    """The hyper-dual gradient equals the hand-derived chain rule of orc_objective_grad."""
    w, bd = ll
    rng = np.random.default_rng(3)
    pts = w.points[rng.choice(len(w.points), 16, replace=False)].astype(np.float64)
    lam = rng.uniform(0.5, 3.0, (16, 3)) / 32.0
    gs = w.mag.hx / 6.0
    phi, grad, H, dl = oracle.hessian(bd, pts, lam, gs)
    f, g, p2, d2 = oracle.objective_grad(bd, pts, lam, gs)
    assert np.allclose(phi, p2, rtol=1e-13, atol=1e-15)
    assert np.abs(grad - d2).max() <= 1e-12 * np.abs(d2).max()
    _, _, dBdl = oracle.field(bd, pts, lam)
    assert np.abs(dl - dBdl).max() <= 1e-12 * np.abs(dBdl).max()


def test_hessian_is_the_difference_of_the_gradient(ll):
    """Central differences of the chain-rule gradient (error O(delta^2)) reproduce H."""
    w, bd = ll
    rng = np.random.default_rng(4)
    pts = w.points[rng.choice(len(w.points), 16, replace=False)].astype(np.float64)
    lam = rng.uniform(0.5, 3.0, (16, 3)) / 32.0
    gs = w.mag.hx / 6.0
    _, _, H, _ = oracle.hessian(bd, pts, lam, gs)
    d = 1e-4 / 32.0
    Hfd = np.zeros_like(H)
    for k in range(3):
        e = np.zeros(3)
        e[k] = d
        gp = oracle.objective_grad(bd, pts, lam + e, gs)[3]
        gm = oracle.objective_grad(bd, pts, lam - e, gs)[3]
        Hfd[:, :, k] = (gp - gm) / (2 * d)
    assert np.abs(H - Hfd).max() <= 1e-7 * np.abs(H).max()
    assert np.array_equal(H, np.transpose(H, (0, 2, 1)))


def test_tied_hessian_is_the_all_ones_contraction(ll):
    """With one shared lambda, d/dt and d^2/dt^2 along (1, 1, 1) are 1.grad and 1^T H 1."""
    w, bd = ll
    rng = np.random.default_rng(5)
    pts = w.points[rng.choice(len(w.points), 12, replace=False)].astype(np.float64)
    t = rng.uniform(0.5, 3.0, 12) / 32.0
    lam = np.repeat(t[:, None], 3, axis=1)
    gs = w.mag.hx / 6.0
    _, grad, H, dl = oracle.hessian(bd, pts, lam, gs)
    _, gt, Ht, dlt = oracle.hessian(bd, pts, lam, gs, lambda_mode=1)
    assert np.allclose(gt[:, 0], grad.sum(1), rtol=1e-12, atol=1e-14 * np.abs(grad).max())
    assert np.allclose(Ht[:, 0, 0], H.sum((1, 2)), rtol=1e-11, atol=1e-13 * np.abs(H).max())
    assert np.allclose(dlt, dl, rtol=1e-13, atol=0)
    assert np.all(gt[:, 1:] == 0) and np.all(Ht.reshape(-1, 9)[:, 1:] == 0)


def _newton(bd, pts, lam, gs, mode):
    """Newton's method on grad Phi = 0 (the fixed point is the stationary point whatever the
    Hessian used; the oracle's own is used for speed)."""
    lam = lam.copy()
    for _ in range(40):
        _, gr, H, _ = oracle.hessian(bd, pts, lam, gs, lambda_mode=mode)
        if mode == 1:
            st = gr[:, 0] / H[:, 0, 0]
            lam -= st[:, None]
        else:
            st = np.linalg.solve(H, gr[:, :, None])[:, :, 0]
            lam -= st
        if np.abs(st).max() < 1e-15:
            break
    return lam


@pytest.fixture(scope="module")
def minima():
    """Stationary points of Phi with a well-conditioned positive-definite Hessian on a 12 x 12
    Low & Lou boundary, per mode: quasi-Newton search, then Newton to |grad| < 1e-12."""
    mag = lowlou_magnetogram(12)
    bd = oracle_boundary(mag)
    gs = mag.hx / 6.0
    rng = np.random.default_rng(5)
    pts = np.stack([rng.uniform(3, 8, 40), rng.uniform(3, 8, 40), rng.uniform(1, 4, 40)], 1)
    out = {}
    for mode in (0, 1):
        r = oracle.solve(bd, pts, oracle.Options(method=1, max_iter=60, tol=1e-14,
                                                   lambda_mode=mode))
        lam = _newton(bd, pts, r["lam"], gs, mode)
        _, gr, H, _ = oracle.hessian(bd, pts, lam, gs, lambda_mode=mode)
        if mode == 1:
            ev = H[:, :1, :1].reshape(-1, 1)
        else:
            ev = np.linalg.eigvalsh(H)
        good = (np.abs(gr).max(1) < 1e-12) & (ev[:, 0] > 0) & (ev[:, -1] < 1e4 * ev[:, 0])
        assert good.sum() >= 6, good.sum()
        out[mode] = (pts[good][:6], lam[good][:6])
    return bd, gs, out


@pytest.mark.parametrize("mode", [0, 1])
def test_implicit_vjp_is_the_derivative_through_the_search(minima, mode):
    """gB0 against central differences of L(B0) = sum gB . B(lambda*(B0), B0), lambda* re-found
    by Newton after each perturbation: B0 +- 2^-6 is exact in float32, the O(delta^2) term is
    ~1e-8 of the result.  The fixed-lambda adjoint differs at the 10 % level here, so a dropped
    implicit term or a wrong sign fails."""
    bd, gs, out = minima
    P, lamP = out[mode]
    rng = np.random.default_rng(7 + mode)
    gB = rng.normal(size=(len(P), 3))
    gB0, v, flags = oracle.implicit_vjp(bd, P, lamP, gB, gs, lambda_mode=mode)
    assert not flags.any()
    fixed = oracle.vjp(bd, P, lamP, gB)

    def L(Bc):
        bd2 = oracle.Boundary(bd.grid, *Bc)
        lam = _newton(bd2, P, lamP, gs, mode)
        return np.sum(gB * oracle.field(bd2, P, lam)[0])

    d = 2.0 ** -6
    rel_fixed = []
    for _ in range(5):
        j, i, p = rng.integers(0, 12), rng.integers(0, 12), rng.integers(0, 3)
        Bp = [b.copy() for b in bd.B]
        Bm = [b.copy() for b in bd.B]
        Bp[p][j, i] += d
        Bm[p][j, i] -= d
        assert Bp[p][j, i] - bd.B[p][j, i] == d and bd.B[p][j, i] - Bm[p][j, i] == d
        fd = (L(Bp) - L(Bm)) / (2 * d)
        assert abs(gB0[j, i, p] - fd) <= 1e-6 * abs(fd) + 1e-12, (gB0[j, i, p], fd)
        rel_fixed.append(abs(fixed[j, i, p] - fd) / abs(fd))
    assert max(rel_fixed) > 1e-2


def test_implicit_vjp_without_a_minimum_is_the_fixed_lambda_adjoint(ll):
    """Points whose Hessian is not positive definite are flagged and keep only the transpose of
    Eq. 16; with gB orthogonal to dB/dlambda (v = 0) the result is the fixed-lambda adjoint too."""
    w, bd = ll
    rng = np.random.default_rng(8)
    pts = w.points[rng.choice(len(w.points), 24, replace=False)].astype(np.float64)
    lam = rng.uniform(0.5, 3.0, (24, 3)) / 32.0
    gs = w.mag.hx / 6.0
    _, _, H, _ = oracle.hessian(bd, pts, lam, gs)
    bad = np.linalg.eigvalsh(H)[:, 0] < 0
    assert bad.sum() >= 4
    gB = rng.normal(size=(24, 3))
    gB0, v, flags = oracle.implicit_vjp(bd, pts[bad], lam[bad], gB[bad], gs)
    assert flags.all() and np.all(v == 0)
    ref = oracle.vjp(bd, pts[bad], lam[bad], gB[bad])
    assert np.abs(gB0 - ref).max() <= 1e-13 * np.abs(ref).max()
    # v = 0 exactly when every dL/dlambda_p = gB_p dB_p/dlambda_p vanishes: gB_p = 0 for all p
    # except where it is multiplied by dB_p/dlambda_p = 0 -- take lambda = 0 (dB/dlambda = 0)
    lam0 = np.zeros((24, 3))
    g0, v0, f0 = oracle.implicit_vjp(bd, pts, lam0, gB, gs)
    assert np.all(v0 == 0)
    ref0 = oracle.vjp(bd, pts, lam0, gB)
    assert np.abs(g0 - ref0).max() <= 1e-13 * np.abs(ref0).max()


def test_noise_variance_is_the_sum_of_squared_impulse_responses():
    """Var B_p = sum_k a_ik^2 s_pk^2 with a_ik read off orc_field for unit one-pixel boundaries."""
    nx, ny = 7, 5
    g = oracle.Grid(nx, ny, x0=-1.0, y0=0.5, hx=0.8, hy=1.1)
    rng = np.random.default_rng(9)
    sig = [rng.uniform(0.5, 2.0, (ny, nx)).astype(np.float32) for _ in range(3)]
    pts = np.stack([rng.uniform(-1, 4, 6), rng.uniform(0, 5, 6), rng.uniform(0.5, 3, 6)], 1)
    lam = rng.uniform(0, 0.8, (6, 3))
    Z = np.zeros((ny, nx), np.float32)
    var = oracle.noise_var(oracle.Boundary(g, Z, Z, Z), pts, lam, sigma=sig)
    ref = np.zeros((6, 3))
    for j in range(ny):
        for i in range(nx):
            one = np.zeros((ny, nx), np.float32)
            one[j, i] = 1.0
            a, _, _ = oracle.field(oracle.Boundary(g, one, one, one), pts, lam)
            for p in range(3):
                ref[:, p] += a[:, p] ** 2 * float(sig[p][j, i]) ** 2
    assert np.allclose(var, ref, rtol=1e-12, atol=0)
    # a NULL array means sigma0 on every pixel
    v1 = oracle.noise_var(oracle.Boundary(g, Z, Z, Z), pts, lam, sigma=[sig[0], None, None],
                          sigma0=1.5)
    assert np.allclose(v1[:, 0], var[:, 0], rtol=1e-14)
    v2 = oracle.noise_var(oracle.Boundary(g, Z, Z, Z), pts, lam, sigma0=1.5)
    assert np.allclose(v1[:, 1:], v2[:, 1:], rtol=1e-14)


@pytest.mark.parametrize("lam,z,tol", [(0.0, 4.0, 5e-7), (0.05, 4.0, 2e-6), (0.2, 3.0, 5e-6)])
def test_noise_variance_is_the_integral_of_the_squared_kernel(lam, z, tol):
    """On a 64 x 64 unit grid, sum_k a_ik^2 = dA^2 sum_k K^2 -> dA * (integral of K^2 over the
    magnetogram's square): the midpoint rule's lattice error is ~exp(-2 pi z) and its edge
    (Euler-Maclaurin) term ~(h^2/24) x edge x d(K^2)/dn, about 1e-7 at lambda = 0 and 1e-6 at
    lambda = 0.2 (K^2 falls only as r^-4 for lambda != 0)."""
    n = 64
    Z = np.zeros((n, n), np.float32)
    bd = oracle.Boundary(oracle.Grid(n, n), Z, Z, Z)
    var = oracle.noise_var(bd, np.array([[31.5, 31.5, z]]), np.full((1, 3), lam))[0]

    def K2(y, x):
        r = np.sqrt(x * x + y * y + z * z)
        return (z * (lam * r * np.sin(lam * r) + np.cos(lam * r)) / (2 * np.pi * r ** 3)) ** 2

    I = sum(integrate.dblquad(K2, xa, xb, ya, yb, epsabs=0, epsrel=1e-13)[0]
            for xa, xb in ((-32, 0), (0, 32)) for ya, yb in ((-32, 0), (0, 32)))
    assert np.allclose(var, I, rtol=tol, atol=0), (var, I)
    if lam == 0.0:   # the infinite-plane value 1 / (8 pi z^2), truncated at R = 32: (z / R)^4
        assert abs(var[0] * 8 * np.pi * z * z - 1) < 2 * (z / 32.0) ** 4
