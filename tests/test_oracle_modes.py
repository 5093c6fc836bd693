"""Pins of the oracle's lambda-dependent kernel against infinite-plane closed forms (Sect. 2.1:
each component of B solves the Helmholtz equation (laplacian + lambda^2) B_p = 0 above the
boundary and decays, so the DBIE with the right lambda reproduces any such field):

- a Fourier mode B0 = cos(k x) maps to cos(k x) exp(-sqrt(k^2 - lambda^2) z) for k > lambda and
  cos(k x) cos(sqrt(lambda^2 - k^2) z) for k < lambda;
- the linear force-free mode B = ((kappa/k) sin kx, (alpha/k) sin kx, cos kx) exp(-kappa z),
  kappa^2 = k^2 - alpha^2 (curl B = alpha B, div B = 0) is reproduced at lambda_p = alpha, its
  force-freeness measure f (Eq. 8) vanishes there, and the (tied) lambda search finds alpha;
- dB/dlambda of uniform data equals the lambda-derivative of the square's closed-form integral.

The lattice is finite, so the infinite-plane forms hold up to a truncation tail that decays like
1 / A (A the half-width); the checks are convergence in A plus a bound far below the difference
between the right answer and the plausible wrong ones (wrong branch, wrong sign of lambda^2)."""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle
from test_oracle_pins import uniform_square


def _cos_mode(k, A):
    n = 2 * A + 1
    g = oracle.Grid(n, n, x0=-A, y0=-A)
    x = -A + np.arange(n, dtype=np.float64)
    b = np.repeat(np.cos(k * x)[None, :], n, axis=0).astype(np.float32)
    return oracle.Boundary(g, b, b, b)


def _response(k, lam, z):
    if k > lam:
        return np.exp(-np.sqrt(k * k - lam * lam) * z)
    return np.cos(np.sqrt(lam * lam - k * k) * z)


@pytest.mark.parametrize("k,lam", [(0.3, 0.1), (0.1, 0.3), (0.5, 0.0)])
def test_fourier_mode_spectrum(k, lam):
    """B0 = cos(k x): B(x, y, z) -> cos(k x) times the Helmholtz response, decaying for k > lambda
    and oscillating in z for k < lambda; the truncation error falls from ~3e-3 (A = 100) to
    ~1e-4 (A = 800), while the wrong branch or a flipped sign of lambda^2 is off by > 3e-2."""
    z, x = 3.0, 1.3
    ex = np.cos(k * x) * _response(k, lam, z)
    wrong = np.cos(k * x) * np.exp(-np.sqrt(k * k + lam * lam) * z)
    errs = []
    for A in (100, 800):
        B, _, _ = oracle.field(_cos_mode(k, A), [[x, 0.0, z]], [[lam] * 3])
        assert np.all(B[0] == B[0, 0])               # three identical components
        errs.append(abs(B[0, 0] - ex))
    assert errs[1] < 5e-4 and errs[1] < errs[0], errs
    if lam > 0:
        assert abs(wrong - ex) > 60 * 5e-4


def _d_square_integral(z, A, lam):
    """lambda-derivative of the square integral: the angular mean of
    d/dlambda [cos(lambda z) - z cos(lambda R')/R'] = -z sin(lambda z) + z sin(lambda R')."""
    def F(th):
        R = A / max(abs(np.cos(th)), abs(np.sin(th)))
        return -z * np.sin(lam * z) + z * np.sin(lam * np.hypot(R, z))

    v, _ = quad(F, 0, 2 * np.pi, points=[np.pi / 4 * (2 * k + 1) for k in range(4)], limit=400,
                epsabs=1e-13, epsrel=1e-13)
    return v / (2 * np.pi)


@pytest.mark.parametrize("lam", [0.05, 0.2])
def test_uniform_field_lambda_derivative_closed_form(lam):
    """dB/dlambda of uniform data at the square's centre against the lambda-
    derivative of the closed-form square integral (angular mean of cos(lambda z) - z cos(lambda R')/R',
    differentiated under the mean).  The
    pixel sum over the square [-40.5, 40.5]^2 carries the midpoint rule's O(h^2) edge term
    (the lambda-derivative of the kernel decays only like 1/r), so it is extrapolated h -> 0 over
    the same square (h = 1, 1/3, 1/9; Richardson on the h^2 and h^4 terms); at z = 3 the lattice
    term and its lambda-derivative are below 1e-8."""
    z, A = 3.0, 40.5
    S = []
    for a, h in [(40, 1.0), (121, 1.0 / 3.0), (364, 1.0 / 9.0)]:
        _, _, dl = oracle.field(uniform_square(a, h), [[0.0, 0.0, z]], [[lam] * 3])
        S.append(dl[0, 0])
    R1 = [(9 * S[1] - S[0]) / 8, (9 * S[2] - S[1]) / 8]     # h^2 term removed
    C = (81 * R1[1] - R1[0]) / 80                           # h^4 term removed
    ref = _d_square_integral(z, A, lam)
    assert abs(C - ref) < 1e-8 * max(1.0, abs(ref)), (C, S, ref)
    assert abs(S[0] - ref) > 1000 * abs(C - ref)       # the extrapolation is what closes the gap


K_MODE, ALPHA = 0.3, 0.2


def _lff_mode(A):
    kap = np.sqrt(K_MODE ** 2 - ALPHA ** 2)
    n = 2 * A + 1
    g = oracle.Grid(n, n, x0=-A, y0=-A)
    x = -A + np.arange(n, dtype=np.float64)
    rows = lambda v: np.repeat(v[None, :], n, axis=0).astype(np.float32)   # noqa: E731
    return oracle.Boundary(g, rows(kap / K_MODE * np.sin(K_MODE * x)),
                           rows(ALPHA / K_MODE * np.sin(K_MODE * x)), rows(np.cos(K_MODE * x)))


def _lff_truth(P):
    kap = np.sqrt(K_MODE ** 2 - ALPHA ** 2)
    e = np.exp(-kap * P[:, 2])
    s, c = np.sin(K_MODE * P[:, 0]), np.cos(K_MODE * P[:, 0])
    return np.stack([kap / K_MODE * s * e, ALPHA / K_MODE * s * e, c * e], 1)


def test_linear_force_free_mode_reproduced_at_alpha():
    """At lambda_p = alpha the DBIE returns the analytic linear force-free field (truncation
    1.9e-3 at A = 200, 1.6e-4 at A = 400), and f there is ~1e-3 of its value at lambda = 0."""
    P = np.array([[1.3, 0.0, 3.0], [4.0, 2.0, 5.0], [-2.2, 1.0, 4.0]])
    errs = []
    for A in (200, 400):
        B, G, _ = oracle.field(_lff_mode(A), P, np.full((3, 3), ALPHA))
        errs.append(np.abs(B - _lff_truth(P)).max())
    assert errs[1] < 5e-4 and errs[1] < errs[0] / 4, errs
    B0, G0, _ = oracle.field(_lff_mode(400), P, np.zeros((3, 3)))
    fa = oracle.objective(B, G, 1.0 / 6.0)[0]
    f0 = oracle.objective(B0, G0, 1.0 / 6.0)[0]
    assert np.all(fa < 0.02 * f0), (fa, f0)


def test_linear_force_free_mode_search_finds_alpha():
    """The lambda search (one lambda per point) started at 0 converges to |lambda*| = alpha.
    (With three free lambdas the minimiser is not unique, as Sect. 2.1 notes.)"""
    P = np.array([[1.3, 0.0, 3.0], [4.0, 2.0, 5.0], [-2.2, 1.0, 4.0]])
    r = oracle.solve(_lff_mode(200), P, oracle.Options(simplex_step=0.05, max_iter=80, tol=1e-12,
                                                        lambda_mode=1))
    assert np.all(np.abs(r["lam"][:, 0] - ALPHA) < 0.005), r["lam"][:, 0]
    assert np.all(r["lam"] == r["lam"][:, :1])
