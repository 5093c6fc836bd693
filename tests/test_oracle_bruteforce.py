"""Brute-force pins of the oracle on tiny grids: Eq. 16 and its derivatives re-derived and summed
in 30-digit arithmetic (mpmath, written here independently of the C oracle: the kernel is
differentiated symbolically by mpmath's own numerical differentiation), and the Downhill Simplex
result checked for local minimality on a dense neighbourhood grid."""
import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")


def _tiny(seed, nx=7, ny=6):
    rng = np.random.default_rng(seed)
    g = oracle.Grid(nx, ny, x0=-1.5, y0=0.25, hx=0.75, hy=1.25)
    comps = [rng.normal(0, 40, (ny, nx)).astype(np.float32) for _ in range(3)]
    return oracle.Boundary(g, *comps), comps, g


def _kernel(x, y, z, xk, yk, lam, area):
    """a_ik of Eq. 16 in mpmath: z [lam r sin(lam r) + cos(lam r)] / (2 pi r^3) dA."""
    r = mp.sqrt((x - xk) ** 2 + (y - yk) ** 2 + z ** 2)
    return z * (lam * r * mp.sin(lam * r) + mp.cos(lam * r)) / (2 * mp.pi * r ** 3) * area


def test_field_matches_30_digit_brute_force():
    bd, comps, g = _tiny(11)
    rng = np.random.default_rng(12)
    pts = np.stack([rng.uniform(-2, 4, 6), rng.uniform(0, 7, 6), rng.uniform(0.3, 3.0, 6)], 1)
    lam = rng.uniform(-0.6, 0.6, (6, 3))
    B, G, dl = oracle.field(bd, pts, lam)
    mp.mp.dps = 30
    area = mp.mpf(g.hx) * mp.mpf(g.hy)
    for i, (x, y, z) in enumerate(pts):
        X, Y, Z = mp.mpf(x), mp.mpf(y), mp.mpf(z)
        for p in range(3):
            L = mp.mpf(lam[i, p])

            def Bp(xx, yy, zz, ll):
                s = mp.mpf(0)
                for j in range(g.ny):
                    for k in range(g.nx):
                        s += _kernel(xx, yy, zz, mp.mpf(g.x0 + k * g.hx), mp.mpf(g.y0 + j * g.hy),
                                     ll, area) * mp.mpf(float(comps[p][j, k]))
                return s

            ref = Bp(X, Y, Z, L)
            assert abs(B[i, p] - float(ref)) <= 1e-13 * (abs(float(ref)) + 1.0)
            # derivatives by mpmath's numerical differentiation at 30 digits
            for jdim, fn in enumerate((lambda t: Bp(t, Y, Z, L), lambda t: Bp(X, t, Z, L),
                                       lambda t: Bp(X, Y, t, L))):
                d = mp.diff(fn, (X, Y, Z)[jdim])
                assert abs(G[i, p, jdim] - float(d)) <= 1e-11 * (abs(float(d)) + 1.0)
            dL = mp.diff(lambda t: Bp(X, Y, Z, t), L)
            assert abs(dl[i, p] - float(dL)) <= 1e-11 * (abs(float(dL)) + 1.0)


@pytest.mark.parametrize("mode", [0, 1])
def test_simplex_ends_at_a_local_minimum(mode):
    """On a tiny grid with a tight tolerance the simplex result is not beaten by any point of a
    dense neighbourhood grid (steps 1e-4 .. 1e-2 of 1/L in every lambda direction)."""
    bd, _, g = _tiny(21, 9, 9)
    rng = np.random.default_rng(22)
    pts = np.stack([rng.uniform(1, 5, 5), rng.uniform(2, 8, 5), rng.uniform(0.8, 3.0, 5)], 1)
    opt = oracle.Options(tol=1e-14, max_iter=2000, eps_f=0.0, eps_g=0.0, lambda_mode=mode)
    r = oracle.solve(bd, pts, opt)
    L = max(g.nx * g.hx, g.ny * g.hy)
    gs = g.hx / 6.0
    dim = 1 if mode else 3
    for i in range(len(pts)):
        lam0 = r["lam"][i].copy()
        best = []
        for scale in (1e-4, 1e-3, 1e-2):
            steps = np.array(np.meshgrid(*[[-1, 0, 1]] * dim, indexing="ij")).reshape(dim, -1).T
            for st in steps:
                if not st.any():
                    continue
                d = np.zeros(3)
                d[:dim] = st * scale / L
                if mode:
                    d[1] = d[2] = d[0]
                lam = lam0 + d
                B, G, _ = oracle.field(bd, pts[i:i + 1], lam[None])
                _, _, phi, _, _ = oracle.objective(B, G, gs)
                best.append(phi[0])
        # |lambda| was reported; Phi is even in each lambda, so the neighbourhood of |lambda*|
        # mirrors that of lambda*
        assert r["phi"][i] <= min(best) + 1e-12, (i, r["phi"][i], min(best))
