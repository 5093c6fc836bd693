"""Low & Lou (1990) axisymmetric nonlinear force-free field, used as a semi-analytic test field.

The paper validates its method on this family (Sect. 2.3, Table 1, after Schrijver et al. 2006).
The field is written from the published separable solution:

  flux function     A = P(mu) / r^n,  mu = cos(theta),
  toroidal function Q = a |A|^(1 + 1/n),  force-free factor alpha = dQ/dA,
  B_r = -P'(mu) / r^(n+2),  B_theta = n P / (r^(n+2) sin theta),
  B_phi = a |P|^(1 + 1/n) / (r^(n+2) sin theta),
  (1 - mu^2) P'' + n (n + 1) P + a^2 (1 + n)/n * P |P|^(2/n) = 0,  P(-1) = P(1) = 0,

normalised by P'(-1) = 10, with a^2 the m-th positive eigenvalue.  The source sits at depth l
below the photosphere with its axis tilted by Phi in the x-z plane.  The box [-1, 1]^2 of the
boundary is mapped onto the magnetogram: pixel centre i sits at (i - (nx - 1)/2) / (nx / 2).

This module is an input generator: it holds none of the DBIE arithmetic.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

_S0 = 1e-7  # start offset from the singular end point mu = -1


def _rhs(n, a2):
    def f(mu, y):
        P, dP = y
        nl = P * np.abs(P) ** (2.0 / n)
        return [dP, -(n * (n + 1) * P + a2 * (1.0 + n) / n * nl) / (1.0 - mu * mu)]
    return f


def _shoot(n, a2, dense=False):
    c1 = 10.0
    c2 = -n * (n + 1) * c1 / 4.0          # series P = c1 s + c2 s^2 about mu = -1 (s = 1 + mu)
    y0 = [c1 * _S0 + c2 * _S0 ** 2, c1 + 2 * c2 * _S0]
    return solve_ivp(_rhs(n, a2), (-1.0 + _S0, 1.0 - _S0), y0, method="DOP853", rtol=1e-12,
                     atol=1e-13, dense_output=dense)


def _end_value(n, a2):
    sol = _shoot(n, a2)
    P, dP = sol.y[:, -1]
    return P + dP * _S0                    # linear extrapolation to mu = 1


@lru_cache(maxsize=16)
def eigen(n: int, m: int):
    """a^2 of the m-th positive eigenmode and a dense solution P(mu), P'(mu)."""
    grid = np.arange(0.01, 20.0, 0.05)
    roots = []
    prev = _end_value(n, grid[0])
    for k in range(len(grid) - 1):
        cur = _end_value(n, grid[k + 1])
        if np.sign(prev) != np.sign(cur):
            roots.append(brentq(lambda t: _end_value(n, t), grid[k], grid[k + 1], xtol=1e-14,
                                rtol=1e-14))
        prev = cur
        if len(roots) >= m:
            break
    if len(roots) < m:
        raise ValueError(f"no eigenvalue m={m} found for n={n}")
    a2 = roots[m - 1]
    return a2, _shoot(n, a2, dense=True)


class LowLou:
    """The field in box units; ``field(x, y, z)`` and ``alpha(x, y, z)`` take box coordinates."""

    def __init__(self, n: int = 1, m: int = 1, l: float = 0.3, Phi: float = np.pi / 4):
        self.n, self.m, self.l, self.Phi = n, m, l, Phi
        self.a2, self._sol = eigen(n, m)
        self.a = np.sqrt(self.a2)

    def _P(self, mu):
        mu = np.asarray(mu, dtype=np.float64)
        lo, hi = -1.0 + _S0, 1.0 - _S0
        inside = np.clip(mu, lo, hi)
        P, dP = self._sol.sol(inside.ravel())
        P, dP = P.reshape(mu.shape), dP.reshape(mu.shape)
        # Outside the integration range, extend linearly (P vanishes at both ends).
        P = P + dP * (mu - inside)
        return P, dP

    def _local(self, x, y, z):
        c, s = np.cos(self.Phi), np.sin(self.Phi)
        X = x * c - (z + self.l) * s
        Y = y
        Z = x * s + (z + self.l) * c
        return X, Y, Z

    def field(self, x, y, z):
        """(Bx, By, Bz) at box coordinates; arrays broadcast."""
        x, y, z = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (x, y, z)))
        X, Y, Z = self._local(x, y, z)
        n = self.n
        r = np.sqrt(X * X + Y * Y + Z * Z)
        mu = Z / r
        st = np.sqrt(np.maximum(1.0 - mu * mu, 0.0))
        ph = np.arctan2(Y, X)
        P, dP = self._P(mu)
        rn2 = r ** (n + 2)
        Br = -dP / rn2
        Bt = n * P / (rn2 * st)
        Bp = self.a * np.abs(P) ** (1.0 + 1.0 / n) / (rn2 * st)
        cp, sp = np.cos(ph), np.sin(ph)
        BX = Br * st * cp + Bt * mu * cp - Bp * sp
        BY = Br * st * sp + Bt * mu * sp + Bp * cp
        BZ = Br * mu - Bt * st
        c, s = np.cos(self.Phi), np.sin(self.Phi)
        Bx = BX * c + BZ * s
        By = BY
        Bz = -BX * s + BZ * c
        return np.stack([Bx, By, Bz], axis=-1)

    def alpha(self, x, y, z):
        """Force-free factor alpha = dQ/dA = a (1 + 1/n) sign(A) |A|^(1/n) in box units."""
        x, y, z = np.broadcast_arrays(*(np.asarray(v, dtype=np.float64) for v in (x, y, z)))
        X, Y, Z = self._local(x, y, z)
        r = np.sqrt(X * X + Y * Y + Z * Z)
        P, _ = self._P(Z / r)
        A = P / r ** self.n
        return self.a * (1.0 + 1.0 / self.n) * np.sign(A) * np.abs(A) ** (1.0 / self.n)


def box_scale(nx: int) -> float:
    """Pixels per box unit when the box [-1, 1] spans nx pixels."""
    return nx / 2.0


def to_box(nx: int, ny: int, xpx, ypx, zpx, scale: float | None = None):
    """Pixel coordinates (pixel (i, j) centred at (i, j), z in pixels) to box coordinates, with
    the magnetogram centred on the box origin and `scale` pixels per unit (default nx / 2)."""
    s = box_scale(nx) if scale is None else scale
    return ((np.asarray(xpx) - (nx - 1) / 2.0) / s, (np.asarray(ypx) - (ny - 1) / 2.0) / s,
            np.asarray(zpx) / s)
