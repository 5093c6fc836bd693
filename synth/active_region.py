"""Seeded synthetic active-region magnetograms and evaluation-point sets.

Stand-ins for the paper's SDO/HMI vector magnetogram of AR 11158 (Sect. 3: 300 x 300 pixels at
720 km/pixel, 250 x 200 x 100 interior points), which is not available here.  Recipe:

  Bz   = sum_q s_q * peak_q * exp(-|x - c_q|^2 / (2 sigma_q^2))      (Gaussian flux patches)
  B_h  = sbar * (-0.5 grad Bz + 1.0 z_hat x grad Bz)                  (sheared along the PIL)
  + i.i.d. N(0, noise) in every component.

Patch signs alternate along a line through the centre; centres lie in the central 60 % of the
field of view and at least 2.5 sigma apart.  This module holds none of the DBIE arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Magnetogram:
    """Vector magnetogram on an nx-by-ny grid; pixel (i, j) centred at (x0 + i hx, y0 + j hy)."""
    nx: int
    ny: int
    Bx: np.ndarray  # float32 (ny, nx)
    By: np.ndarray
    Bz: np.ndarray
    x0: float = 0.0
    y0: float = 0.0
    hx: float = 1.0
    hy: float = 1.0

    @property
    def dA(self) -> float:
        return self.hx * self.hy

    @property
    def npix(self) -> int:
        return self.nx * self.ny


def _place_centres(rng, nx, ny, sig, sep=2.5, tries=10000):
    k = len(sig)
    lo = np.array([0.2 * nx, 0.2 * ny])
    span = np.array([0.6 * nx, 0.6 * ny])
    # Signs alternate along a line through the centre: draw its angle, order centres along it.
    for _ in range(tries):
        c = lo + rng.random((k, 2)) * span
        ok = True
        for a in range(k):
            for b in range(a):
                if np.hypot(*(c[a] - c[b])) < sep * max(sig[a], sig[b]):
                    ok = False
        if ok:
            return c
    raise RuntimeError("could not place flux patches")


def active_region(nx: int, ny: int, npatch: int, seed: int, peak=(2000.0, 2000.0),
                  sigma=(8.0, 15.0), shear_len: float = 10.0, noise: float = 10.0) -> Magnetogram:
    rng = np.random.default_rng(seed)
    sig = rng.uniform(sigma[0], sigma[1], npatch)
    pk = rng.uniform(peak[0], peak[1], npatch)
    cen = _place_centres(rng, nx, ny, sig)
    theta = rng.uniform(0.0, np.pi)
    axis = np.array([np.cos(theta), np.sin(theta)])
    order = np.argsort(cen @ axis)
    signs = np.empty(npatch)
    signs[order] = [1.0 if q % 2 == 0 else -1.0 for q in range(npatch)]
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    Bz = np.zeros((ny, nx)); dBx = np.zeros((ny, nx)); dBy = np.zeros((ny, nx))
    for q in range(npatch):
        dx, dy = x - cen[q, 0], y - cen[q, 1]
        gq = signs[q] * pk[q] * np.exp(-(dx * dx + dy * dy) / (2 * sig[q] ** 2))
        Bz += gq
        dBx += -dx / sig[q] ** 2 * gq
        dBy += -dy / sig[q] ** 2 * gq
    Bx = shear_len * (-0.5 * dBx - 1.0 * dBy)
    By = shear_len * (-0.5 * dBy + 1.0 * dBx)
    Bx += rng.normal(0.0, noise, Bx.shape)
    By += rng.normal(0.0, noise, By.shape)
    Bz += rng.normal(0.0, noise, Bz.shape)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    m = Magnetogram(nx, ny, f32(Bx), f32(By), f32(Bz))
    m.patches = dict(centre=cen, sigma=sig, peak=pk, sign=signs)
    return m


def monopole_field(m: Magnetogram, pts):
    """Potential field of one submerged monopole per patch (depth sigma_q, charge = patch flux).

    Used only to trace field-line sample points for the large workload."""
    P = m.patches
    pts = np.asarray(pts, dtype=np.float64)
    B = np.zeros_like(pts)
    for q in range(len(P["sigma"])):
        flux = P["sign"][q] * P["peak"][q] * 2 * np.pi * P["sigma"][q] ** 2
        src = np.array([P["centre"][q, 0], P["centre"][q, 1], -P["sigma"][q]])
        d = pts - src
        r = np.linalg.norm(d, axis=-1, keepdims=True)
        B += flux / (2 * np.pi) * d / r ** 3
    return B


def trace_samples(m: Magnetogram, nsamples: int, seed: int, step: float = 0.5,
                  zmin: float = 1.0, zmax: float = 128.0, seed_thresh: float = 200.0,
                  max_steps: int = 4000, stride: int = 4, batch: int = 4096) -> np.ndarray:
    """Field-line samples: RK4 traces (step `step` px) through the monopole potential field,
    seeded at pixels with |Bz| > seed_thresh, each line followed until it leaves the box
    zmin <= z <= zmax inside the field of view; every `stride`-th point along the lines is a
    candidate and nsamples of them are drawn uniformly."""
    rng = np.random.default_rng(seed)
    cand = np.argwhere(np.abs(m.Bz) > seed_thresh)
    pool, have = [], 0
    while have < nsamples:
        pick = cand[rng.integers(0, len(cand), batch)]
        p = np.stack([pick[:, 1] + rng.uniform(-0.5, 0.5, batch),
                      pick[:, 0] + rng.uniform(-0.5, 0.5, batch), np.full(batch, zmin)], axis=1)
        sgn = np.sign(m.Bz[pick[:, 0], pick[:, 1]]).astype(np.float64)[:, None]

        def v(q, s):
            b = monopole_field(m, q)
            return s * b / np.maximum(np.linalg.norm(b, axis=1, keepdims=True), 1e-30)

        # only lines still inside the box are stepped (a line that left stays out)
        for it in range(max_steps):
            k1 = v(p, sgn); k2 = v(p + 0.5 * step * k1, sgn)
            k3 = v(p + 0.5 * step * k2, sgn); k4 = v(p + step * k3, sgn)
            p = p + step / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
            inside = ((p[:, 2] >= zmin) & (p[:, 2] <= zmax) & (p[:, 0] >= 0) & (p[:, 0] <= m.nx - 1)
                      & (p[:, 1] >= 0) & (p[:, 1] <= m.ny - 1))
            p, sgn = p[inside], sgn[inside]
            if len(p) == 0:
                break
            if it % stride == 0:
                pool.append(p.copy())
                have += len(p)
    allp = np.concatenate(pool)
    idx = rng.choice(len(allp), nsamples, replace=False)
    return allp[np.sort(idx)].astype(np.float32)
