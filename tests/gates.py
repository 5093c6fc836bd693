"""Parity gates of the GPU path against the FP64 oracle (tolerances written out here).

Mixed precision evaluates every pair term in FP32 with the SFU sine and cosine, whose absolute
error is about 2^-21, so each term carries a relative error of order 1e-6 and a sum over pixels is
accurate to delta * S_i with S_i = sum_k |a_ik| |B0_k| (the absolute-value sum) and delta <~ 1e-6
(measured on GB300: at most 6e-7).  The gates follow from that:

  B:     per point |dB_i| <= max(1e-5 |B_i|, 1e-6 |S_i|): 1e-5 relative wherever the sum is
         well conditioned (S_i <= 10 |B_i|), the FP32 floor where cancellation dominates; and the
         Frobenius error over all points <= 1e-5 relative.
  grads: relative Frobenius <= 1e-4, and elementwise <= 1e-4 of the absolute-value sum scale.
  FP64 GPU form: 1e-10 of the absolute-value sum scale.
"""
import numpy as np

import oracle

TOL_B_MIXED = 1e-5
FLOOR_B_MIXED = 1e-6   # delta: FP32 / SFU per-term floor relative to the absolute-value sum
TOL_GRAD_MIXED = 1e-4
TOL_FP64 = 1e-10


def oracle_boundary(mag):
    g = oracle.Grid(mag.nx, mag.ny, x0=mag.x0, y0=mag.y0, hx=mag.hx, hy=mag.hy, dA=mag.dA)
    return oracle.Boundary(g, mag.Bx, mag.By, mag.Bz)


def abs_scales(mag, xyz, lam):
    """Per point and component: sum_k |a_ik(lambda_p)| |B0_p,k| and the same for the gradient
    weights (|da/dx| + |da/dy| + |da/dz|) -- tolerance scales only."""
    xyz = np.asarray(xyz, np.float64).reshape(-1, 3)
    lam = np.asarray(lam, np.float64).reshape(-1, 3)
    j, i = np.mgrid[0:mag.ny, 0:mag.nx].astype(np.float64)
    xk = (mag.x0 + i * mag.hx).ravel()
    yk = (mag.y0 + j * mag.hy).ravel()
    B0 = [np.abs(np.asarray(c, np.float64).ravel()) for c in (mag.Bx, mag.By, mag.Bz)]
    w = mag.dA / (2 * np.pi)
    sB = np.zeros((len(xyz), 3))
    sG = np.zeros((len(xyz), 3))
    for n, (x, y, z) in enumerate(xyz):
        dx, dy = x - xk, y - yk
        r = np.sqrt(dx * dx + dy * dy + z * z)
        for p in range(3):
            lr = lam[n, p] * r
            u = lr * np.sin(lr) + np.cos(lr)
            psi = (lam[n, p] ** 2 * np.cos(lr) - 3 * u / r ** 2) / r ** 3
            a = np.abs(z * u / r ** 3) * w
            g = (np.abs(z * dx * psi) + np.abs(z * dy * psi) + np.abs(u / r ** 3 + z * z * psi)) * w
            sB[n, p] = np.sum(a * B0[p])
            sG[n, p] = np.sum(g * B0[p])
    return sB, sG


def check_B(B_gpu, B_ref, sB, tol=TOL_B_MIXED, floor=FLOOR_B_MIXED):
    B_gpu = np.asarray(B_gpu, np.float64).reshape(-1, 3)
    B_ref = np.asarray(B_ref, np.float64).reshape(-1, 3)
    S = np.linalg.norm(np.asarray(sB).reshape(-1, 3), axis=1)
    nB = np.linalg.norm(B_ref, axis=1)
    err = np.linalg.norm(B_gpu - B_ref, axis=1)
    bound = np.maximum(tol * nB, floor * S)
    bad = np.nonzero(err > bound)[0]
    well = S <= 10 * nB
    rel = err / np.maximum(nB, 1e-300)
    frob = float(np.linalg.norm(B_gpu - B_ref) / max(np.linalg.norm(B_ref), 1e-300))
    if frob > tol:
        bad = np.union1d(bad, [-1])
    return dict(max_rel_well=float(rel[well].max(initial=0.0)), max_err_over_S=float(
        (err / np.maximum(S, 1e-300)).max(initial=0.0)), frob=frob, n_well=int(well.sum()),
        frac_rel_1e5=float(np.mean(rel <= tol)) if len(rel) else 1.0, bad=bad)


def check_grad(G_gpu, G_ref, scale, tol=TOL_GRAD_MIXED):
    G_gpu = np.asarray(G_gpu, np.float64)
    G_ref = np.asarray(G_ref, np.float64)
    frob = np.linalg.norm(G_gpu - G_ref) / max(np.linalg.norm(G_ref), 1e-300)
    scale = np.broadcast_to(np.asarray(scale, np.float64), G_ref.shape) if np.ndim(scale) else scale
    elem = np.max(np.abs(G_gpu - G_ref) / np.maximum(scale, 1e-300))
    return dict(frob=float(frob), elem=float(elem), ok=bool(frob <= tol and elem <= tol))
