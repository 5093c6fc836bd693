"""FP64 CPU oracle for the DBIE quadrature -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct restatement of what Wang, Yan & Tan (arXiv 1306.1122) compute:
the quadrature of Eq. 6 in the discrete form of Eq. 16 (midpoint rule at pixel centres), its
spatial derivatives at fixed lambda (the zeroth-order rule of Eq. 13), J = curl B (Eq. 14), the
measures f (Eq. 8) and g (Eq. 9), and the per-point Downhill Simplex search for lambda
(Sect. 2.1, Nelder & Mead 1965).  The arithmetic lives in ``dbie_oracle.c`` (FP64, Neumaier
compensated, row-major order); this module only marshals numpy arrays.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  It shares no code with the CUDA path and never imports it.

Parity pins (closed forms, invariants, a library Nelder-Mead) live in ``tests/test_oracle_*.py``.
Parity unpinned: the reading of Delta V / Delta sigma in Eq. 9 (``g_scale``), the objective
combination Phi = f + w_g g, the initial simplex and the thresholds eps_f / eps_g, which the paper
leaves open.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, FP64, no FMA contraction, OpenMP over points)."""
    src = os.path.join(_HERE, "dbie_oracle.c")
    hdr = os.path.join(_HERE, "dbie_oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Boundary(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("dA", ctypes.c_double),
                ("Bx", ctypes.c_void_p), ("By", ctypes.c_void_p), ("Bz", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("eps_f", ctypes.c_double), ("eps_g", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("lambda_mode", ctypes.c_int32),
                ("simplex_step", ctypes.c_double), ("w_g", ctypes.c_double),
                ("g_scale", ctypes.c_double), ("deriv", ctypes.c_int32),
                ("fd_delta", ctypes.c_double), ("method", ctypes.c_int32),
                ("quad_order", ctypes.c_int32), ("pxe_near_z", ctypes.c_double)]


class _NMResult(ctypes.Structure):
    _fields_ = [("x", ctypes.c_double * 3), ("fx", ctypes.c_double), ("iters", ctypes.c_int32),
                ("nfev", ctypes.c_int32), ("status", ctypes.c_int32), ("ncodes", ctypes.c_int32)]


FUN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_int32))
FUN_GRAD = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_field.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, P, P, P, P]
            lib.orc_objective.argtypes = [P, P, ctypes.c_double, ctypes.c_double, P, P, P, P, P]
            lib.orc_eval_many.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int32, ctypes.c_double,
                                          P, P, P, ctypes.c_int32]
            lib.orc_solve_many.argtypes = [P, ctypes.c_int64, P, P, P, P, P, P, P, P, P, P, P, P,
                                           ctypes.c_int32, ctypes.c_int32]
            lib.orc_vjp.argtypes = [P, ctypes.c_int64, P, P, P, P, ctypes.c_int32]
            lib.orc_nelder_mead_sim.argtypes = [ctypes.c_int32, P, ctypes.c_double, ctypes.c_int32,
                                                FUN, P, P, P, ctypes.c_int32]
            lib.orc_bfgs.argtypes = [ctypes.c_int32, P, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int32, FUN_GRAD, P, P]
            lib.orc_objective_many.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, P, P,
                                               ctypes.c_int32]
            lib.orc_field_dl.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, P,
                                         P, P, P, P]
            lib.orc_gauss_legendre.argtypes = [ctypes.c_int32, P, P]
            lib.orc_node_weights_q9.argtypes = [P, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_int32, P]
            lib.orc_eval_many_q9.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int32, P, P, P,
                                             ctypes.c_int32]
            lib.orc_vjp_q9.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.c_int32, P, ctypes.c_int32]
            lib.orc_hessian_many.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int32,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             P, P, P, P, ctypes.c_int32]
            lib.orc_implicit_vjp.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.c_int32,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             P, P, P, ctypes.c_int32]
            lib.orc_rect_exact.argtypes = [ctypes.c_double] * 5 + [P]
            lib.orc_pxe_correction.argtypes = [P, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, P, P]
            lib.orc_eval_many_pxe.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_double, P, P, P,
                                              ctypes.c_int32]
            lib.orc_vjp_pxe.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.c_double, P,
                                        ctypes.c_int32]
            lib.orc_noise_var.argtypes = [P, ctypes.c_int64, P, P, P, P, P, ctypes.c_double, P,
                                          ctypes.c_int32]
            _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a.reshape(shape) if shape is not None else a


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Grid:
    """Magnetogram geometry (Eq. 3): pixel (i, j) centred at (x0 + i hx, y0 + j hy, 0)."""
    nx: int
    ny: int
    x0: float = 0.0
    y0: float = 0.0
    hx: float = 1.0
    hy: float = 1.0
    dA: float | None = None

    @property
    def area(self) -> float:
        return self.hx * self.hy if self.dA is None else self.dA


class Boundary:
    """Boundary data held as float32 (ny, nx) arrays, the precision the library receives."""

    def __init__(self, grid: Grid, Bx, By, Bz):
        self.grid = grid
        self.B = [np.ascontiguousarray(np.asarray(c, dtype=np.float32).reshape(grid.ny, grid.nx))
                  for c in (Bx, By, Bz)]
        g = grid
        self._c = _Boundary(g.nx, g.ny, g.x0, g.y0, g.hx, g.hy, g.area,
                            self.B[0].ctypes.data, self.B[1].ctypes.data, self.B[2].ctypes.data)

    @property
    def ref(self):
        return ctypes.byref(self._c)


@dataclass
class Options:
    """Lambda-search options; defaults are the readings stated in the design notes."""
    eps_f: float = 1e-3
    eps_g: float = 1e-4
    tol: float = 1e-6
    max_iter: int = 50
    lambda_mode: int = 0
    simplex_step: float = 0.0   # 0 -> 1 / (max(nx, ny) * hx)
    w_g: float = 1.0
    g_scale: float = 0.0        # 0 -> hx / 6 (cubic cell: dV / dSigma = h^3 / 6 h^2)
    deriv: int = 0
    fd_delta: float = 0.0       # 0 -> 1e-3 * hx (one thousandth of a pixel, Sect. 2.1)
    method: int = 0             # 0: Downhill Simplex (the paper), 1: quasi-Newton (BFGS)
    quad_order: int = 0         # 0: midpoint rule (Eq. 16); g: nine-node elements, g x g Gauss (Eq. 15);
                                # -1: pixel-exact near field (field(..., pxe_near_z=...))
    pxe_near_z: float = 0.0     # quad_order -1: correction for z <= this (0 -> 2 hx)

    def resolved(self, grid: Grid) -> "Options":
        o = Options(**self.__dict__)
        if o.simplex_step == 0.0:
            o.simplex_step = 1.0 / (max(grid.nx, grid.ny) * grid.hx)
        if o.g_scale == 0.0:
            o.g_scale = grid.hx / 6.0
        if o.fd_delta == 0.0:
            o.fd_delta = 1e-3 * grid.hx
        if o.pxe_near_z == 0.0:
            o.pxe_near_z = 2.0 * grid.hx
        return o

    def c(self, grid: Grid) -> _Options:
        o = self.resolved(grid)
        if o.quad_order > 0 and o.method:
            raise ValueError("the oracle's element rule (quad_order > 0) runs with the simplex only")
        if o.quad_order < -1:
            raise ValueError("quad_order must be -1, 0 or a Gauss order")
        return _Options(o.eps_f, o.eps_g, o.tol, o.max_iter, o.lambda_mode, o.simplex_step,
                        o.w_g, o.g_scale, o.deriv, o.fd_delta, o.method, o.quad_order,
                        o.pxe_near_z if o.quad_order == -1 else 0.0)


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def field(bd: Boundary, xyz, lam, deriv: int = 0, fd_delta: float = 1e-3, nthreads=None,
          quad_order: int = 0, pxe_near_z: float | None = None):
    """B (n,3), G (n,3,3) with G[i,p,j] = dB_p/dx_j, and dB/dlambda (n,3) at given lambda (n,3).
    quad_order 0: midpoint rule (Eq. 16); g >= 1: nine-node elements with g x g Gauss points
    (Eq. 15; nx, ny odd); -1: pixel-exact near field for z <= pxe_near_z (default 2 hx)."""
    lib = _load()
    xyz = _f64(xyz).reshape(-1, 3)
    lam = _f64(lam).reshape(-1, 3)
    n = xyz.shape[0]
    B = np.zeros((n, 3)); G = np.zeros((n, 3, 3)); dl = np.zeros((n, 3))
    if quad_order == -1:
        nz = 2.0 * bd.grid.hx if pxe_near_z is None else float(pxe_near_z)
        lib.orc_eval_many_pxe(bd.ref, n, _ptr(xyz), _ptr(lam), nz, _ptr(B), _ptr(G), _ptr(dl),
                              _threads(nthreads))
    elif quad_order:
        _check_q9(bd)
        lib.orc_eval_many_q9(bd.ref, n, _ptr(xyz), _ptr(lam), quad_order, _ptr(B), _ptr(G),
                             _ptr(dl), _threads(nthreads))
    else:
        lib.orc_eval_many(bd.ref, n, _ptr(xyz), _ptr(lam), deriv, fd_delta, _ptr(B), _ptr(G),
                          _ptr(dl), _threads(nthreads))
    return B, G, dl


def _check_q9(bd: Boundary):
    if bd.grid.nx < 3 or bd.grid.ny < 3 or bd.grid.nx % 2 == 0 or bd.grid.ny % 2 == 0:
        raise ValueError("nine-node elements need odd nx, ny >= 3")


def rect_exact(xa, xb, ya, yb, z):
    """Exact integral of z / (2 pi r^3) over [xa, xb] x [ya, yb] (corner minus point coordinates)
    and its derivatives with respect to the point's x, y, z."""
    lib = _load()
    out = np.zeros(4)
    lib.orc_rect_exact(float(xa), float(xb), float(ya), float(yb), float(z), _ptr(out))
    return out


def pxe_correction(bd: Boundary, point):
    """The pixel-exact correction of B (3,) and of G (3, 3) at one point, whatever its z."""
    lib = _load()
    dB = np.zeros(3); dG = np.zeros(9)
    lib.orc_pxe_correction(bd.ref, float(point[0]), float(point[1]), float(point[2]), _ptr(dB),
                           _ptr(dG))
    return dB, dG.reshape(3, 3)


def gauss_legendre(m: int):
    """The oracle's own Gauss-Legendre nodes and weights on [-1, 1]."""
    lib = _load()
    x = np.zeros(m); w = np.zeros(m)
    lib.orc_gauss_legendre(m, _ptr(x), _ptr(w))
    return x, w


def node_weights_q9(bd: Boundary, point, lam: float, order: int):
    """Per node (ny, nx, 5): a_ik, da/dx_i, da/dy_i, da/dz_i, da/dlambda of Eq. 15's elements."""
    lib = _load()
    _check_q9(bd)
    out = np.zeros((bd.grid.ny * bd.grid.nx, 5))
    lib.orc_node_weights_q9(bd.ref, float(point[0]), float(point[1]), float(point[2]), float(lam),
                            order, _ptr(out))
    return out.reshape(bd.grid.ny, bd.grid.nx, 5)


def field_dl(bd: Boundary, xyz, lam):
    """B, G as field(), dB/dlambda (n,3) and dGdl (n,3,3) = d^2 B_p / (dx_j dlambda_p)."""
    lib = _load()
    xyz = _f64(xyz).reshape(-1, 3)
    lam = _f64(lam).reshape(-1, 3)
    n = xyz.shape[0]
    B = np.zeros((n, 3)); G = np.zeros((n, 9)); dl = np.zeros((n, 3)); dG = np.zeros((n, 9))
    for i in range(n):
        lib.orc_field_dl(bd.ref, xyz[i, 0], xyz[i, 1], xyz[i, 2], _ptr(lam[i]),
                         B[i].ctypes.data_as(ctypes.c_void_p), G[i].ctypes.data_as(ctypes.c_void_p),
                         dl[i].ctypes.data_as(ctypes.c_void_p), dG[i].ctypes.data_as(ctypes.c_void_p))
    return B, G.reshape(n, 3, 3), dl, dG.reshape(n, 3, 3)


def objective_grad(bd: Boundary, xyz, lam, g_scale: float, w_g: float = 1.0, nthreads=None,
                   pxe_near_z: float = 0.0):
    """f, g, Phi (n,) and dPhi/dlambda (n,3) at given lambda (n,3) (pxe_near_z > 0: with the
    pixel-exact correction at points with z <= pxe_near_z)."""
    lib = _load()
    xyz = _f64(xyz).reshape(-1, 3)
    lam = _f64(lam).reshape(-1, 3)
    n = xyz.shape[0]
    fgp = np.zeros((n, 3)); dphi = np.zeros((n, 3))
    lib.orc_objective_many(bd.ref, n, _ptr(xyz), _ptr(lam), g_scale, w_g, float(pxe_near_z),
                           _ptr(fgp), _ptr(dphi), _threads(nthreads))
    return fgp[:, 0], fgp[:, 1], fgp[:, 2], dphi


def bfgs(fun_grad, x0, step: float, tol: float, max_iter: int):
    """The oracle's quasi-Newton search on a Python objective: fun_grad(x) -> (value, grad, flag)."""
    lib = _load()
    x0 = _f64(x0)
    n = x0.shape[0]

    def cb(_ctx, xp, gp, flagp):
        v, g, fl = fun_grad(np.array([xp[d] for d in range(n)]))
        for d in range(n):
            gp[d] = float(g[d])
        flagp[0] = int(fl)
        return float(v)

    cfun = FUN_GRAD(cb)
    res = _NMResult()
    x3 = np.zeros(3); x3[:n] = x0
    lib.orc_bfgs(n, _ptr(x3), step, tol, max_iter, cfun, None, ctypes.byref(res))
    return dict(x=np.array(res.x[:n]), fx=res.fx, iters=res.iters, nfev=res.nfev,
                status=res.status)


def objective(B, G, g_scale: float, w_g: float = 1.0):
    """Per-point f (Eq. 8), g (Eq. 9), Phi, J = curl B (Eq. 14) and div B."""
    lib = _load()
    B = _f64(B).reshape(-1, 3)
    G = _f64(G).reshape(-1, 9)
    n = B.shape[0]
    f = np.zeros(n); g = np.zeros(n); phi = np.zeros(n); J = np.zeros((n, 3)); D = np.zeros(n)
    fv, gv, pv, dv = (ctypes.c_double() for _ in range(4))
    Jv = (ctypes.c_double * 3)()
    for i in range(n):
        lib.orc_objective(_ptr(B[i]), _ptr(G[i]), g_scale, w_g, ctypes.byref(fv), ctypes.byref(gv),
                          ctypes.byref(pv), Jv, ctypes.byref(dv))
        f[i], g[i], phi[i], D[i] = fv.value, gv.value, pv.value, dv.value
        J[i] = list(Jv)
    return f, g, phi, J, D


def solve(bd: Boundary, xyz, opt: Options | None = None, lam0=None, nthreads=None, codes_cap=128):
    """Per-point Downhill Simplex over lambda; returns a dict of per-point results."""
    lib = _load()
    opt = opt or Options()
    xyz = _f64(xyz).reshape(-1, 3)
    n = xyz.shape[0]
    oc = opt.c(bd.grid)
    lam = np.zeros((n, 3)); B = np.zeros((n, 3))
    f = np.zeros(n); g = np.zeros(n); phi = np.zeros(n)
    iters = np.zeros(n, np.int32); nfev = np.zeros(n, np.int32); status = np.zeros(n, np.int32)
    codes = np.zeros((n, codes_cap), np.uint8)
    l0 = None if lam0 is None else _f64(lam0).reshape(-1, 3)
    lib.orc_solve_many(bd.ref, n, _ptr(xyz), ctypes.byref(oc), None if l0 is None else _ptr(l0),
                       _ptr(lam), _ptr(B), _ptr(f), _ptr(g), _ptr(phi), _ptr(iters), _ptr(nfev),
                       _ptr(status), _ptr(codes), codes_cap, _threads(nthreads))
    code_str = [bytes(row[: int(it)]).decode() for row, it in zip(codes, np.minimum(iters, codes_cap))]
    return dict(lam=lam, B=B, f=f, g=g, phi=phi, iters=iters, nfev=nfev, status=status,
                codes=code_str)


def vjp(bd: Boundary, xyz, lam, gB, nthreads=None, quad_order: int = 0,
        pxe_near_z: float | None = None):
    """dL/dB0 (ny, nx, 3) for dL/dB = gB (n, 3) at fixed lambda: the transpose of Eq. 16 (of the
    element weights of Eq. 15 when quad_order > 0; with the pixel-exact correction when -1)."""
    lib = _load()
    xyz = _f64(xyz).reshape(-1, 3)
    lam = _f64(lam).reshape(-1, 3)
    gB = _f64(gB).reshape(-1, 3)
    g = bd.grid
    out = np.zeros((g.ny * g.nx, 3))
    if quad_order == -1:
        nz = 2.0 * g.hx if pxe_near_z is None else float(pxe_near_z)
        lib.orc_vjp_pxe(bd.ref, xyz.shape[0], _ptr(xyz), _ptr(lam), _ptr(gB), nz, _ptr(out),
                        _threads(nthreads))
    elif quad_order:
        _check_q9(bd)
        lib.orc_vjp_q9(bd.ref, xyz.shape[0], _ptr(xyz), _ptr(lam), _ptr(gB), quad_order, _ptr(out),
                       _threads(nthreads))
    else:
        lib.orc_vjp(bd.ref, xyz.shape[0], _ptr(xyz), _ptr(lam), _ptr(gB), _ptr(out),
                    _threads(nthreads))
    return out.reshape(g.ny, g.nx, 3)


def hessian(bd: Boundary, xyz, lam, g_scale: float, w_g: float = 1.0, lambda_mode: int = 0,
            nthreads=None, pxe_near_z: float = 0.0):
    """Phi (n,), dPhi/dlambda (n,3), the lambda-Hessian (n,3,3) and dB_p/dlambda_p (n,3), all by
    hyper-dual arithmetic through the quadrature.  Tied mode: entry 0 (and H[:,0,0]) only.
    pxe_near_z > 0: with the pixel-exact correction at points with z <= pxe_near_z."""
    lib = _load()
    xyz = _f64(xyz).reshape(-1, 3)
    lam = _f64(lam).reshape(-1, 3)
    n = xyz.shape[0]
    phi = np.zeros(n); grad = np.zeros((n, 3)); H = np.zeros((n, 9)); dl = np.zeros((n, 3))
    lib.orc_hessian_many(bd.ref, n, _ptr(xyz), _ptr(lam), lambda_mode, g_scale, w_g,
                         float(pxe_near_z), _ptr(phi), _ptr(grad), _ptr(H), _ptr(dl),
                         _threads(nthreads))
    return phi, grad, H.reshape(n, 3, 3), dl


def implicit_vjp(bd: Boundary, xyz, lam, gB, g_scale: float, w_g: float = 1.0,
                 lambda_mode: int = 0, nthreads=None, pxe_near_z: float = 0.0):
    """dL/dB0 (ny, nx, 3) through the lambda search (lambda* a stationary point of Phi), the
    adjoint vectors v = H^-1 dL/dlambda (n, 3) and flags (n,) = 1 where H is not positive
    definite.  pxe_near_z > 0: with the pixel-exact correction (as hessian)."""
    lib = _load()
    xyz = _f64(xyz).reshape(-1, 3)
    lam = _f64(lam).reshape(-1, 3)
    gB = _f64(gB).reshape(-1, 3)
    n = xyz.shape[0]
    g = bd.grid
    out = np.zeros((g.ny * g.nx, 3)); v = np.zeros((n, 3)); flags = np.zeros(n, np.int32)
    lib.orc_implicit_vjp(bd.ref, n, _ptr(xyz), _ptr(lam), _ptr(gB), lambda_mode, g_scale, w_g,
                         float(pxe_near_z), _ptr(out), _ptr(v), _ptr(flags), _threads(nthreads))
    return out.reshape(g.ny, g.nx, 3), v, flags


def noise_var(bd: Boundary, xyz, lam, sigma=None, sigma0: float = 1.0, nthreads=None):
    """Var B_p (n, 3) at fixed lambda for independent pixel noise: sigma = None (sigma0 on every
    pixel) or three (ny, nx) arrays of standard deviations (entries may be None)."""
    lib = _load()
    xyz = _f64(xyz).reshape(-1, 3)
    lam = _f64(lam).reshape(-1, 3)
    n = xyz.shape[0]
    g = bd.grid
    sig = [None, None, None] if sigma is None else list(sigma)
    keep = [None if a is None else np.ascontiguousarray(np.asarray(a, np.float32).reshape(g.ny, g.nx))
            for a in sig]
    var = np.zeros((n, 3))
    lib.orc_noise_var(bd.ref, n, _ptr(xyz), _ptr(lam),
                      *[None if a is None else _ptr(a) for a in keep], sigma0, _ptr(var),
                      _threads(nthreads))
    return var


def nelder_mead(fun, sim0, tol: float, max_iter: int, codes_cap: int = 256):
    """Generic simplex search (the oracle's own) from an explicit (n+1, n) initial simplex.

    ``fun(x) -> (value, flag)``; flag != 0 means the point meets the stopping test of Eq. 12."""
    lib = _load()
    sim0 = _f64(sim0)
    n = sim0.shape[1]

    def cb(_ctx, xp, flagp):
        v, fl = fun(np.array([xp[d] for d in range(n)]))
        flagp[0] = int(fl)
        return float(v)

    cfun = FUN(cb)
    res = _NMResult()
    codes = ctypes.create_string_buffer(codes_cap)
    lib.orc_nelder_mead_sim(n, _ptr(sim0), tol, max_iter, cfun, None, ctypes.byref(res), codes,
                            codes_cap)
    return dict(x=np.array(res.x[:n]), fx=res.fx, iters=res.iters, nfev=res.nfev,
                status=res.status, codes=codes.value.decode())
