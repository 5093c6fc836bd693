"""PyTorch front end of the DBIE library: device memory, streams and autograd wiring.

All arithmetic runs in libdbie.so; this module allocates tensors, passes their pointers and the
current CUDA stream, and reshapes results.

  DBIEField(Bx, By, Bz, x0, y0, hx, hy)      one magnetogram (Eq. 3) held on the GPU
    .eval(xyz, lam, ...)                      Eq. 16 at fixed lambda (+ gradient, dB/dlambda, f, g)
    .solve(xyz, ...)                          per-point Downhill Simplex lambda search (Sect. 2.1)
    .vjp(xyz, lam, gB)                        dL/dB0 (transpose of Eq. 16) and dL/dlambda
  solve_batched(fields, points, ...)          many magnetograms in one persistent launch per round
  dbie_apply(field, B0, lam, xyz)             autograd function (B0, lambda) -> B
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _native as N

QUAD_PIXEL_EXACT = -1   # DBIE_QUAD_PIXEL_EXACT: exact near-field integration of the lambda = 0 kernel


@dataclass
class Options:
    """Lambda-search and arithmetic options (mirrors dbie_options; None keeps the default)."""
    eps_f: float = 1e-3
    eps_g: float = 1e-4
    tol: float = 1e-6
    max_iter: int = 50
    lambda_mode: int = N.DBIE_LAMBDA_PER_COMPONENT
    simplex_step: float = 0.0
    w_g: float = 1.0
    g_scale: float = 0.0
    precision: int = N.DBIE_PREC_MIXED
    method: int = N.DBIE_METHOD_SIMPLEX
    near_z: float = -1.0
    certify: float = 0.02
    certify_ref: float = 0.02

    def c(self) -> N.dbie_options:
        o = N.dbie_default_options()
        for k, v in self.__dict__.items():
            setattr(o, k, v)
        return o


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_f32(x, device):
    return torch.as_tensor(x).to(device=device, dtype=torch.float32).contiguous()


def _dev_f64(x, device):
    return torch.as_tensor(x).to(device=device, dtype=torch.float64).contiguous()


class DBIEField:
    """One magnetogram: components (ny, nx); pixel (i, j) centred at (x0 + i hx, y0 + j hy)."""

    def __init__(self, Bx, By, Bz, x0=0.0, y0=0.0, hx=1.0, hy=1.0, pixel_area=None,
                 device="cuda"):
        self.device = torch.device(device)
        comps = [_dev_f32(b, self.device) for b in (Bx, By, Bz)]
        self.ny, self.nx = comps[0].shape
        self.x0, self.y0, self.hx, self.hy = float(x0), float(y0), float(hx), float(hy)
        self.pixel_area = float(hx * hy if pixel_area is None else pixel_area)
        with torch.cuda.device(self.device):
            self._h = N.dbie_create(self.nx, self.ny, self.x0, self.y0, self.hx, self.hy,
                                    self.pixel_area, *(_ptr(c) for c in comps),
                                    N.DBIE_MEM_DEVICE, _stream())
        self._keep = None

    @classmethod
    def from_magnetogram(cls, m, device="cuda"):
        return cls(m.Bx, m.By, m.Bz, m.x0, m.y0, m.hx, m.hy, m.dA, device=device)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            N.dbie_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_boundary(self, Bx, By, Bz):
        comps = [_dev_f32(b, self.device).reshape(self.ny, self.nx) for b in (Bx, By, Bz)]
        N.dbie_set_boundary(self._h, *(_ptr(c) for c in comps), N.DBIE_MEM_DEVICE, _stream())
        self._keep = comps  # kept alive until the asynchronous staging has run

    def eval(self, xyz, lam, grad=False, dlam=False, objective=False, options: Options | None = None):
        xyz = _dev_f32(xyz, self.device).reshape(-1, 3)
        lam = _dev_f32(lam, self.device).reshape(-1, 3)
        n = xyz.shape[0]
        kw = dict(device=self.device, dtype=torch.float64)
        B = torch.empty((n, 3), **kw)
        G = torch.empty((n, 3, 3), **kw) if grad else None
        L = torch.empty((n, 3), **kw) if dlam else None
        F = torch.empty((n, 3), **kw) if objective else None
        N.dbie_eval(self._h, n, _ptr(xyz), _ptr(lam), None if options is None else options.c(),
                    N.DBIE_MEM_DEVICE, _ptr(B), _ptr(G), _ptr(L), _ptr(F), _stream())
        out = dict(B=B)
        if grad:
            out["gradB"] = G
        if dlam:
            out["dBdlam"] = L
        if objective:
            out["f"], out["g"], out["phi"] = F[:, 0], F[:, 1], F[:, 2]
        return out

    def objective(self, xyz, lam, options: Options | None = None):
        """f, g, Phi and dPhi/dlambda (n, 3) at fixed lambda."""
        xyz = _dev_f32(xyz, self.device).reshape(-1, 3)
        lam = _dev_f32(lam, self.device).reshape(-1, 3)
        n = xyz.shape[0]
        F = torch.empty((n, 3), device=self.device, dtype=torch.float64)
        D = torch.empty((n, 3), device=self.device, dtype=torch.float64)
        N.dbie_objective(self._h, n, _ptr(xyz), _ptr(lam), None if options is None else options.c(),
                         N.DBIE_MEM_DEVICE, _ptr(F), _ptr(D), _stream())
        return dict(f=F[:, 0], g=F[:, 1], phi=F[:, 2], dphi=D)

    def eval_difference(self, xyz, lam, lam_ref, tied=False, bound=True):
        """Change of the 12 objective sums between lam_ref and lam (n, 12 float64; per component
        S0, S1, Sx, Sy) and, with bound, the worst-case bound of each entry's error."""
        xyz = _dev_f32(xyz, self.device).reshape(-1, 3)
        lam = _dev_f64(lam, self.device).reshape(-1, 3)
        lam_ref = _dev_f64(lam_ref, self.device).reshape(-1, 3)
        n = xyz.shape[0]
        dS = torch.empty((n, 12), device=self.device, dtype=torch.float64)
        dSb = torch.empty((n, 12), device=self.device, dtype=torch.float64) if bound else None
        N.dbie_eval_difference(self._h, n, _ptr(xyz), _ptr(lam), _ptr(lam_ref), int(bool(tied)),
                               _ptr(dS), _ptr(dSb), _stream())
        return (dS, dSb) if bound else dS

    def _solve_out(self, n, codes):
        kw = dict(device=self.device)
        r = dict(B=torch.empty((n, 3), dtype=torch.float64, **kw),
                 lam=torch.empty((n, 3), dtype=torch.float64, **kw),
                 iters=torch.empty(n, dtype=torch.int32, **kw),
                 status=torch.empty(n, dtype=torch.int32, **kw),
                 f=torch.empty(n, dtype=torch.float64, **kw),
                 g=torch.empty(n, dtype=torch.float64, **kw),
                 nfev=torch.empty(n, dtype=torch.int32, **kw))
        so = N.dbie_solve_out()
        so.B, so.lambda_, so.iters, so.status = (_ptr(r[k]) for k in ("B", "lam", "iters", "status"))
        so.f, so.g, so.nfev = _ptr(r["f"]), _ptr(r["g"]), _ptr(r["nfev"])
        if codes:
            r["codes"] = torch.zeros((n, codes), dtype=torch.uint8, **kw)
            so.codes = _ptr(r["codes"])
            so.codes_stride = codes
        return r, so

    def solve(self, xyz, options: Options | None = None, lambda_init=None, codes: int = 0):
        xyz = _dev_f32(xyz, self.device).reshape(-1, 3)
        n = xyz.shape[0]
        l0 = None if lambda_init is None else _dev_f64(lambda_init, self.device).reshape(-1, 3)
        r, so = self._solve_out(n, codes)
        N.dbie_solve(self._h, n, _ptr(xyz), None if options is None else options.c(), _ptr(l0),
                     N.DBIE_MEM_DEVICE, so, _stream())
        return r

    def vjp(self, xyz, lam, gB, glam=True, options: Options | None = None, gB0=None):
        xyz = _dev_f32(xyz, self.device).reshape(-1, 3)
        lam = _dev_f64(lam, self.device).reshape(-1, 3)
        gB = _dev_f64(gB, self.device).reshape(-1, 3)
        n = xyz.shape[0]
        acc = gB0 is not None
        if gB0 is None:
            gB0 = torch.empty((self.ny, self.nx, 3), device=self.device, dtype=torch.float64)
        gl = torch.empty((n, 3), device=self.device, dtype=torch.float64) if glam else None
        N.dbie_vjp(self._h, n, _ptr(xyz), _ptr(lam), _ptr(gB),
                   None if options is None else options.c(), N.DBIE_MEM_DEVICE, _ptr(gB0),
                   _ptr(gl), int(acc), _stream())
        return gB0, gl

    def set_quadrature(self, order: int):
        """0: midpoint rule at pixel centres (Eq. 16); g in 1..8: nine-node elements with g x g
        Gauss points (Eq. 15; nx, ny odd); QUAD_PIXEL_EXACT (-1): the midpoint rule plus the
        exact integration of the lambda = 0 kernel over every pixel at points with
        z <= Options.near_z (the lambda-dependent remainder stays on the midpoint rule)."""
        N.dbie_set_quadrature(self._h, int(order), _stream())

    def hessian(self, xyz, lam, options: Options | None = None):
        """Phi (n,), dPhi/dlambda (n, 3) and the lambda-Hessian (n, 3, 3) at fixed lambda (tied
        mode: the derivatives along the shared lambda in entry 0)."""
        xyz = _dev_f32(xyz, self.device).reshape(-1, 3)
        lam = _dev_f64(lam, self.device).reshape(-1, 3)
        n = xyz.shape[0]
        kw = dict(device=self.device, dtype=torch.float64)
        P, G, H = torch.empty(n, **kw), torch.empty((n, 3), **kw), torch.empty((n, 3, 3), **kw)
        N.dbie_hessian(self._h, n, _ptr(xyz), _ptr(lam), None if options is None else options.c(),
                       N.DBIE_MEM_DEVICE, _ptr(P), _ptr(G), _ptr(H), _stream())
        return dict(phi=P, grad=G, hess=H)

    def vjp_implicit(self, xyz, lam, gB, options: Options | None = None, gB0=None):
        """dL/dB0 (ny, nx, 3) through the lambda search at a stationary lambda (n, 3), plus the
        adjoint vectors v = H^-1 dL/dlambda (n, 3) and flags (n,) (1: H not positive definite,
        only the fixed-lambda term kept).  gB0 given: accumulated into it."""
        xyz = _dev_f32(xyz, self.device).reshape(-1, 3)
        lam = _dev_f64(lam, self.device).reshape(-1, 3)
        gB = _dev_f64(gB, self.device).reshape(-1, 3)
        n = xyz.shape[0]
        acc = gB0 is not None
        if gB0 is None:
            gB0 = torch.empty((self.ny, self.nx, 3), device=self.device, dtype=torch.float64)
        v = torch.empty((n, 3), device=self.device, dtype=torch.float64)
        fl = torch.empty(n, device=self.device, dtype=torch.int32)
        N.dbie_vjp_implicit(self._h, n, _ptr(xyz), _ptr(lam), _ptr(gB),
                            None if options is None else options.c(), N.DBIE_MEM_DEVICE,
                            _ptr(gB0), _ptr(v), _ptr(fl), int(acc), _stream())
        return gB0, v, fl

    def noise_var(self, xyz, lam, sigma=None, sigma0: float = 1.0, options: Options | None = None):
        """Var B (n, 3) at fixed lambda for independent pixel noise: sigma None (sigma0 on every
        pixel) or three (ny, nx) standard-deviation maps (entries may be None)."""
        xyz = _dev_f32(xyz, self.device).reshape(-1, 3)
        lam = _dev_f64(lam, self.device).reshape(-1, 3)
        n = xyz.shape[0]
        sg = [None, None, None] if sigma is None else [
            None if a is None else _dev_f32(a, self.device).reshape(self.ny, self.nx) for a in sigma]
        var = torch.empty((n, 3), device=self.device, dtype=torch.float64)
        N.dbie_noise_var(self._h, n, _ptr(xyz), _ptr(lam), *(_ptr(a) for a in sg), float(sigma0),
                         None if options is None else options.c(), N.DBIE_MEM_DEVICE, _ptr(var),
                         _stream())
        return var

    def autotune(self):
        """Time every launch configuration on this boundary and keep the fastest (cached)."""
        N.dbie_autotune(self._h, _stream())
        return N.dbie_get_config(self._h)

    def set_config(self, cfg):
        N.dbie_set_config(self._h, cfg)

    def set_profiling(self, on=True):
        N.dbie_set_profiling(self._h, on)

    def stats(self, reset=False):
        s = N.dbie_get_stats(self._h, reset)
        return {k: getattr(s, k) for k, _ in s._fields_}


def solve_batched(fields, points, options: Options | None = None, lambda_init=None, codes=0):
    """Solve many magnetograms (each with its own points) with one pair-sum launch per round."""
    assert len(fields) == len(points) and fields
    dev = fields[0].device
    pts = [_dev_f32(p, dev).reshape(-1, 3) for p in points]
    outs, sos = [], []
    for f, p in zip(fields, pts):
        r, so = f._solve_out(p.shape[0], codes)
        outs.append(r)
        sos.append(so)
    l0 = None
    if lambda_init is not None:
        l0t = [None if l is None else _dev_f64(l, dev).reshape(-1, 3) for l in lambda_init]
        l0 = [None if t is None else t.data_ptr() for t in l0t]
    N.dbie_solve_batched(len(fields), [f.handle for f in fields], [p.shape[0] for p in pts],
                         [p.data_ptr() for p in pts], None if options is None else options.c(),
                         l0, N.DBIE_MEM_DEVICE, sos, _stream())
    return outs


class _DBIEFunction(torch.autograd.Function):
    """(B0 (ny, nx, 3), lambda (n, 3)) -> B (n, 3) at fixed points; backward via dbie_vjp."""

    @staticmethod
    def forward(ctx, B0, lam, field: DBIEField, xyz, options):
        field.set_boundary(B0[..., 0], B0[..., 1], B0[..., 2])
        out = field.eval(xyz, lam.detach().to(torch.float32), options=options)
        ctx.field, ctx.options = field, options
        ctx.save_for_backward(xyz, lam)
        ctx.B0_dtype = B0.dtype
        return out["B"]

    @staticmethod
    def backward(ctx, gB):
        xyz, lam = ctx.saved_tensors
        gB0, glam = ctx.field.vjp(xyz, lam.detach().to(torch.float64), gB.contiguous(),
                                  glam=ctx.needs_input_grad[1], options=ctx.options)
        gB0 = gB0.to(ctx.B0_dtype) if ctx.needs_input_grad[0] else None
        if glam is not None:
            glam = glam.to(lam.dtype)
        return gB0, glam, None, None, None


def dbie_apply(field: DBIEField, B0, lam, xyz, options: Options | None = None):
    """Differentiable DBIE evaluation: B = A(lambda) B0 at the points xyz (Eq. 16)."""
    return _DBIEFunction.apply(B0, lam, field, xyz, options)


class _DBIESolveFunction(torch.autograd.Function):
    """B0 (ny, nx, 3) -> B (n, 3) at the searched lambda*(B0); backward through the search
    (dbie_vjp_implicit: lambda* treated as a stationary point of Phi)."""

    @staticmethod
    def forward(ctx, B0, field: DBIEField, xyz, options):
        field.set_boundary(B0[..., 0], B0[..., 1], B0[..., 2])
        r = field.solve(xyz, options)
        ctx.field, ctx.options = field, options
        ctx.save_for_backward(xyz, r["lam"])
        ctx.B0_dtype = B0.dtype
        ctx.mark_non_differentiable(r["lam"])
        return r["B"], r["lam"]

    @staticmethod
    def backward(ctx, gB, _glam):
        xyz, lam = ctx.saved_tensors
        gB0, _, _ = ctx.field.vjp_implicit(xyz, lam, gB.contiguous(), options=ctx.options)
        return gB0.to(ctx.B0_dtype), None, None, None


def dbie_solve_apply(field: DBIEField, B0, xyz, options: Options | None = None):
    """Differentiable solve: (B, lambda*) with B = A(lambda*(B0)) B0 at the points xyz; the
    gradient with respect to B0 includes the change of lambda* (implicit differentiation of the
    lambda search's stationarity condition)."""
    return _DBIESolveFunction.apply(B0, field, xyz, options)
