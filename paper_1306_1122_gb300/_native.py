"""ctypes binding of libdbie.so (the C ABI in include/dbie.h): argument marshalling only.

Every function here has the name and argument order of its C counterpart.  There is no
fallback: if the library is missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# DBIE_LIBRARY may name another build of the same library (e.g. one compiled with other kernel
# knobs); by default the in-tree libdbie.so is loaded.
LIB_PATH = os.environ.get("DBIE_LIBRARY") or os.path.join(_PKG, "libdbie.so")

DBIE_OK, DBIE_EINVAL, DBIE_ENOMEM, DBIE_ECUDA, DBIE_ETIMEOUT, DBIE_EINTERNAL = range(6)
DBIE_MEM_HOST, DBIE_MEM_DEVICE = 0, 1
DBIE_PREC_MIXED, DBIE_PREC_FP64, DBIE_PREC_FLOAT_FLOAT = 0, 1, 2
DBIE_LAMBDA_PER_COMPONENT, DBIE_LAMBDA_TIED = 0, 1
DBIE_PT_CONVERGED, DBIE_PT_MAXITER = 0, 1
DBIE_METHOD_SIMPLEX, DBIE_METHOD_QUASI_NEWTON = 0, 1
STATUS_NAMES = {0: "DBIE_OK", 1: "DBIE_EINVAL", 2: "DBIE_ENOMEM", 3: "DBIE_ECUDA",
                4: "DBIE_ETIMEOUT", 5: "DBIE_EINTERNAL"}


class dbie_options(ctypes.Structure):
    _fields_ = [("eps_f", ctypes.c_double), ("eps_g", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("lambda_mode", ctypes.c_int32),
                ("simplex_step", ctypes.c_double), ("w_g", ctypes.c_double),
                ("g_scale", ctypes.c_double), ("precision", ctypes.c_int32),
                ("method", ctypes.c_int32), ("near_z", ctypes.c_double),
                ("certify", ctypes.c_double), ("certify_ref", ctypes.c_double)]


class dbie_solve_out(ctypes.Structure):
    _fields_ = [("B", ctypes.c_void_p), ("lambda_", ctypes.c_void_p), ("iters", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("f", ctypes.c_void_p), ("g", ctypes.c_void_p),
                ("nfev", ctypes.c_void_p), ("codes", ctypes.c_void_p),
                ("codes_stride", ctypes.c_int32), ("reserved0", ctypes.c_int32)]


class dbie_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("kernel_ms", ctypes.c_double),
                ("pair_evals", ctypes.c_double), ("objective_pairs", ctypes.c_double),
                ("objective_ms", ctypes.c_double), ("rounds", ctypes.c_int64),
                ("queries", ctypes.c_int64), ("ties", ctypes.c_int64),
                ("refine_pairs", ctypes.c_double), ("refine_ms", ctypes.c_double),
                ("b_refined", ctypes.c_int64), ("difs", ctypes.c_int64),
                ("dif_pairs", ctypes.c_double), ("dif_ms", ctypes.c_double)]


class DBIEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libdbie.so not found at {LIB_PATH}; build it with "
                      "`python paper_1306_1122_gb300/build.py` (needs nvcc)")
lib = ctypes.CDLL(LIB_PATH)

_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "dbie_default_options": (None, [ctypes.POINTER(dbie_options)]),
    "dbie_create": (_I32, [ctypes.POINTER(_P), _I32, _I32, _D, _D, _D, _D, _D, _P, _P, _P, _I32, _P]),
    "dbie_set_boundary": (_I32, [_P, _P, _P, _P, _I32, _P]),
    "dbie_eval": (_I32, [_P, _I64, _P, _P, ctypes.POINTER(dbie_options), _I32, _P, _P, _P, _P, _P]),
    "dbie_objective": (_I32, [_P, _I64, _P, _P, ctypes.POINTER(dbie_options), _I32, _P, _P, _P]),
    "dbie_eval_difference": (_I32, [_P, _I64, _P, _P, _P, _I32, _P, _P, _P]),
    "dbie_solve": (_I32, [_P, _I64, _P, ctypes.POINTER(dbie_options), _P, _I32,
                          ctypes.POINTER(dbie_solve_out), _P]),
    "dbie_solve_batched": (_I32, [_I32, _P, _P, _P, ctypes.POINTER(dbie_options), _P, _I32,
                                  ctypes.POINTER(dbie_solve_out), _P]),
    "dbie_vjp": (_I32, [_P, _I64, _P, _P, _P, ctypes.POINTER(dbie_options), _I32, _P, _P, _I32, _P]),
    "dbie_set_quadrature": (_I32, [_P, _I32, _P]),
    "dbie_hessian": (_I32, [_P, _I64, _P, _P, ctypes.POINTER(dbie_options), _I32, _P, _P, _P, _P]),
    "dbie_vjp_implicit": (_I32, [_P, _I64, _P, _P, _P, ctypes.POINTER(dbie_options), _I32, _P, _P,
                                 _P, _I32, _P]),
    "dbie_noise_var": (_I32, [_P, _I64, _P, _P, _P, _P, _P, _D, ctypes.POINTER(dbie_options),
                              _I32, _P, _P]),
    "dbie_eval_noalloc": (_I32, [_I32, _I32, _D, _D, _D, _D, _D, _P, _P, _P, _I64, _P, _P, _P, _P]),
    "dbie_set_profiling": (_I32, [_P, _I32]),
    "dbie_get_stats": (_I32, [_P, ctypes.POINTER(dbie_stats), _I32]),
    "dbie_autotune": (_I32, [_P, _P]),
    "dbie_get_config": (_I32, [_P, _P]),
    "dbie_set_config": (_I32, [_P, _P]),
    "dbie_destroy": (None, [_P]),
    "dbie_last_error": (ctypes.c_char_p, []),
    "dbie_version": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def check(status: int) -> None:
    if status != DBIE_OK:
        raise DBIEError(status, lib.dbie_last_error().decode())


def dbie_default_options() -> dbie_options:
    o = dbie_options()
    lib.dbie_default_options(ctypes.byref(o))
    return o


def dbie_create(nx, ny, x0, y0, hx, hy, pixel_area, Bx, By, Bz, mem_kind, stream):
    h = _P()
    check(lib.dbie_create(ctypes.byref(h), nx, ny, x0, y0, hx, hy, pixel_area, Bx, By, Bz,
                          mem_kind, stream))
    return h


def dbie_set_boundary(ctx, Bx, By, Bz, mem_kind, stream):
    check(lib.dbie_set_boundary(ctx, Bx, By, Bz, mem_kind, stream))


def dbie_eval(ctx, n, xyz, lam, opt, mem_kind, B, gradB, dBdlam, fgphi, stream):
    check(lib.dbie_eval(ctx, n, xyz, lam, None if opt is None else ctypes.byref(opt), mem_kind, B,
                        gradB, dBdlam, fgphi, stream))


def dbie_objective(ctx, n, xyz, lam, opt, mem_kind, fgphi, dphi, stream):
    check(lib.dbie_objective(ctx, n, xyz, lam, None if opt is None else ctypes.byref(opt),
                             mem_kind, fgphi, dphi, stream))


def dbie_eval_difference(ctx, n, xyz, lam, lam_ref, tied, dS, dS_bound, stream):
    check(lib.dbie_eval_difference(ctx, n, xyz, lam, lam_ref, tied, dS, dS_bound, stream))


def dbie_solve(ctx, n, xyz, opt, lambda_init, mem_kind, out: dbie_solve_out, stream):
    check(lib.dbie_solve(ctx, n, xyz, None if opt is None else ctypes.byref(opt), lambda_init,
                         mem_kind, ctypes.byref(out), stream))


def dbie_solve_batched(nprob, ctxs, n, xyz, opt, lambda_init, mem_kind, outs, stream):
    """ctxs, xyz, lambda_init: sequences of pointers; n: sequence of ints; outs: sequence of
    dbie_solve_out."""
    C = (_P * nprob)(*ctxs)
    N = (_I64 * nprob)(*n)
    X = (_P * nprob)(*xyz)
    L = None if lambda_init is None else (_P * nprob)(*lambda_init)
    O = (dbie_solve_out * nprob)(*outs)
    check(lib.dbie_solve_batched(nprob, C, N, X, None if opt is None else ctypes.byref(opt), L,
                                 mem_kind, O, stream))


def dbie_vjp(ctx, n, xyz, lam, gB, opt, mem_kind, gB0, glam, accumulate, stream):
    check(lib.dbie_vjp(ctx, n, xyz, lam, gB, None if opt is None else ctypes.byref(opt), mem_kind,
                       gB0, glam, accumulate, stream))


def dbie_set_quadrature(ctx, order, stream):
    check(lib.dbie_set_quadrature(ctx, order, stream))


def dbie_hessian(ctx, n, xyz, lam, opt, mem_kind, phi, grad, hess, stream):
    check(lib.dbie_hessian(ctx, n, xyz, lam, None if opt is None else ctypes.byref(opt), mem_kind,
                           phi, grad, hess, stream))


def dbie_vjp_implicit(ctx, n, xyz, lam, gB, opt, mem_kind, gB0, v, flags, accumulate, stream):
    check(lib.dbie_vjp_implicit(ctx, n, xyz, lam, gB, None if opt is None else ctypes.byref(opt),
                                mem_kind, gB0, v, flags, accumulate, stream))


def dbie_noise_var(ctx, n, xyz, lam, sigma_x, sigma_y, sigma_z, sigma0, opt, mem_kind, var,
                   stream):
    check(lib.dbie_noise_var(ctx, n, xyz, lam, sigma_x, sigma_y, sigma_z, sigma0,
                             None if opt is None else ctypes.byref(opt), mem_kind, var, stream))


def dbie_eval_noalloc(nx, ny, x0, y0, hx, hy, pixel_area, Bx, By, Bz, n, xyz, lam, B, stream):
    """Evaluation that allocates nothing: all scratch lives in one fixed device array of the
    library (for callers that may not allocate while they run).  Device pointers only."""
    status = lib.dbie_eval_noalloc(nx, ny, x0, y0, hx, hy, pixel_area, Bx, By, Bz, n, xyz, lam, B,
                                   stream)
    if status != DBIE_OK:
        raise DBIEError(status, "dbie_eval_noalloc failed (message on stderr)")


def dbie_set_profiling(ctx, enable):
    check(lib.dbie_set_profiling(ctx, int(enable)))


def dbie_get_stats(ctx, reset=False) -> dbie_stats:
    st = dbie_stats()
    check(lib.dbie_get_stats(ctx, ctypes.byref(st), int(reset)))
    return st


def dbie_autotune(ctx, stream):
    check(lib.dbie_autotune(ctx, stream))


NCONFIG = 15   # seven pair-sum variants x {per-component, tied} + adjoint


def dbie_get_config(ctx):
    cfg = (_I32 * NCONFIG)()
    check(lib.dbie_get_config(ctx, cfg))
    return list(cfg)


def dbie_set_config(ctx, cfg):
    arr = (_I32 * NCONFIG)(*cfg)
    check(lib.dbie_set_config(ctx, arr))


def dbie_destroy(ctx):
    lib.dbie_destroy(ctx)


def dbie_last_error() -> str:
    return lib.dbie_last_error().decode()


def dbie_version() -> str:
    return lib.dbie_version().decode()
