"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every function that
include/dbie.h declares, and rejects bad arguments on the host before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    import __graft_entry__
    __graft_entry__._load_builder().build()
    from paper_1306_1122_gb300 import _native
    return _native


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dbie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dbie_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(native):
    names = declared_functions()
    assert len(names) >= 12, names
    for name in names:
        assert hasattr(native.lib, name), name
        assert name in native.EXPORTED, name


def test_struct_layouts_match_header(native):
    # dbie_options: 3 doubles, 2 int32, 3 doubles, 2 int32, 3 doubles = 88 bytes
    assert ctypes.sizeof(native.dbie_options) == 88
    assert ctypes.sizeof(native.dbie_solve_out) == 8 * 8 + 8
    # dbie_stats: int64, 4 doubles, 2 int64, int64, 2 doubles, int64, int64, 2 doubles = 112 bytes
    assert ctypes.sizeof(native.dbie_stats) == 112


def test_default_options(native):
    o = native.dbie_default_options()
    assert (o.eps_f, o.eps_g, o.tol, o.max_iter) == (1e-3, 1e-4, 1e-6, 50)
    assert o.lambda_mode == native.DBIE_LAMBDA_PER_COMPONENT
    assert o.precision == native.DBIE_PREC_MIXED
    assert o.near_z < 0 and o.simplex_step == 0.0 and o.g_scale == 0.0 and o.w_g == 1.0
    assert o.certify == 0.02 and o.certify_ref == 0.02
    assert native.dbie_version().startswith("dbie-gb300")


def test_argument_errors_are_reported_on_host(native):
    lib = native.lib
    h = ctypes.c_void_p()
    B = np.zeros((4, 4), np.float32)
    p = B.ctypes.data_as(ctypes.c_void_p)
    bad_calls = [
        lambda: lib.dbie_create(None, 4, 4, 0, 0, 1, 1, 1, p, p, p, 0, None),
        lambda: lib.dbie_create(ctypes.byref(h), 0, 4, 0, 0, 1, 1, 1, p, p, p, 0, None),
        lambda: lib.dbie_create(ctypes.byref(h), 4, 4, 0, 0, -1, 1, 1, p, p, p, 0, None),
        lambda: lib.dbie_create(ctypes.byref(h), 4, 4, 0, 0, 1, 1, 0, p, p, p, 0, None),
        lambda: lib.dbie_create(ctypes.byref(h), 4, 4, 0, 0, 1, 1, 1, None, p, p, 0, None),
        lambda: lib.dbie_create(ctypes.byref(h), 4, 4, 0, 0, 1, 1, 1, p, p, p, 7, None),
        lambda: lib.dbie_eval(None, 1, p, p, None, 0, p, None, None, None, None),
        lambda: lib.dbie_solve(None, 1, p, None, None, 0, None, None),
        lambda: lib.dbie_vjp(None, 1, p, p, p, None, 0, p, None, 0, None),
        lambda: lib.dbie_solve_batched(0, None, None, None, None, None, 0, None, None),
        lambda: lib.dbie_set_profiling(None, 1),
        lambda: lib.dbie_set_boundary(None, p, p, p, 0, None),
        lambda: lib.dbie_set_quadrature(None, 0, None),
        lambda: lib.dbie_objective(None, 1, p, p, None, 0, p, None, None),
        lambda: lib.dbie_eval_difference(None, 1, p, p, p, 0, p, None, None),
        lambda: lib.dbie_hessian(None, 1, p, p, None, 0, p, None, None, None),
        lambda: lib.dbie_vjp_implicit(None, 1, p, p, p, None, 0, p, None, None, 0, None),
        lambda: lib.dbie_noise_var(None, 1, p, p, None, None, None, 1.0, None, 0, p, None),
        lambda: lib.dbie_autotune(None, None),
        lambda: lib.dbie_get_config(None, p),
        lambda: lib.dbie_set_config(None, p),
        lambda: lib.dbie_get_stats(None, None, 0),
    ]
    for call in bad_calls:
        assert call() == native.DBIE_EINVAL
        assert native.dbie_last_error() != ""
    # the no-allocation entry point checks its sizes on the host too (its message goes to stderr)
    assert lib.dbie_eval_noalloc(0, 4, 0.0, 0.0, 1.0, 1.0, 1.0, p, p, p, 1, p, p, p,
                                 None) == native.DBIE_EINVAL
    assert lib.dbie_eval_noalloc(256, 257, 0.0, 0.0, 1.0, 1.0, 1.0, p, p, p, 1, p, p, p,
                                 None) == native.DBIE_EINVAL
    lib.dbie_destroy(None)  # no-op


def test_product_has_no_cpu_fallback():
    """The package imports only its native binding: no oracle, numpy or CPU compute path."""
    pkg = os.path.join(ROOT, "paper_1306_1122_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f
