"""The oracle's OpenMP loops give the same bits for any thread count: every point (and, for the
transposed sums, every pixel) is reduced by one thread in a fixed order, so a race or a
thread-dependent reduction order would show as a difference here.  This is what lets the
parity tests and the timed CPU baseline run the oracle with all host cores."""
import numpy as np

import oracle


def _case(seed, n=40):
    rng = np.random.default_rng(seed)
    nx, ny = 23, 17
    comps = [rng.normal(0, 30, (ny, nx)).astype(np.float32) for _ in range(3)]
    bd = oracle.Boundary(oracle.Grid(nx, ny), *comps)
    xyz = np.stack([rng.uniform(0, 22, n), rng.uniform(0, 16, n), rng.uniform(0.5, 8, n)], 1)
    lam = rng.uniform(-0.2, 0.2, (n, 3))
    gB = rng.normal(size=(n, 3))
    return bd, xyz, lam, gB


def test_field_and_vjp_do_not_depend_on_the_thread_count():
    bd, xyz, lam, gB = _case(900)
    ref_f = oracle.field(bd, xyz, lam, nthreads=1)
    ref_v = oracle.vjp(bd, xyz, lam, gB, nthreads=1)
    ref_p = oracle.field(bd, xyz, lam, nthreads=1, quad_order=-1, pxe_near_z=4.0)
    for t in (2, 3, 8):
        for a, b in zip(oracle.field(bd, xyz, lam, nthreads=t), ref_f):
            assert np.array_equal(a, b)
        assert np.array_equal(oracle.vjp(bd, xyz, lam, gB, nthreads=t), ref_v)
        for a, b in zip(oracle.field(bd, xyz, lam, nthreads=t, quad_order=-1, pxe_near_z=4.0),
                        ref_p):
            assert np.array_equal(a, b)


def test_search_and_second_order_do_not_depend_on_the_thread_count():
    bd, xyz, lam, gB = _case(910, n=24)
    opt = oracle.Options(max_iter=12)
    ref_s = oracle.solve(bd, xyz, opt, nthreads=1)
    ref_h = oracle.hessian(bd, xyz, lam, 1.0 / 6.0, nthreads=1)
    ref_i = oracle.implicit_vjp(bd, xyz, lam, gB, 1.0 / 6.0, nthreads=1)
    for t in (2, 5):
        s = oracle.solve(bd, xyz, opt, nthreads=t)
        for k in ("lam", "B", "iters", "nfev"):
            assert np.array_equal(s[k], ref_s[k]), k
        for a, b in zip(oracle.hessian(bd, xyz, lam, 1.0 / 6.0, nthreads=t), ref_h):
            assert np.array_equal(a, b)
        for a, b in zip(oracle.implicit_vjp(bd, xyz, lam, gB, 1.0 / 6.0, nthreads=t), ref_i):
            assert np.array_equal(a, b)
