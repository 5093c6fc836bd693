"""GPU parity of the fixed-lambda quadrature (dbie_eval) against the FP64 oracle.

Ragged boundaries (not a tile multiple), ragged point counts (not a CTA multiple), tiny and
large z, large lambda r, every output variant, both precisions, host and device memory."""
import ctypes

import numpy as np
import pytest

import oracle
from gates import (TOL_FP64, abs_scales, check_B, check_grad, oracle_boundary)
from synth.active_region import Magnetogram

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbie():
    import paper_1306_1122_gb300 as d
    return d


def random_mag(nx, ny, seed, x0=0.0, y0=0.0, h=1.0, smooth=True):
    rng = np.random.default_rng(seed)
    j, i = np.mgrid[0:ny, 0:nx].astype(np.float64)
    comps = []
    for c in range(3):
        v = rng.normal(0, 30, (ny, nx))
        if smooth:
            cx, cy, s = rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(3, 10)
            v += rng.choice([-1, 1]) * 800 * np.exp(-((i - cx) ** 2 + (j - cy) ** 2) / (2 * s * s))
        comps.append(v.astype(np.float32))
    return Magnetogram(nx, ny, *comps, x0=x0, y0=y0, hx=h, hy=h)


def random_points(mag, n, seed, zlo=0.5, zhi=20.0, lam=0.3):
    rng = np.random.default_rng(seed)
    x = rng.uniform(mag.x0 - 2, mag.x0 + (mag.nx - 1) * mag.hx + 2, n)
    y = rng.uniform(mag.y0 - 2, mag.y0 + (mag.ny - 1) * mag.hy + 2, n)
    z = rng.uniform(zlo, zhi, n)
    xyz = np.stack([x, y, z], 1).astype(np.float32)
    lm = rng.uniform(-lam, lam, (n, 3)).astype(np.float32)
    return xyz, lm


def run_eval(dbie, mag, xyz, lam, precision, near_z=-1.0):
    f = dbie.DBIEField.from_magnetogram(mag)
    opt = dbie.Options(precision=precision, near_z=near_z)
    # (the float-float form, precision 2, evaluates B, its gradient and the objective only)
    r = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), grad=True, dlam=precision != 2,
               objective=True, options=opt)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in r.items()}
    f.close()
    return out


CASES = [(17, 13, 1, 0), (50, 37, 31, 1), (64, 64, 33, 2), (129, 70, 300, 3), (256, 3, 129, 4)]


@pytest.mark.parametrize("nx,ny,n,seed", CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_eval_matches_oracle(dbie, nx, ny, n, seed, precision):
    mag = random_mag(nx, ny, seed, x0=-3.0, y0=5.0)
    xyz, lam = random_points(mag, n, seed + 100)
    got = run_eval(dbie, mag, xyz, lam, precision)
    bd = oracle_boundary(mag)
    B, G, dl = oracle.field(bd, xyz.astype(np.float64), lam.astype(np.float64))
    sB, sG = abs_scales(mag, xyz, lam)
    if precision == 1:
        assert np.all(np.abs(got["B"] - B) <= TOL_FP64 * sB)
        assert np.all(np.abs(got["gradB"] - G) <= TOL_FP64 * sG[:, :, None])
        assert np.all(np.abs(got["dBdlam"] - dl) <= TOL_FP64 * (np.abs(dl) + sB * 100))
    else:
        rb = check_B(got["B"], B, sB)
        assert rb["bad"].size == 0, rb
        rg = check_grad(got["gradB"], G, sG[:, :, None])
        assert rg["ok"], rg
        rl = check_grad(got["dBdlam"], dl, np.abs(dl).max() + 1e-30)
        assert rl["ok"], rl
    # the objective of Eq. 8 / 9 computed on the GPU from its own B and gradient equals the
    # oracle's objective function applied to the same B and gradient
    f, g, phi, _, _ = oracle.objective(got["B"], got["gradB"], g_scale=mag.hx / 6.0)
    assert np.allclose(got["f"], f, rtol=1e-12, atol=1e-14)
    assert np.allclose(got["g"], g, rtol=1e-12, atol=1e-14)
    assert np.allclose(got["phi"], phi, rtol=1e-12, atol=1e-14)


def test_eval_large_lambda_r(dbie):
    """lambda r up to ~90 rad: the SFU sine and cosine over many periods."""
    mag = random_mag(64, 64, 11)
    xyz, _ = random_points(mag, 200, 12, zlo=1.0, zhi=30.0)
    lam = np.full((200, 3), 1.0, np.float32) * np.array([1.0, -0.7, 0.45], np.float32)
    got = run_eval(dbie, mag, xyz, lam, 0)
    B, G, _ = oracle.field(oracle_boundary(mag), xyz.astype(np.float64), lam.astype(np.float64))
    sB, sG = abs_scales(mag, xyz, lam)
    rb = check_B(got["B"], B, sB)
    assert rb["bad"].size == 0, rb
    assert check_grad(got["gradB"], G, sG[:, :, None])["ok"]


def test_eval_lambda_r_at_search_limit(dbie):
    """lambda r up to ~280 rad, above the largest lambda r the searches reach on the workloads
    (about 175 rad on ll128: |lambda| <= 0.97 at distances to 185 px; about 275 rad on ar512:
    |lambda| <= 0.48 at distances to 570 px).  In the mixed form the angle theta = lambda r is
    itself an FP32 value (r from the SFU reciprocal square root, 1.25e-7 relative, times lambda),
    so sin and cos carry a phase error of about 1.5e-7 |theta| on top of the SFU's own (which
    scales its argument by 1/(2 pi) in FP32: 1.1e-7 |theta| measured beyond pi).  An argument
    reduction before the SFU would not remove the first part, so the mixed form's floor relative
    to the absolute-value sum is stated as 1e-6 max(1, theta_max / 100) for a point whose largest
    angle is theta_max; the float-float form, which carries theta and its reduction in
    float-float, stays within 1e-11 of the absolute-value sum here."""
    mag = random_mag(96, 96, 13)
    rng = np.random.default_rng(14)
    n = 300
    xyz = np.stack([rng.uniform(0, 95, n), rng.uniform(0, 95, n), rng.uniform(1.0, 30.0, n)],
                   1).astype(np.float32)
    lam = rng.uniform(1.5, 2.1, (n, 3)).astype(np.float32) * rng.choice([-1, 1], (n, 3))
    lam = lam.astype(np.float32)
    jj, ii = np.mgrid[0:96, 0:96]
    rmax = np.sqrt(np.maximum(xyz[:, 0], 95 - xyz[:, 0]) ** 2 +
                   np.maximum(xyz[:, 1], 95 - xyz[:, 1]) ** 2 + xyz[:, 2] ** 2)
    assert (np.abs(lam).max(axis=1) * rmax).max() > 270
    got = run_eval(dbie, mag, xyz, lam, 0)
    B, G, _ = oracle.field(oracle_boundary(mag), xyz.astype(np.float64), lam.astype(np.float64))
    sB, sG = abs_scales(mag, xyz, lam)
    theta_max = np.abs(lam).max(axis=1) * rmax
    grow = np.maximum(1.0, theta_max / 100.0)[:, None]
    rb = check_B(got["B"], B, sB * grow)
    print(f"lambda r to {theta_max.max():.0f}: mixed max |dB| / S = {rb['max_err_over_S']:.2e}")
    assert rb["bad"].size == 0, rb
    assert check_grad(got["gradB"], G, sG[:, :, None])["ok"]
    ff = run_eval(dbie, mag, xyz, lam, dbie._native.DBIE_PREC_FLOAT_FLOAT)
    assert (np.abs(ff["B"] - B) / sB).max() <= 1e-11


def test_near_field_fp64_correction(dbie):
    """Points at z <= 2 pixels get their near-field pixels in FP64: the mixed result must meet the
    B gate there, and be closer to the oracle than without the correction."""
    mag = random_mag(48, 40, 21)
    rng = np.random.default_rng(22)
    n = 400
    xyz = np.stack([rng.uniform(5, 40, n), rng.uniform(5, 33, n), rng.uniform(0.2, 2.0, n)],
                   1).astype(np.float32)
    xyz[:50, :2] = np.round(xyz[:50, :2])     # exactly above pixel centres
    lam = rng.uniform(-0.2, 0.2, (n, 3)).astype(np.float32)
    with_c = run_eval(dbie, mag, xyz, lam, 0, near_z=-1.0)
    without = run_eval(dbie, mag, xyz, lam, 0, near_z=0.0)
    B, G, _ = oracle.field(oracle_boundary(mag), xyz.astype(np.float64), lam.astype(np.float64))
    sB, sG = abs_scales(mag, xyz, lam)
    rb = check_B(with_c["B"], B, sB)
    assert rb["bad"].size == 0, rb
    assert check_grad(with_c["gradB"], G, sG[:, :, None])["ok"]
    e_with = np.abs(with_c["gradB"] - G).sum()
    e_without = np.abs(without["gradB"] - G).sum()
    assert e_with < e_without
    assert np.abs(with_c["B"] - B).sum() < np.abs(without["B"] - B).sum()


def test_uniform_field_closed_form_on_gpu(dbie):
    """End-to-end physical check: uniform B0 at lambda = 0 gives the solid angle / 2 pi of the
    square plus the lattice term (the same closed form that pins the oracle)."""
    a = 200
    n = 2 * a + 1
    one = np.ones((n, n), np.float32)
    mag = Magnetogram(n, n, one, one, one, x0=-a, y0=-a)
    z = np.array([1.0, 2.0, 3.0], np.float32)
    xyz = np.stack([np.zeros(3), np.zeros(3), z], 1).astype(np.float32)
    lam = np.zeros((3, 3), np.float32)
    for prec in (0, 1):
        got = run_eval(dbie, mag, xyz, lam, prec)
        A = a + 0.5
        for k, zz in enumerate(z.astype(np.float64)):
            lat = sum(np.exp(-2 * np.pi * zz * np.hypot(m1, m2)) for m1 in range(-12, 13)
                      for m2 in range(-12, 13) if m1 or m2)
            exact = 2 / np.pi * np.arctan(A * A / (zz * np.sqrt(2 * A * A + zz * zz))) + lat
            # 5e-8: the midpoint rule's edge term on a 401^2 square (as in the oracle's pin)
            assert np.all(np.abs(got["B"][k] - exact) < (1e-6 if prec == 0 else 5e-8)), (prec, zz)


def test_host_memory_and_determinism(dbie):
    import paper_1306_1122_gb300._native as N
    mag = random_mag(40, 30, 31)
    xyz, lam = random_points(mag, 257, 32)
    dev = run_eval(dbie, mag, xyz, lam, 0)
    dev2 = run_eval(dbie, mag, xyz, lam, 0)
    for k in dev:
        assert np.array_equal(dev[k], dev2[k]), k
    h = N.dbie_create(mag.nx, mag.ny, mag.x0, mag.y0, mag.hx, mag.hy, mag.dA,
                      *(c.ctypes.data_as(ctypes.c_void_p) for c in (mag.Bx, mag.By, mag.Bz)),
                      N.DBIE_MEM_HOST, None)
    B = np.zeros((257, 3))
    G = np.zeros((257, 9))
    L = np.zeros((257, 3))
    F = np.zeros((257, 3))
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    # same outputs as the device run -> same kernel variant, same split count, same bits
    N.dbie_eval(h, 257, P(xyz), P(lam), None, N.DBIE_MEM_HOST, P(B), P(G), P(L), P(F), None)
    N.dbie_destroy(h)
    assert np.array_equal(B, dev["B"])
    assert np.array_equal(G.reshape(-1, 3, 3), dev["gradB"])
    assert np.array_equal(L, dev["dBdlam"])


def test_invalid_points_rejected_and_context_survives(dbie):
    import paper_1306_1122_gb300._native as N
    mag = random_mag(20, 20, 41)
    f = dbie.DBIEField.from_magnetogram(mag)
    bad = np.array([[1.0, 1.0, 0.0]], np.float32)
    B = np.zeros((1, 3))
    lam = np.zeros((1, 3), np.float32)
    st = N.lib.dbie_eval(f.handle, 1, bad.ctypes.data_as(ctypes.c_void_p),
                         lam.ctypes.data_as(ctypes.c_void_p), None, N.DBIE_MEM_HOST,
                         B.ctypes.data_as(ctypes.c_void_p), None, None, None, None)
    assert st == N.DBIE_EINVAL and "z <= 0" in N.dbie_last_error()
    ok = np.array([[1.0, 1.0, 1.0]], np.float32)
    r = f.eval(torch.from_numpy(ok), torch.from_numpy(lam))
    torch.cuda.synchronize()
    assert np.all(np.isfinite(r["B"].cpu().numpy()))
    empty = f.eval(torch.zeros((0, 3)), torch.zeros((0, 3)))
    assert empty["B"].shape == (0, 3)
    f.close()


@pytest.mark.parametrize("cfg", range(6))
def test_every_launch_configuration(dbie, cfg):
    """Each launch configuration the autotuner may pick gives the same sums (FP32 form: within
    the gate; the item split differs between configurations)."""
    mag = random_mag(70, 45, 50 + cfg)
    xyz, lam = random_points(mag, 700, 60 + cfg)
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_config([cfg] * 15)
    r = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), grad=True, dlam=True)
    gB = np.random.default_rng(cfg).normal(0, 1, (700, 3))
    gB0, _ = f.vjp(torch.from_numpy(xyz), torch.from_numpy(lam.astype(np.float64)),
                   torch.from_numpy(gB), glam=False)
    torch.cuda.synchronize()
    bd = oracle_boundary(mag)
    B, G, _ = oracle.field(bd, xyz.astype(np.float64), lam.astype(np.float64))
    sB, sG = abs_scales(mag, xyz, lam)
    rb = check_B(r["B"].cpu().numpy(), B, sB)
    assert rb["bad"].size == 0, rb
    assert check_grad(r["gradB"].cpu().numpy(), G, sG[:, :, None])["ok"]
    ref0 = oracle.vjp(bd, xyz.astype(np.float64), lam.astype(np.float64), gB)
    assert np.linalg.norm(gB0.cpu().numpy() - ref0) / np.linalg.norm(ref0) < 1e-5
    # the solve's objective kernels of this configuration, both lambda modes: the field the
    # search returns equals the oracle's at the returned lambda
    for mode in (0, 1):
        s = f.solve(torch.from_numpy(xyz[:200]), dbie.Options(lambda_mode=mode, max_iter=4))
        torch.cuda.synchronize()
        ls = s["lam"].cpu().numpy()
        Bs, _, _ = oracle.field(bd, xyz[:200].astype(np.float64), ls)
        sBs, _ = abs_scales(mag, xyz[:200], ls)
        assert check_B(s["B"].cpu().numpy(), Bs, sBs)["bad"].size == 0, (cfg, mode)
    f.close()


def test_autotune_picks_valid_configs(dbie):
    mag = random_mag(64, 64, 70)
    f = dbie.DBIEField.from_magnetogram(mag)
    cfg = f.autotune()
    assert len(cfg) == 15 and all(0 <= c < 6 for c in cfg)
    f.close()
