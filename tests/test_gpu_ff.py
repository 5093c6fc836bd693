"""GPU parity of the float-float form (DBIE_PREC_FLOAT_FLOAT) of Eq. 16 and its fixed-lambda
derivatives (Eq. 13) against the FP64 oracle.

Every pair term and running sum is a pair of floats (about 48 bits), so the sums must agree with
the oracle's to a small multiple of 2^-44 of their absolute-value sums: the gate is 1e-11 of that
scale for B and the gradient (against 1e-10 for the FP64 GPU form, whose libm-grade sine and
cosine are the looser part), and f, g, Phi recomputed by the oracle from the GPU's B and
gradient agree to rounding.  Ragged boundaries and point counts, z from 0.2 to 30 px, lambda r
up to ~400 rad (the Cody-Waite reduction's range), positive and negative lambda."""
import numpy as np
import pytest

import oracle
from gates import abs_scales, oracle_boundary
from test_gpu_eval import random_mag, random_points, run_eval

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FF = 1e-11
CASES = [(17, 13, 1, 0), (50, 37, 31, 1), (64, 64, 33, 2), (129, 70, 300, 3), (256, 3, 129, 4)]


@pytest.fixture(scope="module")
def dbie():
    import paper_1306_1122_gb300 as d
    return d


def _ff_eval(dbie, mag, xyz, lam):
    f = dbie.DBIEField.from_magnetogram(mag)
    opt = dbie.Options(precision=dbie._native.DBIE_PREC_FLOAT_FLOAT)
    r = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), grad=True, objective=True, options=opt)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in r.items()}
    f.close()
    return out


@pytest.mark.parametrize("nx,ny,n,seed", CASES)
def test_ff_eval_matches_oracle(dbie, nx, ny, n, seed):
    mag = random_mag(nx, ny, seed, x0=-3.0, y0=5.0)
    xyz, lam = random_points(mag, n, seed + 100, zlo=0.2, zhi=30.0)
    got = _ff_eval(dbie, mag, xyz, lam)
    B, G, _ = oracle.field(oracle_boundary(mag), xyz.astype(np.float64), lam.astype(np.float64))
    sB, sG = abs_scales(mag, xyz, lam)
    eB = np.abs(got["B"] - B) / sB
    eG = np.abs(got["gradB"] - G) / sG[:, :, None]
    print(f"FF vs oracle: B {eB.max():.2e}, grad B {eG.max():.2e} of the abs-value sums")
    assert eB.max() <= TOL_FF, eB.max()
    assert eG.max() <= TOL_FF, eG.max()
    f, g, phi, _, _ = oracle.objective(got["B"], got["gradB"], g_scale=mag.hx / 6.0)
    assert np.allclose(got["f"], f, rtol=1e-12, atol=1e-14)
    assert np.allclose(got["g"], g, rtol=1e-12, atol=1e-14)
    assert np.allclose(got["phi"], phi, rtol=1e-12, atol=1e-14)


def test_ff_large_lambda_r_and_value_only(dbie):
    """lambda r up to ~400 rad (k up to ~250 quarter turns in the reduction), B without the
    gradient (the value-only kernel), and the FP64 GPU form on the same points."""
    mag = random_mag(96, 80, 7)
    xyz, _ = random_points(mag, 300, 8, zlo=0.5, zhi=40.0)
    lam = (np.random.default_rng(9).uniform(-3.0, 3.0, (300, 3))).astype(np.float32)
    f = dbie.DBIEField.from_magnetogram(mag)
    X, L = torch.from_numpy(xyz), torch.from_numpy(lam)
    Bff = f.eval(X, L, options=dbie.Options(precision=dbie._native.DBIE_PREC_FLOAT_FLOAT))["B"]
    B64 = f.eval(X, L, options=dbie.Options(precision=1))["B"]
    torch.cuda.synchronize()
    f.close()
    B, _, _ = oracle.field(oracle_boundary(mag), xyz.astype(np.float64), lam.astype(np.float64))
    sB, _ = abs_scales(mag, xyz, lam)
    e_ff = (np.abs(Bff.cpu().numpy() - B) / sB).max()
    e_64 = (np.abs(B64.cpu().numpy() - B) / sB).max()
    print(f"lambda r to 400: FF {e_ff:.2e}, FP64 form {e_64:.2e} of the abs-value sums")
    assert e_ff <= TOL_FF, e_ff


def test_far_lambda_beyond_the_reduction_range(dbie):
    """lambda r past the float-float sine/cosine's Cody-Waite range (12,000 rad), as a quasi-Newton
    trial step with a tiny curvature estimate can produce: the float-float form takes FP64 sincos
    there and still matches the oracle (within the float-float rounding of lambda r itself,
    ~2^-44 |lambda r|), and the mixed form, whose FP64 near field uses the same routine, returns
    finite values up to lambda r ~ 1e9 (its FP32 terms mean little that far out)."""
    mag = random_mag(48, 40, 11)
    rng = np.random.default_rng(12)
    xyz, _ = random_points(mag, 96, 13, zlo=0.3, zhi=3.0)
    # log-uniform |lambda| from 10 to 300 per component, both signs: lambda r to ~2e4
    lam = (rng.choice([-1.0, 1.0], (96, 3)) * 10.0 ** rng.uniform(1.0, 2.5, (96, 3))).astype(
        np.float32)
    got = _ff_eval(dbie, mag, xyz, lam)
    B, G, _ = oracle.field(oracle_boundary(mag), xyz.astype(np.float64), lam.astype(np.float64))
    sB, sG = abs_scales(mag, xyz, lam)
    corners = np.array([[0.0, 0.0], [mag.nx - 1.0, 0.0], [0.0, mag.ny - 1.0],
                        [mag.nx - 1.0, mag.ny - 1.0]])
    r_far = np.sqrt(((xyz[:, None, :2] - corners[None]) ** 2).sum(-1).max(1) + xyz[:, 2] ** 2)
    th_max = float((np.abs(lam).max(1) * r_far).max())      # largest lambda r over all pairs
    tol = TOL_FF * max(1.0, th_max / 400.0)
    eB = (np.abs(got["B"] - B) / sB).max()
    eG = (np.abs(got["gradB"] - G) / sG[:, :, None]).max()
    print(f"lambda r to {th_max:.0f}: FF B {eB:.2e}, grad B {eG:.2e} of the abs-value sums "
          f"(gate {tol:.1e})")
    assert th_max > 12000.0                                    # the fallback range is reached
    assert eB <= tol and eG <= tol
    f = dbie.DBIEField.from_magnetogram(mag)
    for scale in (1e3, 1e5, 1e7):
        far = (np.sign(lam) * scale).astype(np.float32)
        for prec in (0, dbie._native.DBIE_PREC_FLOAT_FLOAT):
            r = f.eval(torch.from_numpy(xyz), torch.from_numpy(far), grad=True,
                       options=dbie.Options(precision=prec))
            torch.cuda.synchronize()
            assert torch.isfinite(r["B"]).all() and torch.isfinite(r["gradB"]).all(), (scale, prec)
    f.close()


def test_ff_rejected_where_not_available(dbie):
    mag = random_mag(20, 20, 3)
    xyz, lam = random_points(mag, 8, 4)
    f = dbie.DBIEField.from_magnetogram(mag)
    opt = dbie.Options(precision=dbie._native.DBIE_PREC_FLOAT_FLOAT)
    with pytest.raises(dbie._native.DBIEError):
        f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), dlam=True, options=opt)
    with pytest.raises(dbie._native.DBIEError):
        f.solve(torch.from_numpy(xyz), opt)
    f.close()
