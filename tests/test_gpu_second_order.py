"""GPU parity of the second-order calls with the oracle: the lambda-Hessian (dbie_hessian), the
gradient through the lambda search (dbie_vjp_implicit, dbie_solve_apply) and the noise variance
(dbie_noise_var).  None of them is in the paper.

Gates: FP64 form 1e-9 relative (the Hessian and the implicit adjoint chain a few FP64 operations
per sum; the sums themselves meet 1e-10); mixed precision: the Hessian's relative Frobenius error
<= 1e-3 over the set (second derivatives of f difference derivative sums, amplifying the FP32
floor), the implicit gradient <= 1e-4 relative Frobenius on well-conditioned minima (H^-1 scales
the sums' 1e-6 error by cond(H) <= 1e3), the variance 1e-5 per element (positive terms, no
cancellation)."""
import numpy as np
import pytest

import oracle
from gates import oracle_boundary
from synth.workloads import small_ll
from test_gpu_eval import random_mag, random_points

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbie():
    import paper_1306_1122_gb300 as d
    return d


def _newton(bd, pts, lam, gs, mode, iters=30):
    lam = lam.copy()
    for _ in range(iters):
        _, gr, H, _ = oracle.hessian(bd, pts, lam, gs, lambda_mode=mode)
        ok = np.linalg.eigvalsh(H[:, :1, :1] if mode == 1 else H)[:, 0] > 0
        if mode == 1:
            st = np.where(ok, gr[:, 0] / np.where(ok, H[:, 0, 0], 1.0), 0.0)
            lam -= st[:, None]
        else:
            Hs = np.where(ok[:, None, None], H, np.eye(3))
            st = np.where(ok[:, None], np.linalg.solve(Hs, gr[:, :, None])[:, :, 0], 0.0)
            lam -= st
        if np.abs(st).max() < 1e-15:
            break
    return lam


@pytest.fixture(scope="module")
def ll_minima():
    """Low & Lou (32 x 32) points at well-conditioned minima of Phi, per lambda mode: the oracle's
    quasi-Newton search, then Newton steps on the oracle's gradient and Hessian."""
    w = small_ll()
    bd = oracle_boundary(w.mag)
    gs = w.mag.hx / 6.0
    idx = np.sort(np.random.default_rng(12).choice(len(w.points), 256, replace=False))
    pts = w.points[idx].astype(np.float64)
    out = {}
    for mode in (0, 1):
        r = oracle.solve(bd, pts, oracle.Options(method=1, max_iter=80, tol=1e-13,
                                                   lambda_mode=mode))
        lam = _newton(bd, pts, r["lam"], gs, mode)
        _, gr, H, _ = oracle.hessian(bd, pts, lam, gs, lambda_mode=mode)
        ev = np.linalg.eigvalsh(H[:, :1, :1] if mode == 1 else H)
        good = (np.abs(gr).max(1) < 1e-10) & (ev[:, 0] > 0) & (ev[:, -1] < 1e3 * ev[:, 0])
        assert good.sum() >= 64, good.sum()
        out[mode] = (pts[good].astype(np.float32), lam[good])
    return w, bd, gs, out


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("mode", [0, 1])
def test_hessian_matches_oracle(dbie, precision, mode):
    mag = random_mag(45, 38, 70 + mode)
    xyz, lam32 = random_points(mag, 300, 71, zlo=0.7, zhi=12.0, lam=0.15)
    lam = np.abs(lam32.astype(np.float64))
    if mode == 1:
        lam[:, 1] = lam[:, 2] = lam[:, 0]
    f = dbie.DBIEField.from_magnetogram(mag)
    r = f.hessian(torch.from_numpy(xyz), torch.from_numpy(lam),
                  dbie.Options(precision=precision, lambda_mode=mode))
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in r.items()}
    bd = oracle_boundary(mag)
    phi, grad, H, _ = oracle.hessian(bd, xyz.astype(np.float64), lam, mag.hx / 6.0,
                                     lambda_mode=mode)
    if precision == 1:
        assert np.allclose(got["phi"], phi, rtol=1e-10, atol=1e-13)
        assert np.abs(got["grad"] - grad).max() <= 1e-9 * np.abs(grad).max()
        assert np.abs(got["hess"] - H).max() <= 1e-9 * np.abs(H).max()
    else:
        assert np.abs(got["phi"] - phi).max() < 1e-4
        assert np.linalg.norm(got["grad"] - grad) <= 1e-3 * np.linalg.norm(grad)
        assert np.linalg.norm(got["hess"] - H) <= 1e-3 * np.linalg.norm(H)
    if mode == 1:
        assert np.all(got["grad"][:, 1:] == 0) and np.all(got["hess"].reshape(-1, 9)[:, 1:] == 0)
    f.close()


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("mode", [0, 1])
def test_implicit_vjp_matches_oracle(dbie, ll_minima, precision, mode):
    w, bd, gs, out = ll_minima
    pts, lam = out[mode]
    gB = np.random.default_rng(13 + mode).normal(size=(len(pts), 3))
    ref, v_ref, fl_ref = oracle.implicit_vjp(bd, pts.astype(np.float64), lam, gB, gs,
                                             lambda_mode=mode)
    fixed = oracle.vjp(bd, pts.astype(np.float64), lam, gB)
    assert not fl_ref.any()
    f = dbie.DBIEField.from_magnetogram(w.mag)
    opt = dbie.Options(precision=precision, lambda_mode=mode)
    gB0, v, fl = f.vjp_implicit(torch.from_numpy(pts), torch.from_numpy(lam),
                                torch.from_numpy(gB), options=opt)
    torch.cuda.synchronize()
    gB0, v, fl = gB0.cpu().numpy(), v.cpu().numpy(), fl.cpu().numpy()
    assert not fl.any()
    # the implicit term is not small here, so a dropped or mis-signed term fails the gate
    assert np.linalg.norm(ref - fixed) > 0.05 * np.linalg.norm(ref)
    err = np.linalg.norm(gB0 - ref) / np.linalg.norm(ref)
    if precision == 1:
        assert err <= 1e-9, err
        assert np.abs(v - v_ref).max() <= 1e-8 * np.abs(v_ref).max()
    else:
        assert err <= 1e-4, err
        assert np.linalg.norm(v - v_ref) <= 1e-3 * np.linalg.norm(v_ref)
    # accumulate adds to what is there
    acc = torch.from_numpy(np.ones_like(ref)).cuda()
    f.vjp_implicit(torch.from_numpy(pts), torch.from_numpy(lam), torch.from_numpy(gB),
                   options=opt, gB0=acc)
    torch.cuda.synchronize()
    assert np.allclose(acc.cpu().numpy() - 1.0, gB0, rtol=1e-12, atol=1e-12 * np.abs(gB0).max())
    f.close()


def test_implicit_vjp_flags_and_empty(dbie):
    """Points without a positive-definite Hessian are flagged (as the oracle flags them) and
    contribute the fixed-lambda adjoint; n = 0 writes zeros."""
    mag = random_mag(30, 26, 80)
    xyz, lam32 = random_points(mag, 200, 81, zlo=1.0, zhi=10.0, lam=0.2)
    lam = np.abs(lam32.astype(np.float64))
    bd = oracle_boundary(mag)
    gs = mag.hx / 6.0
    _, _, H, _ = oracle.hessian(bd, xyz.astype(np.float64), lam, gs)
    ev = np.linalg.eigvalsh(H)
    # away from the boundary of the positive-definite set, so both sides decide the same way
    clear = (ev[:, 0] < -1e-3 * np.abs(ev).max(1)) | (ev[:, 0] > 1e-3 * np.abs(ev).max(1))
    xyz, lam = xyz[clear], lam[clear]
    gB = np.random.default_rng(82).normal(size=(len(xyz), 3))
    ref, v_ref, fl_ref = oracle.implicit_vjp(bd, xyz.astype(np.float64), lam, gB, gs)
    assert fl_ref.sum() >= 5 and (1 - fl_ref).sum() >= 5
    f = dbie.DBIEField.from_magnetogram(mag)
    gB0, v, fl = f.vjp_implicit(torch.from_numpy(xyz), torch.from_numpy(lam), torch.from_numpy(gB),
                                options=dbie.Options(precision=1))
    torch.cuda.synchronize()
    assert np.array_equal(fl.cpu().numpy(), fl_ref)
    assert np.all(v.cpu().numpy()[fl_ref == 1] == 0)
    assert np.linalg.norm(gB0.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)
    e0, _, _ = f.vjp_implicit(torch.zeros((0, 3)), torch.zeros((0, 3), dtype=torch.float64),
                              torch.zeros((0, 3), dtype=torch.float64))
    torch.cuda.synchronize()
    assert e0.shape == (mag.ny, mag.nx, 3) and float(e0.abs().max()) == 0.0
    f.close()


def test_solve_apply_backward_is_the_implicit_adjoint(dbie):
    """dbie_solve_apply: forward = dbie_solve's B; backward = dbie_vjp_implicit at the returned
    lambda (checked against a direct call)."""
    w = small_ll()
    pts = torch.from_numpy(w.points[::16].copy()).cuda()
    f = dbie.DBIEField.from_magnetogram(w.mag)
    B0 = torch.from_numpy(np.stack([w.mag.Bx, w.mag.By, w.mag.Bz], -1)).cuda().requires_grad_(True)
    opt = dbie.Options(method=1, max_iter=40)
    B, lam = dbie.dbie_solve_apply(f, B0, pts, opt)
    gB = torch.randn_like(B)
    (B * gB).sum().backward()
    ref = f.solve(pts, opt)
    assert torch.equal(ref["B"], B.detach()) and torch.equal(ref["lam"], lam)
    g_direct, _, _ = f.vjp_implicit(pts, lam, gB, options=opt)
    torch.cuda.synchronize()
    assert torch.allclose(B0.grad.double(), g_direct.to(B0.grad.device).double(), rtol=1e-5,
                          atol=1e-6 * float(g_direct.abs().max()))
    f.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_noise_var_matches_oracle(dbie, precision, mode):
    mag = random_mag(57, 41, 90)
    xyz, lam32 = random_points(mag, 333, 91, zlo=0.5, zhi=20.0, lam=0.3)
    lam = lam32.astype(np.float64)
    if mode == 1:
        lam[:, 1] = lam[:, 2] = lam[:, 0]
    rng = np.random.default_rng(92)
    sig = [rng.uniform(1.0, 20.0, (mag.ny, mag.nx)).astype(np.float32), None,
           rng.uniform(0.5, 5.0, (mag.ny, mag.nx)).astype(np.float32)]
    f = dbie.DBIEField.from_magnetogram(mag)
    opt = dbie.Options(precision=precision, lambda_mode=mode)
    var = f.noise_var(torch.from_numpy(xyz), torch.from_numpy(lam),
                      sigma=[None if s is None else torch.from_numpy(s) for s in sig], sigma0=7.5,
                      options=opt)
    torch.cuda.synchronize()
    ref = oracle.noise_var(oracle_boundary(mag), xyz.astype(np.float64), lam, sigma=sig, sigma0=7.5)
    rel = np.abs(var.cpu().numpy() - ref) / ref
    assert rel.max() <= (1e-12 if precision == 1 else 1e-5), rel.max()
    e = f.noise_var(torch.zeros((0, 3)), torch.zeros((0, 3), dtype=torch.float64))
    assert e.shape == (0, 3)
    f.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_hessian_on_element_rule_matches_oracle_differences(dbie, precision):
    """dbie_hessian with Eq. 15's nine-node elements (3 x 3 Gauss points; the split-position
    pair-sum kernels): Phi, its lambda-gradient and lambda-Hessian against central differences of
    the oracle's element-rule Phi (steps 2^-14 in lambda, all evaluations in one oracle call).
    FP64 form 1e-5, mixed 1e-3 relative Frobenius over the set (the differences carry ~1e-6)."""
    mag = random_mag(25, 25, 230)
    rng = np.random.default_rng(231)
    n = 16
    pts = np.stack([rng.uniform(4, 20, n), rng.uniform(4, 20, n), rng.uniform(1, 6, n)],
                   1).astype(np.float32)
    lam = rng.uniform(0.02, 0.08, (n, 3)) * rng.choice([-1.0, 1.0], (n, 3))
    gs = mag.hx / 6.0
    h = 2.0 ** -14
    E = np.eye(3)
    shifts = [np.zeros(3)]
    for j in range(3):
        shifts += [2 * h * E[j], -2 * h * E[j]]
    for j in range(3):
        for k in range(j + 1, 3):
            shifts += [h * (E[j] + E[k]), h * (E[j] - E[k]), h * (E[k] - E[j]), -h * (E[j] + E[k])]
    S = np.array(shifts)                                   # (19, 3)
    L = (lam[:, None, :] + S[None]).reshape(-1, 3)
    X = np.repeat(pts.astype(np.float64), len(S), axis=0)
    bd = oracle_boundary(mag)
    B, G, _ = oracle.field(bd, X, L, quad_order=3)
    _, _, phi, _, _ = oracle.objective(B, G, g_scale=gs)
    P = phi.reshape(n, len(S))
    H = np.zeros((n, 3, 3))
    grad = np.zeros((n, 3))
    for j in range(3):
        grad[:, j] = (P[:, 1 + 2 * j] - P[:, 2 + 2 * j]) / (4 * h)
        H[:, j, j] = (P[:, 1 + 2 * j] - 2 * P[:, 0] + P[:, 2 + 2 * j]) / (4 * h * h)
    c = 7
    for j in range(3):
        for k in range(j + 1, 3):
            H[:, j, k] = H[:, k, j] = (P[:, c] - P[:, c + 1] - P[:, c + 2] + P[:, c + 3]) / (4 * h * h)
            c += 4
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(3)
    r = f.hessian(torch.from_numpy(pts), torch.from_numpy(lam),
                  dbie.Options(precision=precision))
    torch.cuda.synchronize()
    f.close()
    got = {k: v.cpu().numpy() for k, v in r.items()}
    tol = 1e-5 if precision == 1 else 1e-3
    assert np.allclose(got["phi"], P[:, 0], rtol=1e-9 if precision == 1 else 1e-4, atol=1e-12)
    eg = np.linalg.norm(got["grad"] - grad) / np.linalg.norm(grad)
    eH = np.linalg.norm(got["hess"] - H) / np.linalg.norm(H)
    print(f"element rule, precision {precision}: gradient {eg:.1e}, Hessian {eH:.1e}")
    assert eg <= tol and eH <= tol, (eg, eH)


def test_implicit_vjp_on_element_rule_matches_perturbation(dbie):
    """dbie_vjp_implicit with Eq. 15's elements (3 x 3 Gauss points; the split-position Hessian
    pass and seven-weight sweep), FP64 form, against the derivative it stands for:
    L(B0) = gB . B(lambda*(B0), B0) along a random direction of +-2^-6 per pixel (exact in
    float32), lambda* re-found by Newton steps on the GPU's own FP64 gradient and Hessian after
    each perturbation, L evaluated as <A(lambda*)^T gB, B0> with the fixed-lambda adjoint (FP64
    lambda); central difference against <dL/dB0, direction>.  The fixed-lambda adjoint misses
    the lambda* term by more than 5 %."""
    mag = random_mag(25, 25, 240)
    rng = np.random.default_rng(241)
    n = 48
    pts = np.stack([rng.uniform(5, 19, n), rng.uniform(5, 19, n), rng.uniform(2, 6, n)],
                   1).astype(np.float32)
    opt = dbie.Options(precision=1)
    f = dbie.DBIEField.from_magnetogram(mag)
    f.set_quadrature(3)
    X = torch.from_numpy(pts)
    lam = f.solve(X, dbie.Options(precision=1, max_iter=60))["lam"].cpu().numpy()

    def newton(xyz, lam, iters):
        for _ in range(iters):
            r = f.hessian(xyz, torch.from_numpy(lam), opt)
            g, H = r["grad"].cpu().numpy(), r["hess"].cpu().numpy()
            lam = lam - np.linalg.solve(H, g[..., None])[..., 0]
        return lam, g, H

    lam, g, H = newton(X, lam, 8)
    ev = np.linalg.eigvalsh(H)
    keep = (ev[:, 0] > 0) & (ev[:, -1] < 1e3 * ev[:, 0]) & (np.abs(g).max(1) < 1e-9)
    assert keep.sum() >= 8, keep.sum()
    Xk, lam = X[torch.from_numpy(keep)], lam[keep]
    gB = rng.normal(size=(int(keep.sum()), 3))
    gB0, _, fl = f.vjp_implicit(Xk, torch.from_numpy(lam), torch.from_numpy(gB), options=opt)
    fixed, _ = f.vjp(Xk, torch.from_numpy(lam), torch.from_numpy(gB), glam=False, options=opt)
    torch.cuda.synchronize()
    assert not fl.cpu().numpy().any()
    gB0, fixed = gB0.cpu().numpy(), fixed.cpu().numpy()
    B0 = np.stack([mag.Bx, mag.By, mag.Bz], -1).astype(np.float64)
    d = (rng.choice([-1.0, 0.0, 1.0], B0.shape) * 2.0 ** -6).astype(np.float32)
    L = []
    for s in (1.0, -1.0):
        Bs = (B0.astype(np.float32) + np.float32(s) * d)
        f.set_boundary(*(torch.from_numpy(np.ascontiguousarray(Bs[..., p])) for p in range(3)))
        ls, _, _ = newton(Xk, lam, 5)
        At, _ = f.vjp(Xk, torch.from_numpy(ls), torch.from_numpy(gB), glam=False, options=opt)
        torch.cuda.synchronize()
        L.append(float((At.cpu().numpy() * Bs.astype(np.float64)).sum()))
    f.close()
    fd = (L[0] - L[1]) / 2.0
    pred = float((gB0 * d).sum())
    pred_fixed = float((fixed * d).sum())
    print(f"element rule implicit adjoint: directional derivative {fd:.6e}, adjoint {pred:.6e}, "
          f"fixed-lambda {pred_fixed:.6e}")
    assert abs(pred - fd) <= 1e-6 * abs(fd), (pred, fd)
    assert abs(pred_fixed - fd) > 0.05 * abs(fd)
