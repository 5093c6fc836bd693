"""GPU parity of the backward pass: the boundary adjoint dL/dB0 (transpose of Eq. 16, kernel
recomputed), dL/dlambda, the adjoint identity, and the autograd function."""
import numpy as np
import pytest

import oracle
from gates import oracle_boundary
from test_gpu_eval import random_mag, random_points

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbie():
    import paper_1306_1122_gb300 as d
    return d


def vjp_scale(mag, xyz, lam, gB):
    """sum_i |gB_pi| |a_ik| per pixel and component (tolerance scale)."""
    j, i = np.mgrid[0:mag.ny, 0:mag.nx].astype(np.float64)
    xk = (mag.x0 + i * mag.hx).ravel()
    yk = (mag.y0 + j * mag.hy).ravel()
    out = np.zeros((mag.ny * mag.nx, 3))
    for (x, y, z), l, g in zip(xyz.astype(np.float64), lam, gB):
        r = np.sqrt((x - xk) ** 2 + (y - yk) ** 2 + z * z)
        for p in range(3):
            lr = l[p] * r
            out[:, p] += np.abs(g[p]) * np.abs(z * (lr * np.sin(lr) + np.cos(lr)) / r ** 3)
    return out.reshape(mag.ny, mag.nx, 3) * mag.dA / (2 * np.pi)


@pytest.mark.parametrize("nx,ny,n,seed", [(17, 13, 5, 0), (64, 48, 700, 1), (130, 9, 257, 2)])
@pytest.mark.parametrize("precision", [0, 1])
def test_vjp_matches_oracle(dbie, nx, ny, n, seed, precision):
    mag = random_mag(nx, ny, seed)
    xyz, lam = random_points(mag, n, seed + 1)
    lam = lam.astype(np.float64)
    gB = np.random.default_rng(seed + 2).normal(0, 1, (n, 3))
    f = dbie.DBIEField.from_magnetogram(mag)
    opt = dbie.Options(precision=precision)
    gB0, glam = f.vjp(torch.from_numpy(xyz), torch.from_numpy(lam), torch.from_numpy(gB),
                      options=opt)
    torch.cuda.synchronize()
    gB0, glam = gB0.cpu().numpy(), glam.cpu().numpy()
    bd = oracle_boundary(mag)
    ref = oracle.vjp(bd, xyz.astype(np.float64), lam, gB)
    scale = vjp_scale(mag, xyz, lam, gB)
    tol = 1e-10 if precision == 1 else 1e-5
    assert np.all(np.abs(gB0 - ref) <= tol * scale + 1e-300), np.max(np.abs(gB0 - ref) / scale)
    _, _, dl = oracle.field(bd, xyz.astype(np.float64), lam)
    gl_ref = gB * dl
    frob = np.linalg.norm(glam - gl_ref) / np.linalg.norm(gl_ref)
    assert frob < (1e-10 if precision == 1 else 1e-4), frob
    # accumulate adds to the existing gradient
    acc = torch.ones((ny, nx, 3), dtype=torch.float64, device="cuda")
    f.vjp(torch.from_numpy(xyz), torch.from_numpy(lam), torch.from_numpy(gB), glam=False,
          options=opt, gB0=acc)
    torch.cuda.synchronize()
    assert np.allclose(acc.cpu().numpy() - 1.0, gB0, rtol=1e-12, atol=1e-12 * np.abs(gB0).max())
    f.close()


def test_adjoint_identity_on_gpu(dbie):
    """<gB, A B0> from the forward kernel equals <A^T gB, B0> from the adjoint kernel."""
    mag = random_mag(96, 80, 5)
    xyz, lam = random_points(mag, 1000, 6)
    gB = np.random.default_rng(7).normal(0, 1, (1000, 3))
    f = dbie.DBIEField.from_magnetogram(mag)
    for prec, tol in ((1, 1e-11), (0, 2e-6)):
        opt = dbie.Options(precision=prec, near_z=0.0)
        B = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), options=opt)["B"].cpu().numpy()
        gB0, _ = f.vjp(torch.from_numpy(xyz), torch.from_numpy(lam.astype(np.float64)),
                       torch.from_numpy(gB), glam=False, options=opt)
        B0 = np.stack([mag.Bx, mag.By, mag.Bz], -1).astype(np.float64)
        lhs, rhs = np.sum(gB * B), np.sum(gB0.cpu().numpy() * B0)
        assert abs(lhs - rhs) <= tol * (np.abs(gB) * np.abs(B)).sum(), (prec, lhs, rhs)
    f.close()


def test_autograd_function(dbie):
    """dbie_apply: gradients of L = sum |B|^2 w.r.t. B0 and lambda equal the oracle's."""
    mag = random_mag(40, 36, 8)
    xyz, lam = random_points(mag, 300, 9)
    f = dbie.DBIEField.from_magnetogram(mag)
    B0 = torch.from_numpy(np.stack([mag.Bx, mag.By, mag.Bz], -1)).cuda().requires_grad_(True)
    lam_t = torch.from_numpy(lam.astype(np.float64)).cuda().requires_grad_(True)
    opt = dbie.Options(precision=1)
    B = dbie.dbie_apply(f, B0, lam_t, torch.from_numpy(xyz).cuda(), opt)
    loss = (B * B).sum()
    loss.backward()
    bd = oracle_boundary(mag)
    Bref, _, dl = oracle.field(bd, xyz.astype(np.float64), lam.astype(np.float64))
    gB = 2 * Bref
    ref0 = oracle.vjp(bd, xyz.astype(np.float64), lam.astype(np.float64), gB)
    g0 = B0.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g0 - ref0) / np.linalg.norm(ref0) < 1e-6   # gradient returned as FP32
    gl = lam_t.grad.cpu().numpy()
    assert np.linalg.norm(gl - gB * dl) / np.linalg.norm(gB * dl) < 1e-9
    f.close()


def test_vjp_column_by_finite_difference(dbie):
    """B is linear in B0: a unit change of one pixel changes B by one column of A (FP64 form)."""
    mag = random_mag(30, 30, 12)
    xyz, lam = random_points(mag, 50, 13)
    gB = np.random.default_rng(14).normal(0, 1, (50, 3))
    f = dbie.DBIEField.from_magnetogram(mag)
    opt = dbie.Options(precision=1)
    gB0, _ = f.vjp(torch.from_numpy(xyz), torch.from_numpy(lam.astype(np.float64)),
                   torch.from_numpy(gB), glam=False, options=opt)
    gB0 = gB0.cpu().numpy()
    B_a = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), options=opt)["B"].cpu().numpy()
    for (jj, ii, p) in [(3, 4, 0), (15, 20, 1), (29, 0, 2)]:
        comps = [mag.Bx.copy(), mag.By.copy(), mag.Bz.copy()]
        comps[p][jj, ii] += np.float32(64.0)
        delta = float(comps[p][jj, ii]) - float((mag.Bx, mag.By, mag.Bz)[p][jj, ii])  # FP32 step
        f.set_boundary(*(torch.from_numpy(c) for c in comps))
        B_b = f.eval(torch.from_numpy(xyz), torch.from_numpy(lam), options=opt)["B"].cpu().numpy()
        col = (B_b[:, p] - B_a[:, p]) / delta
        assert abs(np.sum(gB[:, p] * col) - gB0[jj, ii, p]) <= 1e-8 * np.abs(gB[:, p] * col).sum()
    f.close()
