"""GPU checks on the paper-shaped synthetic workloads (beyond the small parity cases).

  ar512   sheared quadrupolar active region 512 x 256: lambda search on the 32^3 sub-volume, then
          dB/dlambda and dL/dB0 for L = sum |B|^2 against central finite differences (FP64 form).
  ar1024  1024 x 512 active region with traced field-line samples and a grid: mixed against the
          FP64 GPU form on 20k points and against the CPU oracle on a 2k subsample; and at full
          size (6.3 M points) forward + adjoint with sampled checks and the adjoint identity.
  ar512   the full 256 x 128 x 64 volume with the lambda search, sampled against the oracle.
"""
import numpy as np
import pytest

import oracle
from gates import abs_scales, check_B, check_grad, oracle_boundary
from synth import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dbie():
    import paper_1306_1122_gb300 as d
    return d


def test_ar512_backward_against_finite_differences(dbie):
    w = workloads.ar512()
    m = w.mag
    sub = workloads.ar512_backward_subvolume(w)
    pts = torch.from_numpy(w.points[sub]).cuda()
    n = pts.shape[0]
    assert n == 32 ** 3
    f = dbie.DBIEField.from_magnetogram(m)
    s = f.solve(pts, dbie.Options(max_iter=15))
    lam = s["lam"]                                      # lambda*, fixed from here on
    mixed = dbie.Options()
    fp64 = dbie.Options(precision=1)
    ev = f.eval(pts, lam.float(), dlam=True, options=mixed)
    B, dBdl = ev["B"], ev["dBdlam"]
    gB = 2.0 * B                                        # L = sum |B|^2
    gB0, glam = f.vjp(pts, lam, gB, options=mixed)

    # dB/dlambda: central differences of the FP64 form on 2048 of the points
    idx = torch.arange(0, n, 16, device="cuda")
    lam32 = lam[idx].float()
    L_side = float(max(m.nx, m.ny))
    dl = torch.clamp(1e-3 * lam32.abs(), min=1e-3 / L_side)
    Bp = f.eval(pts[idx], lam32 + dl, options=fp64)["B"]
    Bm = f.eval(pts[idx], lam32 - dl, options=fp64)["B"]
    # the perturbed lambdas as the kernel sees them (FP32 inputs)
    h = ((lam32 + dl).double() - (lam32 - dl).double())
    fd = (Bp - Bm) / h
    r = check_grad(dBdl[idx].cpu().numpy(), fd.cpu().numpy(), fd.abs().max().item())
    assert r["ok"], r
    gl_fd = (gB[idx] * fd)
    rl = check_grad(glam[idx].cpu().numpy(), gl_fd.cpu().numpy(), gl_fd.abs().max().item())
    assert rl["ok"], rl

    # dL/dB0 at 64 random pixels: B is linear in B0, so L(B0 + d e_k) and L(B0 - d e_k) follow
    # from the FP64 field and the FP64 response to a single unit pixel (one-pixel magnetogram
    # at the same position), and the central difference of the quadratic L is exact.
    B64 = f.eval(pts, lam.float(), options=fp64)["B"]
    rng = np.random.default_rng(31)
    pix = rng.choice(m.npix, 64, replace=False)
    comp = rng.integers(0, 3, 64)
    fd0, got = [], []
    for k, p in zip(pix, comp):
        j, i = divmod(int(k), m.nx)
        comps = [np.full((1, 1), 1.0 if c == p else 0.0, np.float32) for c in range(3)]
        col_field = dbie.DBIEField(*comps, x0=m.x0 + i * m.hx, y0=m.y0 + j * m.hy, hx=m.hx,
                                   hy=m.hy, pixel_area=m.dA)
        col = col_field.eval(pts, lam.float(), options=fp64)["B"][:, p]
        col_field.close()
        d = 1.0
        Lp = ((B64[:, p] + d * col) ** 2).sum()
        Lm = ((B64[:, p] - d * col) ** 2).sum()
        fd0.append(float((Lp - Lm) / (2 * d)))
        got.append(float(gB0[j, i, p]))
    fd0, got = np.array(fd0), np.array(got)
    assert np.all(np.abs(got - fd0) <= 1e-4 * np.abs(fd0).max()), np.abs(got - fd0).max()
    assert np.linalg.norm(got - fd0) / np.linalg.norm(fd0) < 1e-5
    f.close()


def test_ar1024_mixed_against_fp64_form_and_oracle(dbie):
    w = workloads.ar1024(nsamples=18000, grid=True, seed=5)
    m = w.mag
    rng = np.random.default_rng(8)
    pick = np.concatenate([np.arange(18000), 18000 + rng.choice(len(w.points) - 18000, 2000,
                                                                  replace=False)])
    pts = w.points[pick]
    lam = rng.uniform(0.0, 0.02, (len(pts), 3)).astype(np.float32)
    f = dbie.DBIEField.from_magnetogram(m)
    P, L = torch.from_numpy(pts).cuda(), torch.from_numpy(lam).cuda()
    mix = f.eval(P, L, grad=True)
    ref = f.eval(P, L, grad=True, options=dbie.Options(precision=1))
    torch.cuda.synchronize()
    Bm, Br = mix["B"].cpu().numpy(), ref["B"].cpu().numpy()
    # mixed vs FP64 GPU form: the gate uses |B| itself as the sum scale proxy for the floor
    rel = np.linalg.norm(Bm - Br, axis=1) / np.linalg.norm(Br, axis=1)
    assert np.median(rel) < 1e-6 and np.percentile(rel, 99) < 1e-5, (np.median(rel), rel.max())
    assert np.linalg.norm(Bm - Br) / np.linalg.norm(Br) < 1e-5
    assert check_grad(mix["gradB"].cpu().numpy(), ref["gradB"].cpu().numpy(),
                      np.abs(ref["gradB"].cpu().numpy()).max())["ok"]
    # the CPU oracle on a subsample (FP64, 524,288 pixels per point)
    sub = rng.choice(len(pts), 500, replace=False)
    Bo, _, _ = oracle.field(oracle_boundary(m), pts[sub].astype(np.float64),
                            lam[sub].astype(np.float64))
    assert np.all(np.abs(Br[sub] - Bo) <= 1e-10 * (np.abs(Bo) + np.abs(Bo).max() * 1e-3))
    rb = check_B(Bm[sub], Bo, np.zeros_like(Bo))
    assert rb["frob"] < 1e-5, rb
    f.close()


def test_ll128_metrics_match_oracle_solution(dbie):
    """Accuracy context on the 128^2 Low & Lou case: the five field-comparison metrics of the
    GPU solution against the analytic field agree with those of the oracle's solution (FP64 CPU)
    on the same points, and B at the GPU's lambda matches the oracle's field there."""
    from oracle.metrics import field_metrics
    w = workloads.ll128(with_truth=True)
    idx = np.sort(np.random.default_rng(12).choice(len(w.points), 768, replace=False))
    pts = w.points[idx]
    f = dbie.DBIEField.from_magnetogram(w.mag)
    r = f.solve(torch.from_numpy(pts).cuda(), dbie.Options())
    torch.cuda.synchronize()
    B_gpu, lam_gpu = r["B"].cpu().numpy(), r["lam"].cpu().numpy()
    bd = oracle_boundary(w.mag)
    ref = oracle.solve(bd, pts.astype(np.float64), oracle.Options())
    mg = field_metrics(B_gpu, w.truth[idx])
    mo = field_metrics(ref["B"], w.truth[idx])
    for k in mg:
        assert abs(mg[k] - mo[k]) < 2e-2 * max(1.0, abs(mo[k])), (k, mg[k], mo[k])
    Bo, _, _ = oracle.field(bd, pts.astype(np.float64), lam_gpu)
    sB, _ = abs_scales(w.mag, pts, lam_gpu)
    assert check_B(B_gpu, Bo, sB)["bad"].size == 0
    # lambda = 0 (potential) field is worse than the searched one on C_vec (the search helps)
    B0 = f.eval(torch.from_numpy(pts).cuda(), torch.zeros((len(pts), 3)).cuda())["B"]
    m0 = field_metrics(B0.cpu().numpy(), w.truth[idx])
    print("metrics searched", mg, "oracle", mo, "lambda=0", m0)
    f.close()


def test_ar1024_full_size_forward_backward(dbie):
    """All 6,291,456 points of the 1024 x 512 workload (4,194,304 traced samples + the 128^3
    grid), mixed precision, forward at a fixed seeded lambda and the adjoint: sampled outputs
    against the FP64 GPU form (20k points) and the oracle (300 points); the adjoint identity
    <gB, A B0> = <A^T gB, B0> over the whole set (a property at any size)."""
    w = workloads.ar1024()
    m = w.mag
    n = len(w.points)
    assert n == 4_194_304 + 128 ** 3
    rng = np.random.default_rng(9)
    lam = rng.uniform(0.0, 0.02, (n, 3)).astype(np.float32)
    f = dbie.DBIEField.from_magnetogram(m)
    f.autotune()
    P, L = torch.from_numpy(w.points).cuda(), torch.from_numpy(lam).cuda()
    B = f.eval(P, L)["B"]
    gB = torch.from_numpy(rng.normal(size=(n, 3))).cuda()
    gB0, _ = f.vjp(P, L.double(), gB, glam=False)
    torch.cuda.synchronize()
    B0 = torch.from_numpy(np.stack([m.Bx, m.By, m.Bz], -1).astype(np.float64)).cuda()
    lhs = float((gB * B).sum())
    rhs = float((gB0 * B0).sum())
    scale = float((gB.abs() * B.abs()).sum())
    assert abs(lhs - rhs) <= 1e-6 * scale, (lhs, rhs, scale)
    sub = torch.from_numpy(np.sort(rng.choice(n, 20000, replace=False))).cuda()
    ref = f.eval(P[sub], L[sub], options=dbie.Options(precision=1))["B"]
    Bm = B[sub].cpu().numpy()
    Br = ref.cpu().numpy()
    rel = np.linalg.norm(Bm - Br, axis=1) / np.linalg.norm(Br, axis=1)
    assert np.median(rel) < 1e-6 and np.percentile(rel, 99) < 1e-5, (np.median(rel), rel.max())
    assert np.linalg.norm(Bm - Br) / np.linalg.norm(Br) < 1e-5
    few = np.sort(rng.choice(n, 300, replace=False))
    Bo, _, _ = oracle.field(oracle_boundary(m), w.points[few].astype(np.float64),
                            lam[few].astype(np.float64))
    assert check_B(B[torch.from_numpy(few).cuda()].cpu().numpy(), Bo,
                   np.zeros_like(Bo))["frob"] < 1e-5
    f.close()


def test_ar512_full_volume_solve(dbie):
    """The 256 x 128 x 64 volume (2,097,152 points) over the 512 x 256 boundary with the lambda
    search (10 simplex iterations): B at the GPU's lambda against the oracle on 200 sampled
    points, and every point ends with a finite lambda and status."""
    w = workloads.ar512()
    n = len(w.points)
    assert n == 256 * 128 * 64
    f = dbie.DBIEField.from_magnetogram(w.mag)
    f.autotune()
    r = f.solve(torch.from_numpy(w.points).cuda(), dbie.Options(max_iter=10))
    torch.cuda.synchronize()
    lam = r["lam"].cpu().numpy()
    assert np.all(np.isfinite(lam)) and np.all(np.isfinite(r["B"].cpu().numpy()))
    st = r["status"].cpu().numpy()
    assert set(np.unique(st)) <= {0, 1}
    rng = np.random.default_rng(10)
    few = np.sort(rng.choice(n, 200, replace=False))
    Bo, _, _ = oracle.field(oracle_boundary(w.mag), w.points[few].astype(np.float64), lam[few])
    sB, _ = abs_scales(w.mag, w.points[few], lam[few])
    rb = check_B(r["B"].cpu().numpy()[few], Bo, sB)
    assert rb["bad"].size == 0, rb
    f.close()
