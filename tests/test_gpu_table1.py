"""The paper's Table 1 case on the GPU: Low & Lou (1990) n=3, m=1, l=0.3, Phi=4 pi/5 on a
192 x 192 boundary, lambda searched at every pixel of the central 64 x 64 x 64 test region, and
the five metrics of Schrijver et al. (2006) against the analytic field over the whole region (the
z = 0 layer being the boundary data itself).

Context, not parity.  What is checked: at lambda = 0 (no search) the quadrature of this setup
reproduces the paper's "boundary integral method, no iteration" row, which pins the test
configuration (box scale, region, truncation).  The searched rows depend on readings the paper
leaves open (the objective's combination and thresholds, Delta V / Delta sigma, the initial
simplex) and are printed next to the paper's DBIE row (tests/golden/table1_metrics.txt) with
sanity bounds only."""
import os

import numpy as np
import pytest

from oracle.metrics import field_metrics
from synth import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_metrics.txt")


def paper_rows():
    rows = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, *vals = line.split()
            rows[name] = dict(zip(("C_vec", "C_cs", "E_n", "E_m", "eps"), map(float, vals)))
    return rows


def test_golden_rows_parse():
    rows = paper_rows()
    assert rows["present_dbie"]["C_vec"] == 0.99 and rows["present_dbie"]["E_m"] == -0.53


@pytest.fixture(scope="module")
def dbie():
    import paper_1306_1122_gb300 as d
    return d


def _metrics(w, B):
    bottom_B = np.stack([w.mag.Bx, w.mag.By, w.mag.Bz], -1)[
        w.meta["bottom"][:, 1].astype(int), w.meta["bottom"][:, 0].astype(int)]
    allB = np.concatenate([bottom_B.astype(np.float64), B])
    allb = np.concatenate([w.meta["bottom_truth"], w.truth])
    return field_metrics(allB, allb)


def test_table1_reproduction(dbie):
    w = workloads.table1()
    pts = torch.from_numpy(w.points).cuda()
    f = dbie.DBIEField.from_magnetogram(w.mag)
    f.autotune()
    out = {}
    r0 = f.eval(pts, torch.zeros_like(pts))
    out["lambda = 0"] = _metrics(w, r0["B"].cpu().numpy())
    for name, opt in (("simplex (paper)", dbie.Options()),
                      ("quasi-Newton", dbie.Options(method=1))):
        r = f.solve(pts, opt)
        torch.cuda.synchronize()
        out[name] = _metrics(w, r["B"].cpu().numpy())
    # the same search with the exact near-field integration for z <= 2 px
    f.set_quadrature(dbie.QUAD_PIXEL_EXACT)
    r = f.solve(pts, dbie.Options())
    torch.cuda.synchronize()
    out["simplex, exact near field"] = _metrics(w, r["B"].cpu().numpy())
    f.close()
    # the same field on the 193-node grid, nine-node elements with 4 x 4 Gauss points
    w9 = workloads.table1(193)
    f9 = dbie.DBIEField.from_magnetogram(w9.mag)
    f9.set_quadrature(4)
    r9 = f9.solve(torch.from_numpy(w9.points).cuda())
    torch.cuda.synchronize()
    B9 = r9["B"].cpu().numpy()
    f9.close()
    out["simplex, Eq. 15 elements"] = _metrics(w, B9)
    paper = paper_rows()
    print("\n%-28s %7s %7s %7s %7s %7s" % ("", "C_vec", "C_cs", "E_n", "E_m", "eps"))
    for name, m in list(out.items()) + [("paper: present DBIE", paper["present_dbie"]),
                                        ("paper: BIE, no iteration",
                                         paper["boundary_integral_no_iteration"])]:
        print("%-28s %7.3f %7.3f %7.3f %7.3f %7.3f" % (name, m["C_vec"], m["C_cs"], m["E_n"],
                                                      m["E_m"], m["eps"]))
    nb, z0 = paper["boundary_integral_no_iteration"], out["lambda = 0"]
    assert abs(z0["C_vec"] - nb["C_vec"]) < 0.01 and abs(z0["C_cs"] - nb["C_cs"]) < 0.01
    assert abs(z0["eps"] - nb["eps"]) < 0.03 and abs(z0["E_n"] - nb["E_n"]) < 0.1
    assert z0["E_m"] < -5 and nb["E_m"] < -5          # both dominated by the upper layers
    for name in ("simplex (paper)", "simplex, Eq. 15 elements", "simplex, exact near field"):
        m = out[name]
        assert m["C_vec"] > 0.9 and 0.8 < m["eps"] < 1.4, (name, m)


def test_table1_search_follows_oracle_on_subsample(dbie):
    """The searched Table 1 field against the oracle on a seeded 96-point subsample of the
    258,048 points: the certified mixed search (the default) takes the oracle's step sequence on
    >= 95 % of them, lambda agrees to 1e-4 max(|lambda|, 1/L) there, and B at the GPU's own
    lambda meets the B gate against the oracle's field."""
    import oracle
    from gates import abs_scales, check_B, oracle_boundary
    w = workloads.table1()
    idx = np.sort(np.random.default_rng(1).choice(len(w.points), 96, replace=False))
    pts = w.points[idx]
    f = dbie.DBIEField.from_magnetogram(w.mag)
    r = f.solve(torch.from_numpy(pts).cuda(), codes=50)
    torch.cuda.synchronize()
    f.close()
    got = {k: v.cpu().numpy() for k, v in r.items()}
    codes = [bytes(row).rstrip(b"\0").decode() for row in got["codes"]]
    ref = oracle.solve(oracle_boundary(w.mag), pts.astype(np.float64), oracle.Options())
    same = np.array([a == b for a, b in zip(codes, ref["codes"])])
    L = float(max(w.mag.nx, w.mag.ny))
    lam_ok = np.all(np.abs(got["lam"] - ref["lam"]) <=
                    1e-4 * np.maximum(np.abs(ref["lam"]), 1.0 / L), axis=1)
    print(f"table 1 subsample: oracle step sequence on {same.mean():.3f}, lambda within 1e-4 on "
          f"{lam_ok[same].mean():.3f} of those")
    assert same.mean() >= 0.95
    assert lam_ok[same].mean() >= 0.99
    B, _, _ = oracle.field(oracle_boundary(w.mag), pts.astype(np.float64), got["lam"])
    sB, _ = abs_scales(w.mag, pts, got["lam"])
    assert check_B(got["B"], B, sB)["bad"].size == 0


def test_table1_upper_layers_decay_too_slowly(dbie):
    """Why the searched field does not reach the paper's DBIE row, as checked numbers.  The
    192 x 192 boundary is flux-balanced (net vertical flux 6e-5 of the unsigned flux), and next to
    it every field built from it by the Eq. 16 quadrature agrees with the analytic field (C_vec
    > 0.98 at z = 1 px).  But the reconstruction decays with height far more slowly than the Low &
    Lou n = 3 field: between z = 8 and 63 px the layer-mean |B| falls with a log-slope (against
    height above the source) of about -1 to -1.7 where the analytic field falls with -2.8 to -4.4,
    so the energy ratio per layer (eps) climbs to about 10^3 at the top and the direction is lost
    (C_vec ~0.3).  Those layers dominate the volume's E'_n and E'_m.  The search minimises f and g
    (Eqs. 8, 9), which are invariant to a rescaling of B, and leaves the excess in place.  Layer
    table printed for the record."""
    w = workloads.table1()
    bz = w.mag.Bz.astype(np.float64)
    net_frac = abs(bz.sum()) / np.abs(bz).sum()
    pts = torch.from_numpy(w.points).cuda()
    f = dbie.DBIEField.from_magnetogram(w.mag)
    B0 = f.eval(pts, torch.zeros_like(pts))["B"].cpu().numpy()
    Bs = f.solve(pts)["B"].cpu().numpy()
    torch.cuda.synchronize()
    f.close()
    z = w.points[:, 2]
    print(f"\nnet vertical flux / unsigned flux of the boundary: {net_frac:.1e}")
    print("%4s %8s %9s %8s %9s %9s %9s %9s" % ("z", "Cvec_0", "eps_0", "Cvec_s", "eps_s",
                                               "|b|", "|B_0|", "|B_s|"))
    rows, mags = {}, {}
    for zz in (1, 2, 4, 8, 16, 32, 63):
        sel = z == zz
        m0 = field_metrics(B0[sel], w.truth[sel])
        ms = field_metrics(Bs[sel], w.truth[sel])
        mags[zz] = [np.linalg.norm(X[sel], axis=1).mean() for X in (w.truth, B0, Bs)]
        rows[zz] = (m0, ms)
        print("%4d %8.3f %9.3f %8.3f %9.3f %9.3g %9.3g %9.3g" % (
            zz, m0["C_vec"], m0["eps"], ms["C_vec"], ms["eps"], *mags[zz]))
    assert net_frac < 1e-3
    for m in rows[1]:
        assert m["C_vec"] > 0.98
    depth = 0.3 * 32.0                        # the source's depth in pixels (l = 0.3 box units)
    span = np.log((63 + depth) / (8 + depth))
    slope = [np.log(mags[63][k] / mags[8][k]) / span for k in range(3)]
    print("log-slope of the layer-mean |field| from z = 8 to 63 px: analytic %.2f, lambda = 0 "
          "%.2f, searched %.2f" % tuple(slope))
    for k in (0, 1):
        eps = [rows[zz][k]["eps"] for zz in (8, 16, 32, 63)]
        assert all(b > a for a, b in zip(eps, eps[1:])), eps      # growing excess with height
        assert eps[-1] > 100
        assert rows[63][k]["C_vec"] < 0.5
        assert slope[k + 1] > slope[0] + 1.5                      # decays much more slowly
