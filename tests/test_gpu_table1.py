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
