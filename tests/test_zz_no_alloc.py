"""dbie_eval_noalloc: the evaluation entry point that allocates nothing (its scratch is one fixed
array in the library's device image), for callers that may not allocate device memory while
they run.  Checked through the C ABI against dbie_eval on calls in a row (the array keeps the
previous call's contents, so every later call checks that the counters are cleared), and
directly against the FP64 oracle; one call is at the stated limits (256 x 256 pixels, 65,536
points), where the scratch layout is fullest.

Collected last on purpose: a failure here leaves the rest of the suite already run."""
import ctypes

import numpy as np
import pytest

import oracle
from gates import abs_scales, check_B, check_grad

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [(100, 90, 3000), (37, 61, 777), (256, 256, 65536)]   # (nx, ny, points)
ORACLE_SAMPLE = 256   # points per case compared with the oracle


def _case(seed, nx, ny, n):
    rng = np.random.default_rng(seed)
    comps = [rng.normal(0, 200, (ny, nx)).astype(np.float32) for _ in range(3)]
    xyz = np.stack([rng.uniform(-2, nx + 1, n), rng.uniform(-2, ny + 1, n),
                    rng.uniform(0.3, 25, n)], 1).astype(np.float32)
    lam = rng.uniform(-0.2, 0.2, (n, 3)).astype(np.float32)
    return comps, xyz, lam


class _Mag:
    def __init__(self, nx, ny, comps):
        self.nx, self.ny = nx, ny
        self.x0 = self.y0 = 0.0
        self.hx = self.hy = self.dA = 1.0
        self.Bx, self.By, self.Bz = comps


def test_noalloc_matches_dbie_eval_and_oracle_on_calls_in_a_row():
    import paper_1306_1122_gb300._native as N
    oracle.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed, (nx, ny, n) in enumerate(CASES):
        comps, xyz, lam = _case(seed, nx, ny, n)
        Bd = [torch.from_numpy(c).to(dev) for c in comps]
        X = torch.from_numpy(xyz).to(dev)
        L = torch.from_numpy(lam).to(dev)
        # existing entry point
        h = N.dbie_create(nx, ny, 0.0, 0.0, 1.0, 1.0, 1.0, *(P(c) for c in Bd), N.DBIE_MEM_DEVICE,
                          stream)
        B_ref = torch.empty((n, 3), dtype=torch.float64, device=dev)
        N.dbie_eval(h, n, P(X), P(L), None, N.DBIE_MEM_DEVICE, P(B_ref), None, None, None, stream)
        torch.cuda.synchronize()
        N.dbie_destroy(h)
        # the entry point that allocates nothing
        B = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev)
        N.dbie_eval_noalloc(nx, ny, 0.0, 0.0, 1.0, 1.0, 1.0, *(P(c) for c in Bd), n, P(X), P(L),
                            P(B), stream)
        torch.cuda.synchronize()
        got, ref = B.cpu().numpy(), B_ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        scale = np.abs(ref).max(axis=1, keepdims=True) * np.ones((1, 3))
        r = check_B(got, ref, scale)
        assert r["bad"].size == 0, r
        assert check_grad(got, ref, np.abs(ref).max())["ok"]
        # directly against the FP64 oracle (Eq. 16) on a seeded sample of the points
        pick = np.sort(np.random.default_rng(100 + seed).choice(n, min(n, ORACLE_SAMPLE),
                                                               replace=False))
        mag = _Mag(nx, ny, comps)
        bd = oracle.Boundary(oracle.Grid(nx, ny), *comps)
        xs, ls = xyz[pick].astype(np.float64), lam[pick].astype(np.float64)
        B_orc, _, _ = oracle.field(bd, xs, ls)
        sB, _ = abs_scales(mag, xs, ls)
        r = check_B(got[pick], B_orc, sB)
        assert r["bad"].size == 0, (nx, ny, n, r)


def test_noalloc_rejects_sizes_beyond_its_limits():
    import paper_1306_1122_gb300._native as N
    null = ctypes.c_void_p(1)
    st = N.lib.dbie_eval_noalloc(300, 300, 0.0, 0.0, 1.0, 1.0, 1.0, null, null, null, 10, null,
                                 null, null, None)
    assert st == N.DBIE_EINVAL
    st = N.lib.dbie_eval_noalloc(10, 10, 0.0, 0.0, 1.0, 1.0, 1.0, null, null, null, 70000, null,
                                 null, null, None)
    assert st == N.DBIE_EINVAL
