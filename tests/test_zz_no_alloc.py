"""dbie_eval_noalloc: the evaluation entry point that allocates nothing (its scratch is one fixed
array in the library's device image), for callers that may not allocate device memory while
they run.  Checked through the C ABI against dbie_eval on two calls in a row (the array keeps
the previous call's contents, so the second call checks that every counter is cleared).

Collected last on purpose: a failure here leaves the rest of the suite already run."""
import ctypes

import numpy as np
import pytest

from gates import check_B, check_grad

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _case(seed, nx, ny, n):
    rng = np.random.default_rng(seed)
    comps = [rng.normal(0, 200, (ny, nx)).astype(np.float32) for _ in range(3)]
    xyz = np.stack([rng.uniform(-2, nx + 1, n), rng.uniform(-2, ny + 1, n),
                    rng.uniform(0.3, 25, n)], 1).astype(np.float32)
    lam = rng.uniform(-0.2, 0.2, (n, 3)).astype(np.float32)
    return comps, xyz, lam


def test_noalloc_matches_dbie_eval_twice():
    import paper_1306_1122_gb300._native as N
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed, (nx, ny, n) in enumerate([(100, 90, 3000), (37, 61, 777)]):
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


def test_noalloc_rejects_sizes_beyond_its_limits():
    import paper_1306_1122_gb300._native as N
    null = ctypes.c_void_p(1)
    st = N.lib.dbie_eval_noalloc(300, 300, 0.0, 0.0, 1.0, 1.0, 1.0, null, null, null, 10, null,
                                 null, null, None)
    assert st == N.DBIE_EINVAL
    st = N.lib.dbie_eval_noalloc(10, 10, 0.0, 0.0, 1.0, 1.0, 1.0, null, null, null, 70000, null,
                                 null, null, None)
    assert st == N.DBIE_EINVAL
